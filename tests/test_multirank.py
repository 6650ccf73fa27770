"""The benchmark's multi-GPU aggregation (one process per GPU, independent poses, no data-path
collective): time is the maximum over ranks, work the sum.  Run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0 + 5.0 * rank, 1.0 * rank]
    work = [1000.0 * (rank + 1), 7.0]
    mx, sm = bench.over_ranks(dist, world, ms, work)
    q.put((rank, mx, sm))
    dist.destroy_process_group()


def test_over_ranks_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm in res:
        assert mx == [15.0, 1.0]          # max over ranks
        assert sm == [3000.0, 14.0]       # sum over ranks


def test_over_ranks_single_rank_is_identity():
    import bench
    assert bench.over_ranks(None, 1, [2.5], [3, 4]) == ([2.5], [3.0, 4.0])
