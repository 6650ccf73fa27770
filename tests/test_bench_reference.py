"""The oracle arm of bench.py (`--impl reference`) on the host: rank 0 prints one JSON line with the
contract's keys (the oracle timed on a bounded sample of the benchmark workload, e2e with no transfers),
and any other rank of a multi-process launch exits 0 without work or output."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = run({"RANK": "0", "WORLD_SIZE": "1"}, "--steps", "1", "--warmup", "0", "--ref-rays", "256")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("clutter")


def test_reference_arm_other_ranks_do_no_work():
    r = run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "0", "--ref-rays", "256")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
