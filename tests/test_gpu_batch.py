"""Batched form (many poses over several scenes in one launch per stage, recorded as a CUDA graph).

Each job's spectra must equal the single-pose path on the same inputs (which the parity tests pin
to the oracle) up to the order of the float32 chunk sums, and match the oracle directly within the
spectra tolerance; a graph replay after the poses are updated in place must give the new poses'
spectra; the autotuner must return launch shapes that give the same results."""
import dataclasses
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4        # against the oracle
TOL_SINGLE = 2e-5  # against the single-pose path (same path sets; only the chunking of the sums differs)


def rel_l2(a, b):
    nb = np.linalg.norm(b.ravel())
    if nb == 0:
        return float(np.linalg.norm(a.ravel()))
    return float(np.linalg.norm((a - b).ravel()) / nb)


@pytest.fixture(scope="module")
def st():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st_
    return st_


def unit_quat(rng):
    q = rng.normal(size=4)
    return (q / np.linalg.norm(q)).astype(np.float32)


def make_case(st, ctx, seed=11, n_scenes=3, poses=3, diffraction=True):
    rng = np.random.default_rng(seed)
    wls, specs = synth.batched_poses(seed=505 + seed, n_scenes=n_scenes, poses_per_scene=poses, tri_lo=2e3, tri_hi=2e4)
    scenes = []
    for wl in wls:
        sc = st.Scene(ctx, wl.verts, wl.tris, wl.tri_mat, wl.tri_obj)
        sc.set_materials(wl.band_hz, wl.k_band, wl.beta_band, wl.diff_band)
        sc.precompute(st.curv_params(sample_budget=50_000))
        scenes.append(sc)
    jobs, wl_jobs = [], []
    for i, sp in enumerate(specs):
        wl = wls[sp["scene"]]
        n = int(rng.integers(700, 4000))
        M = min(sp["n_mics"], 12)
        F = int(rng.integers(17, 200))
        fov = float(np.float32(math.pi if i % 2 == 0 else math.pi / 2))
        wj = dataclasses.replace(wl, emitter=sp["emitter"], emitter_quat=unit_quat(rng),
                                 dirs=synth.fibonacci_directions(n), mics=sp["mics"][:M].astype(np.float32), n_bins=F,
                                 bounces=sp["bounces"], max_distance=60.0, diffraction=diffraction, fov_half=fov)
        jobs.append(st.BatchJob(scenes[sp["scene"]], wj.emitter, wj.emitter_quat, wj.dirs, wj.mics, F, wl.f_lo,
                                wl.f_hi, wj.bounces, pose_index=sp["pose_index"], fov_half=fov))
        wl_jobs.append(wj)
    return scenes, jobs, wl_jobs


def single(st, ctx, sc, wj, pose, **kw):
    ctx.set_frequencies(wj.n_bins, wj.f_lo, wj.f_hi)
    ctx.set_emitter(wj.emitter, wj.emitter_quat, wj.dirs, None, wj.fov_half)
    ctx.set_receivers(wj.mics)
    p = st.sim_params(max_bounces=wj.bounces, max_distance=60.0, pose_index=pose, **kw)
    return ctx.simulate(sc, p).cpu().numpy()


def test_batch_equals_single_pose_and_oracle(st):
    import oracle
    ctx = st.Context(0)
    scenes, jobs, wl_jobs = make_case(st, ctx)
    p = st.sim_params(max_distance=60.0)
    outs = [o.cpu().numpy() for o in ctx.simulate_batch(jobs, p)]
    n_nonzero = 0
    for j, (job, wj) in enumerate(zip(jobs, wl_jobs)):
        ref = single(st, ctx, job.scene, wj, job.job.pose_index)
        for c in range(3):
            assert rel_l2(outs[j][c], ref[c]) <= TOL_SINGLE, (j, c, rel_l2(outs[j][c], ref[c]))
        n_nonzero += int(np.abs(outs[j][0]).sum() > 0) + int(np.abs(outs[j][1]).sum() > 0)
    assert n_nonzero >= len(jobs)
    # the oracle on two jobs (all three components)
    for j in (0, len(jobs) - 1):
        wj = wl_jobs[j]
        o = oracle.simulate(wj, curv=dict(budget=50_000), pose=jobs[j].job.pose_index)
        for c in range(3):
            assert rel_l2(outs[j][c], o["spectra"][c]) <= TOL, (j, c, rel_l2(outs[j][c], o["spectra"][c]))


def test_batch_graph_replay_after_pose_update(st):
    ctx = st.Context(0)
    scenes, jobs, wl_jobs = make_case(st, ctx, seed=12, n_scenes=2, poses=3)
    p = st.sim_params(max_distance=60.0)
    first = [o.cpu().numpy().copy() for o in ctx.simulate_batch(jobs, p)]
    again = [o.cpu().numpy().copy() for o in ctx.simulate_batch(jobs, p)]  # replay, same poses
    for a, b in zip(first, again):
        assert np.array_equal(a, b)  # deterministic reductions
    rng = np.random.default_rng(99)
    new_wl = []
    for job, wj in zip(jobs, wl_jobs):
        shift = rng.uniform(-0.5, 0.5, size=3).astype(np.float32)
        shift[2] *= 0.2
        e = (wj.emitter + shift).astype(np.float32)
        q = unit_quat(rng)
        m = (wj.mics + shift).astype(np.float32)
        job.set_pose(emitter=e, emitter_quat=q, mics=m)
        new_wl.append(dataclasses.replace(wj, emitter=e, emitter_quat=q, mics=m))
    outs = [o.cpu().numpy() for o in ctx.simulate_batch(jobs, p)]  # replay with the new poses
    changed = 0
    for j, (job, wj) in enumerate(zip(jobs, new_wl)):
        ref = single(st, ctx, job.scene, wj, job.job.pose_index)
        for c in range(3):
            assert rel_l2(outs[j][c], ref[c]) <= TOL_SINGLE, (j, c)
        changed += int(not np.array_equal(outs[j], first[j]))
    assert changed == len(jobs)


def test_batch_components_and_empty_jobs(st):
    """Specular only, a job with no rays, and single-mic / single-bin jobs."""
    ctx = st.Context(0)
    scenes, jobs, wl_jobs = make_case(st, ctx, seed=13, n_scenes=1, poses=2, diffraction=False)
    wl0 = wl_jobs[0]
    sc = jobs[0].scene
    extra = [
        (dataclasses.replace(wl0, dirs=np.zeros((0, 3), np.float32), n_bins=5), 0),
        (dataclasses.replace(wl0, mics=wl0.mics[:1].copy(), n_bins=1, bounces=1), 1),
    ]
    for wj, pose in extra:
        jobs.append(st.BatchJob(sc, wj.emitter, wj.emitter_quat, wj.dirs, wj.mics, wj.n_bins, wj.f_lo, wj.f_hi,
                                wj.bounces, pose_index=pose, fov_half=wj.fov_half))
        wl_jobs.append(wj)
    for comps in (st.ST_COMP_SPECULAR, st.ST_COMP_SPECULAR | st.ST_COMP_DIRECT):
        p = st.sim_params(max_distance=60.0, components=comps)
        outs = [o.cpu().numpy() for o in ctx.simulate_batch(jobs, p)]
        for j, (job, wj) in enumerate(zip(jobs, wl_jobs)):
            if wj.dirs.shape[0] == 0:
                assert np.all(outs[j][0] == 0) and np.all(outs[j][1] == 0)
                continue
            ref = single(st, ctx, job.scene, wj, job.job.pose_index, components=comps)
            for c in range(3):
                assert rel_l2(outs[j][c], ref[c]) <= TOL_SINGLE, (comps, j, c)


def test_several_emitters_in_one_call(st):
    """Three emitters sending the same ray set into one scene towards one array (Context.simulate_emitters):
    each emitter's specular, diffraction and direct spectra against the oracle run for that emitter alone
    (same diffraction samples: one pose index), then a replay with every emitter moved and turned."""
    import oracle
    rng = np.random.default_rng(21)
    wl = synth.clutter(seed=203, target_tris=20_000, n_rays=20_000, bounces=3, n_mics=8, n_bins=96)
    wl = dataclasses.replace(wl, max_distance=60.0, fov_half=float(np.float32(math.pi / 2)))
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=100_000))
    p = st.sim_params(max_distance=wl.max_distance)
    for call in range(2):
        E = (wl.emitter + rng.uniform(-1.5, 1.5, (3, 3)) * np.array([1.0, 1.0, 0.2])).astype(np.float32)
        Q = np.stack([unit_quat(rng) for _ in range(3)])
        out = ctx.simulate_emitters(sc, E, Q, wl.dirs, wl.mics, wl.n_bins, wl.f_lo, wl.f_hi, wl.bounces, p,
                                    pose_index=4, fov_half=wl.fov_half).cpu().numpy()
        assert out.shape == (3, 3, len(wl.mics), wl.n_bins)
        for e in range(3):
            o = oracle.simulate(dataclasses.replace(wl, emitter=E[e], emitter_quat=Q[e]),
                                curv=dict(budget=100_000), pose=4)
            for c in range(3):
                assert np.abs(o["spectra"][c]).sum() > 0
                assert rel_l2(out[e, c], o["spectra"][c]) <= TOL, (call, e, c, rel_l2(out[e, c], o["spectra"][c]))
        assert not np.array_equal(out[0], out[1])


def test_batch_per_microphone_receiver_test(st):
    """The per-microphone receiver test in the batched form: three poses in the clutter scene with
    microphones spread over 16 x 16 m (hits that some microphones see and others do not; the first job
    with two microphones, the narrow accumulator) against the single-pose per-microphone path (2e-5), the
    first job against the oracle (1e-4), and the specular spectra differ from the reference-point test's."""
    import oracle
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=8_000, bounces=3, n_mics=12, n_bins=48)
    wl = dataclasses.replace(wl, max_distance=60.0)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=50_000))
    rng = np.random.default_rng(17)
    jobs, wl_jobs = [], []
    for k in range(3):
        M = 2 if k == 0 else 12
        mics = np.stack([rng.uniform(2, 18, M), rng.uniform(2, 18, M), rng.uniform(0.3, 2.0, M)], 1).astype(np.float32)
        e = (wl.emitter + rng.uniform(-0.3, 0.3, 3) * np.array([1.0, 1.0, 0.2])).astype(np.float32)
        wj = dataclasses.replace(wl, mics=mics, emitter=e, emitter_quat=unit_quat(rng))
        jobs.append(st.BatchJob(sc, wj.emitter, wj.emitter_quat, wj.dirs, wj.mics, wj.n_bins, wj.f_lo, wj.f_hi,
                                wj.bounces, pose_index=k, fov_half=wj.fov_half))
        wl_jobs.append(wj)
    p = st.sim_params(max_distance=60.0, los_mode=st.ST_LOS_PER_MIC)
    outs = [o.cpu().numpy().copy() for o in ctx.simulate_batch(jobs, p)]
    ref_mode = [o.cpu().numpy().copy() for o in ctx.simulate_batch(jobs, st.sim_params(max_distance=60.0))]
    again = [o.cpu().numpy().copy() for o in ctx.simulate_batch(jobs, p)]  # recorded again for this mode
    for j, (job, wj) in enumerate(zip(jobs, wl_jobs)):
        assert np.array_equal(again[j], outs[j])
        ref = single(st, ctx, sc, wj, j, los_mode=st.ST_LOS_PER_MIC)
        for c in range(3):
            assert rel_l2(outs[j][c], ref[c]) <= TOL_SINGLE, (j, c, rel_l2(outs[j][c], ref[c]))
        assert rel_l2(outs[j][0], ref_mode[j][0]) > 1e-3, j  # the masks change the specular spectra
    o = oracle.simulate(wl_jobs[0], curv=dict(budget=50_000), pose=0, los_mode=1)
    m0 = o["rec"]["mask"][o["rec"]["tri"] >= 0]
    assert np.sum(m0 == 1) + np.sum(m0 == 2) > 100  # records that reach one microphone of the two
    for c in range(3):
        assert rel_l2(outs[0][c], o["spectra"][c]) <= TOL, (c, rel_l2(outs[0][c], o["spectra"][c]))


def test_autotune_shapes_give_same_results(st):
    ctx = st.Context(0)
    scenes, jobs, wl_jobs = make_case(st, ctx, seed=14, n_scenes=1, poses=2)
    p = st.sim_params(max_distance=60.0)
    base = [o.cpu().numpy().copy() for o in ctx.simulate_batch(jobs, p)]
    t = ctx.autotune(jobs[0], p)
    assert t.rays_per_block in (64, 128, 256)
    assert 1 <= t.mic_pairs_per_cta <= 16 and 32 <= t.smem_kb <= 160
    assert t.bins_per_thread in (8, 16) and t.stack_depth in (0, 48, 24) and t.refill_lanes in (0, 12, 20, 32)
    tuned = [o.cpu().numpy() for o in ctx.simulate_batch(jobs, p, t)]
    for a, b in zip(tuned, base):
        for c in range(3):
            assert rel_l2(a[c], b[c]) <= TOL_SINGLE


def test_batch_stack_restarts_keep_results_exact():
    """The batched kernels take the stack limit of their tune: with 2-entry stacks (most queries restart
    stackless from the root) every job's spectra equal those of the default stack bit for bit."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st
    wl = synth.clutter(seed=212, target_tris=6000, n_rays=3000, bounces=3, n_mics=4, n_bins=32)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=20_000))
    jobs = [st.BatchJob(sc, wl.emitter + np.float32(0.1 * i), wl.emitter_quat, wl.dirs, wl.mics, wl.n_bins, wl.f_lo,
                        wl.f_hi, wl.bounces, pose_index=i) for i in range(3)]
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    ctx.simulate_batch(jobs, p)
    ref = [j.out.cpu().numpy().copy() for j in jobs]
    ctx.simulate_batch(jobs, p, tune=st.Tune(0, 0, 0, 2))
    for j, r in zip(jobs, ref):
        assert np.array_equal(j.out.cpu().numpy(), r)


def test_single_pose_tuning_parameters(st):
    """Each tuned parameter of the single-pose path: the stack depth and the lane-refill threshold change
    only the order in which queries are traced (spectra bit-identical), the accumulator's 8 or 16 bins per
    thread only the order of its float32 sums (within the single-pose tolerance)."""
    wl = synth.clutter(seed=214, target_tris=6000, n_rays=4000, bounces=3, n_mics=8, n_bins=100)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=20_000))
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    ref = ctx.simulate(sc, p).cpu().numpy()
    for kw in (dict(refill_lanes=8), dict(refill_lanes=32), dict(stack_depth=24, refill_lanes=20)):
        ctx.set_tune(**kw)
        assert np.array_equal(ctx.simulate(sc, p).cpu().numpy(), ref), kw
    ctx.set_tune(bins_per_thread=8)
    S8 = ctx.simulate(sc, p).cpu().numpy()
    for c in range(3):
        assert rel_l2(S8[c], ref[c]) <= TOL_SINGLE
    with pytest.raises(st.SonotraceError):
        ctx.set_tune(bins_per_thread=4)


def test_batch_directivity(st):
    """Directional jobs in one batch (Sec. III-F) over a leaf-disc scene: the bat's two ears with ear tables
    and the piston emitter table (narrow accumulator), an 8-microphone array with receiver tables, random
    orientations and an emitter table (general accumulator, launched on its own), an emitter table alone
    (the work queue) and an omni job.  Every job against the single-pose path with the same tables (2e-5),
    the two-ear job against the oracle (1e-4, all three components)."""
    import oracle
    wl = synth.vegetation(seed=313, target_tris=30_000, n_rays=8_000, bounces=3, n_bins=96, leaves_per_mesh=64)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=100_000))
    rng = np.random.default_rng(77)
    fov = float(np.float32(math.pi / 2))

    def quats(n):
        return np.stack([unit_quat(rng) for _ in range(n)])

    specs = []
    # (emitter table, mic quats, mic tables, mics, F)
    specs.append((wl.emitter_table, wl.mic_quats, wl.mic_tables, wl.mics, wl.n_bins))
    F1 = 64
    m8 = (wl.mics[:1] + rng.uniform(-0.05, 0.05, (8, 3))).astype(np.float32)
    specs.append((synth.piston_table(0.002, np.linspace(wl.f_lo, wl.f_hi, F1)), quats(8).astype(np.float32),
                  np.stack([synth.ear_table(rng) for _ in range(8)]).astype(np.float32), m8, F1))
    F2 = 40
    specs.append((synth.piston_table(0.003, np.linspace(wl.f_lo, wl.f_hi, F2)), None, None, m8[:5].copy(), F2))
    specs.append((None, None, None, m8[:4].copy(), 33))
    jobs, wjs = [], []
    for i, (et, mq, mt, mics, F) in enumerate(specs):
        q = unit_quat(rng) if i > 0 else wl.emitter_quat
        wj = dataclasses.replace(wl, emitter_quat=q, mics=mics, n_bins=F, emitter_table=et, mic_quats=mq, mic_tables=mt,
                                 fov_half=fov)
        jobs.append(st.BatchJob(sc, wj.emitter, q, wj.dirs, mics, F, wl.f_lo, wl.f_hi, wl.bounces, pose_index=0,
                                fov_half=fov, emitter_table=et, mic_quats=mq, mic_tables=mt))
        wjs.append(wj)
    p = st.sim_params(max_distance=wl.max_distance)
    for rep in range(2):  # the eager run, then the recorded graph
        outs = [o.cpu().numpy().copy() for o in ctx.simulate_batch(jobs, p)]
        for j, wj in enumerate(wjs):
            ctx.set_frequencies(wj.n_bins, wj.f_lo, wj.f_hi)
            ctx.set_emitter(wj.emitter, wj.emitter_quat, wj.dirs, wj.emitter_table, wj.fov_half)
            ctx.set_receivers(wj.mics, wj.mic_quats, wj.mic_tables)
            ref = ctx.simulate(sc, st.sim_params(max_bounces=wj.bounces, max_distance=wj.max_distance)).cpu().numpy()
            for c in range(3):
                assert rel_l2(outs[j][c], ref[c]) <= TOL_SINGLE, (rep, j, c, rel_l2(outs[j][c], ref[c]))
            assert np.abs(ref[0]).sum() > 0 and np.abs(ref[1]).sum() > 0
    o = oracle.simulate(wjs[0], curv=dict(budget=100_000))
    for c in range(3):
        assert rel_l2(outs[0][c], o["spectra"][c]) <= TOL, (c, rel_l2(outs[0][c], o["spectra"][c]))
    # the tables are read at run time: a replay after scaling one in place gives the scaled spectra
    jobs[1].mic_tables.mul_(0.5)
    half = [o.cpu().numpy().copy() for o in ctx.simulate_batch(jobs, p)]
    for c in range(3):
        assert rel_l2(half[1][c], 0.5 * outs[1][c]) <= 1e-6


def test_batch_tensor_diffraction(st):
    """Diffraction paths of omni jobs with three or more microphones and 128 or more bins are accumulated on
    the tensor cores in the batch too (the candidates sorted by job and material): jobs spanning several
    microphone and bin blocks with ragged tails, and one job of a million paths accumulated on its own,
    against the single-pose path and, for two jobs, the oracle."""
    import oracle
    ctx = st.Context(0)
    scenes, jobs0, wl_jobs0 = make_case(st, ctx, seed=21, n_scenes=2, poses=3)
    rng = np.random.default_rng(2121)
    shapes = [(3, 128), (5, 700), (12, 513), (4, 300), (9, 1100), (7, 256)]
    jobs, wl_jobs = [], []
    for i, (job, wj) in enumerate(zip(jobs0, wl_jobs0)):
        M, F = shapes[i % len(shapes)]
        mics = (wj.emitter + rng.uniform(-0.3, 0.3, size=(M, 3))).astype(np.float32)
        n = 262_144 if i == 1 else wj.dirs.shape[0]
        bounces = 4 if i == 1 else wj.bounces
        w = dataclasses.replace(wj, mics=mics, n_bins=F, dirs=synth.fibonacci_directions(n), bounces=bounces)
        jobs.append(st.BatchJob(job.scene, w.emitter, w.emitter_quat, w.dirs, w.mics, F, w.f_lo, w.f_hi, bounces,
                                pose_index=job.job.pose_index, fov_half=w.fov_half))
        wl_jobs.append(w)
    p = st.sim_params(max_distance=60.0)
    outs = [o.cpu().numpy() for o in ctx.simulate_batch(jobs, p)]
    n_diff = 0
    for j, (job, wj) in enumerate(zip(jobs, wl_jobs)):
        ref = single(st, ctx, job.scene, wj, job.job.pose_index)
        for c in range(3):
            assert rel_l2(outs[j][c], ref[c]) <= TOL_SINGLE, (j, c, rel_l2(outs[j][c], ref[c]))
        n_diff += int(np.abs(outs[j][1]).sum() > 0)
    assert n_diff >= len(jobs) - 1
    for j in (0, 2):
        wj = wl_jobs[j]
        o = oracle.simulate(wj, curv=dict(budget=50_000), pose=jobs[j].job.pose_index)
        for c in range(3):
            assert rel_l2(outs[j][c], o["spectra"][c]) <= TOL, (j, c, rel_l2(outs[j][c], o["spectra"][c]))


def test_batch_tensor_diffraction_long_accumulation(st):
    """A job whose diffraction accumulation runs as few chunks of many tiles (62 microphones x 1902 bins,
    about 25k kept samples, in a batch): the matrix-product accumulators are flushed into the spectrum
    registers every few tiles, so the error stays at the level of a single chunk's, well inside the
    spectra tolerance, against the oracle's float64 diffraction spectrum."""
    import oracle
    wls, specs = synth.batched_poses(seed=505)
    sp = specs[233]
    wl = wls[sp["scene"]]
    rng = np.random.default_rng(7)
    q = unit_quat(rng)
    wj = dataclasses.replace(wl, emitter=sp["emitter"], emitter_quat=q, dirs=synth.fibonacci_directions(1000),
                             mics=sp["mics"], n_bins=sp["n_bins"], bounces=sp["bounces"], max_distance=60.0,
                             diffraction=True, fov_half=math.pi)
    assert len(wj.mics) >= 32 and wj.n_bins > 1024
    ctx = st.Context(0)
    sc = st.Scene(ctx, wj.verts, wj.tris, wj.tri_mat, wj.tri_obj)
    sc.set_materials(wj.band_hz, wj.k_band, wj.beta_band, wj.diff_band)
    sc.precompute(st.curv_params(sample_budget=65536))
    job = st.BatchJob(sc, wj.emitter, wj.emitter_quat, wj.dirs, wj.mics, wj.n_bins, wj.f_lo, wj.f_hi, wj.bounces,
                      pose_index=sp["pose_index"])
    out = ctx.simulate_batch([job], st.sim_params(max_distance=60.0))[0].cpu().numpy()
    o = oracle.simulate(wj, curv=dict(budget=65536), pose=sp["pose_index"], components=2)
    assert np.abs(o["spectra"][1]).sum() > 0
    err = rel_l2(out[1], o["spectra"][1])
    assert err <= 3e-5, err
