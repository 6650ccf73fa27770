"""GPU vs oracle parity through the C ABI.

Bars: path sets (hit triangle per bounce, hit points, reflected directions, float64 path lengths,
visibility flags), curvature, diffraction samples and filters bit-exact; spectra within 1e-4
relative L2 error per component (the target tolerance of the path; float32 amplitudes with
float-float range-reduced phases on the GPU against float64 throughout in the oracle)."""
import dataclasses
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


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


def gpu_run(st, wl, curv=None, **kw):
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, curv)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, **kw)
    S, stats = ctx.simulate(sc, p, stats=True)
    return ctx, sc, S.cpu().numpy(), stats


def compare_paths(g, o, rows=None):
    for k in ("tri", "los", "p", "d", "r"):
        a, b = g[k], o[k]
        if rows is not None:
            a = a[rows]
        mism = np.argwhere(~((a == b) | (np.isnan(a) & np.isnan(b))).reshape(len(a), -1).all(1)) if a.dtype.kind == "f" \
            else np.argwhere(~(a == b).reshape(len(a), -1).all(1))
        assert len(mism) == 0, f"{k}: {len(mism)} rays differ, first {mism[:5].ravel()}"


def test_shoebox_paths_and_spectra(st):
    import oracle
    wl = synth.shoebox(seed=101)
    ctx, sc, S, stats = gpu_run(st, wl)
    g = ctx.paths(wl.bounces)
    o = oracle.simulate(wl)
    compare_paths(g, o["rec"])
    assert stats.visible_records == (o["rec"]["los"] == 1).sum()
    for c in (0, 2):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, c
    assert np.all(S[1] == 0)


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_workload_forward(st, mode):
    import oracle
    wl = synth.gradient_problem(n_rays=3000)
    ctx, sc, S, _ = gpu_run(st, wl, reflection_mode=mode)
    o = oracle.simulate(wl, reflection_mode=mode)
    compare_paths(ctx.paths(wl.bounces), o["rec"])
    for c in (0, 2):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, c


def small_clutter(**kw):
    args = dict(seed=202, target_tris=20_000, n_rays=20_000, bounces=5, n_mics=8, n_bins=96)
    args.update(kw)
    return synth.clutter(**args)


def test_clutter_small_full_parity(st):
    import oracle
    wl = small_clutter()
    curv = dict(budget=200_000)
    ctx, sc, S, stats = gpu_run(st, wl, curv=st.curv_params(sample_budget=200_000))
    o = oracle.simulate(wl, curv=curv)
    compare_paths(ctx.paths(wl.bounces), o["rec"])
    G, C, ns = sc.curvature()
    assert np.array_equal(G, o["G"])
    assert np.array_equal(C, o["C"])
    assert np.array_equal(ns, o["cdf"]["n_samples"])
    ct, cp, keep = ctx.diffraction()
    assert np.array_equal(ct, o["cand_tri"])
    assert np.array_equal(cp, o["cand_p"])
    assert np.array_equal(keep, o["cand_keep"])
    assert np.array_equal(ctx.direct_visibility(), o["direct_vis"])
    assert keep.sum() > 100 and stats.visible_records > 1000
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))


def test_ragged_sizes_and_single_mic_bin(st):
    """M = 1, F = 1 and sizes that are not multiples of any tile."""
    import oracle
    for M, F in [(1, 1), (3, 17), (33, 35)]:
        wl = small_clutter(target_tris=3000, n_rays=1537, n_mics=M, n_bins=F, bounces=3, diffraction=False)
        ctx, sc, S, _ = gpu_run(st, wl)
        o = oracle.simulate(wl)
        compare_paths(ctx.paths(wl.bounces), o["rec"])
        for c in (0, 2):
            assert rel_l2(S[c], o["spectra"][c]) <= TOL, (M, F, c)


@pytest.mark.parametrize("M,F", [(12, 196), (5, 84), (33, 35), (32, 512)])
def test_ragged_sizes_with_diffraction(st, M, F):
    """Diffraction accumulated at tile shapes with partial warps and ragged bin runs (12 mics x 196 bins: 78
    threads per CTA, 13 runs of 16 bins), each CTA running several path tiles."""
    import oracle
    wl = small_clutter(target_tris=3000, n_rays=1537, n_mics=M, n_bins=F, bounces=2)
    ctx, sc, S, stats = gpu_run(st, wl, curv=st.curv_params(sample_budget=60_000))
    o = oracle.simulate(wl, curv=dict(budget=60_000))
    ct, cp, keep = ctx.diffraction()
    assert np.array_equal(keep, o["cand_keep"])
    assert keep.sum() > 2000
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (M, F, c, rel_l2(S[c], o["spectra"][c]))


@pytest.mark.parametrize("los_mode", [0, 1])
def test_zero_rays_direct_and_diffraction_only(st, los_mode):
    """An emitter with no rays: no specular records (the specular spectra are exactly zero) while the
    direct path and diffraction still follow the oracle, in both receiver-test modes."""
    import oracle
    wl = dataclasses.replace(small_clutter(target_tris=3000, n_rays=1, n_mics=3, n_bins=20, bounces=2),
                             dirs=np.zeros((0, 3), np.float32))
    ctx, sc, S, stats = gpu_run(st, wl, curv=st.curv_params(sample_budget=60_000), los_mode=los_mode)
    o = oracle.simulate(wl, curv=dict(budget=60_000), los_mode=los_mode)
    assert stats.records == 0 and ctx.paths(wl.bounces)["tri"].shape == (0, wl.bounces)
    if los_mode:
        assert ctx.receiver_masks(wl.bounces).shape == (0, wl.bounces)
    assert np.all(S[0] == 0)
    _, _, keep = ctx.diffraction()
    assert np.array_equal(keep, o["cand_keep"]) and keep.sum() > 1000
    assert np.array_equal(ctx.direct_visibility(), o["direct_vis"])
    for c in (1, 2):
        assert np.abs(o["spectra"][c]).sum() > 0
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))


@pytest.mark.parametrize("T", [1, 2, 3, 4, 5, 7, 8, 9, 31, 32, 33, 1000])
def test_bvh_small_triangle_counts(st, T):
    """Leaf-size and warp boundaries of the LBVH: GPU closest hits equal brute force."""
    import oracle
    rng = np.random.default_rng(T)
    c = rng.uniform(-1, 1, size=(T, 1, 3))
    v = (c + 0.3 * rng.normal(size=(T, 3, 3))).reshape(-1, 3).astype(np.float32)
    tris = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    n_bands = 2
    wl = synth.Workload(name="soup", verts=v, tris=tris, tri_mat=np.zeros(T, np.int32),
                        tri_obj=np.zeros(T, np.int32), band_hz=np.array([20e3, 80e3], np.float32),
                        k_band=np.full((1, n_bands), 0.9, np.float32), beta_band=np.full((1, n_bands), 0.3, np.float32),
                        diff_band=np.full((1, n_bands), 0.05, np.float32), emitter=np.zeros(3, np.float32),
                        emitter_quat=np.array([1, 0, 0, 0], np.float32), dirs=synth.fibonacci_directions(4096),
                        mics=np.array([[0.1, 0.2, 0.05]], np.float32), n_bins=4, f_lo=20e3, f_hi=80e3, bounces=4)
    ctx, sc, S, _ = gpu_run(st, wl)
    o = oracle.simulate(wl, use_bvh=False)
    compare_paths(ctx.paths(wl.bounces), o["rec"])
    assert rel_l2(S[0], o["spectra"][0]) <= TOL


def test_vegetation_directivity_parity(st):
    """Leaf-disc vegetation with a piston emitter table, two ears with directivity tables (bilinear in
    azimuth/elevation, linear between bands) and the field-of-view filter (half-angle pi/2)."""
    import oracle
    wl = synth.vegetation(seed=303, target_tris=40_000, n_rays=30_000, bounces=4, n_bins=96, leaves_per_mesh=64)
    ctx, sc, S, stats = gpu_run(st, wl, curv=st.curv_params(sample_budget=200_000))
    o = oracle.simulate(wl, curv=dict(budget=200_000))
    compare_paths(ctx.paths(wl.bounces), o["rec"])
    ct, cp, keep = ctx.diffraction()
    assert np.array_equal(ct, o["cand_tri"]) and np.array_equal(cp, o["cand_p"])
    assert np.array_equal(keep, o["cand_keep"])
    assert 0 < keep.sum() < len(keep)
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))


@pytest.mark.parametrize("M,F,mode", [(2, 1, 0), (1, 17, 0), (2, 1000, 0), (2, 1000, 1), (2, 2048, 0), (1, 4100, 0)])
def test_narrow_arrays(st, M, F, mode):
    """One microphone pair (the narrow-array accumulator): bin counts from 1 to beyond one CTA's
    4096 bins, both reflection modes, diffraction on."""
    import oracle
    wl = small_clutter(target_tris=5000, n_rays=3000, n_mics=M, n_bins=F, bounces=4)
    ctx, sc, S, _ = gpu_run(st, wl, curv=st.curv_params(sample_budget=20_000), reflection_mode=mode)
    o = oracle.simulate(wl, curv=dict(budget=20_000), reflection_mode=mode)
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (M, F, mode, c, rel_l2(S[c], o["spectra"][c]))


@pytest.mark.parametrize("mode", [0, 1])
def test_eight_bounces(st, mode):
    """The largest chain length the interface accepts (B = 8, every byte of the packed material chain in
    use): the four-material room with the 32-microphone array (general accumulator) in both reflection
    modes, and a clutter scene with diffraction and one microphone pair (narrow accumulator)."""
    import oracle
    wl = synth.shoebox(seed=404, n_rays=3000, bounces=8, n_bins=128, n_mics=32, four_materials=True)
    ctx, sc, S, stats = gpu_run(st, wl, reflection_mode=mode)
    o = oracle.simulate(wl, reflection_mode=mode)
    g = ctx.paths(wl.bounces)
    compare_paths(g, o["rec"])
    assert (g["tri"][:, 7] >= 0).sum() > 1000
    for c in (0, 2):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))
    wl = small_clutter(target_tris=5000, n_rays=4000, n_mics=2, n_bins=300, bounces=8)
    ctx, sc, S, stats = gpu_run(st, wl, curv=st.curv_params(sample_budget=20_000), reflection_mode=mode)
    o = oracle.simulate(wl, curv=dict(budget=20_000), reflection_mode=mode)
    compare_paths(ctx.paths(wl.bounces), o["rec"])
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))


def test_phase_at_the_largest_f_r_over_c(st):
    """The phase far from the origin of the range reduction: one ray to a mirror 60 m away and back to a
    microphone beside the emitter and to one 100 m behind it on the reflected ray (paths of about 120 and
    220 m), and the direct paths (0.5 and 100 m), over 1024 bins from 20 to 120 kHz, the vegetation
    workload's band: up to 7.7e4 cycles of f r / c.  Air absorption is off so that every amplitude stays
    well inside float32's range.  Every bin of the specular and direct spectra is compared on its own with
    the oracle's float64 value (relative error 1e-5 per bin, far inside the 1e-4 relative L2 bar)."""
    import oracle
    v = np.array([[60, -80, -80], [60, 80, -80], [60, 0, 120]], np.float32)
    d = np.array([[60.0, 0.25, 0.0]]) / np.linalg.norm([60.0, 0.25, 0.0])
    wl = synth.Workload(name="mirror", verts=v, tris=np.array([[0, 1, 2]], np.int32), tri_mat=np.zeros(1, np.int32),
                        tri_obj=np.zeros(1, np.int32), band_hz=np.array([20e3, 120e3], np.float32),
                        k_band=np.array([[0.9, 0.7]], np.float32), beta_band=np.array([[0.3, 0.2]], np.float32),
                        diff_band=np.full((1, 2), 0.05, np.float32), emitter=np.zeros(3, np.float32),
                        emitter_quat=np.array([1, 0, 0, 0], np.float32), dirs=d.astype(np.float32),
                        mics=np.array([[0.0, 0.5, 0.0], [-100.0, 0.917, 0.0]], np.float32), n_bins=1024,
                        f_lo=20e3, f_hi=120e3, bounces=1)
    comp = st.ST_COMP_SPECULAR | st.ST_COMP_DIRECT
    ctx, sc, S, stats = gpu_run(st, wl, components=comp, alpha1_db_m_khz=0.0)
    o = oracle.simulate(wl, components=5, a1_per_khz=0.0)
    compare_paths(ctx.paths(wl.bounces), o["rec"])
    assert o["rec"]["los"][0, 0] == 1 and o["rec"]["r"][0, 0] > 59.0
    for c in (0, 2):
        ref = o["spectra"][c]
        assert np.abs(ref).min() > 0
        err = np.abs(S[c] - ref) / np.abs(ref)
        assert err.max() <= 1e-5, (c, err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("depth", [1, 2, 3, 6])
def test_stack_restarts_keep_results_exact(st, depth):
    """A query whose short stack would overflow restarts from the root with the stackless walk (fixed child
    order, parent references in the nodes) and keeps its best hit: with stacks of 1 to 6 entries, where most
    queries restart, every path record, diffraction filter, direct visibility and spectrum is bit-identical
    to the default 128-entry stack, and the path records equal the oracle's."""
    import oracle
    wl = small_clutter(target_tris=8000, n_rays=6000, bounces=4, n_mics=4, n_bins=48)
    curv = st.curv_params(sample_budget=40_000)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, curv)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    S0, s0 = ctx.simulate(sc, p, stats=True)
    S0 = S0.cpu().numpy()
    g0 = ctx.paths(wl.bounces)
    ct0, cp0, k0 = ctx.diffraction()
    dv0 = ctx.direct_visibility()
    assert s0.stack_restarts == 0
    ctx.set_tune(stack_depth=depth)
    S1, s1 = ctx.simulate(sc, p, stats=True)
    assert s1.stack_restarts > 0
    g1 = ctx.paths(wl.bounces)
    for k in ("tri", "p", "d", "r", "los"):
        assert np.array_equal(g0[k], g1[k]), k
    ct1, cp1, k1 = ctx.diffraction()
    assert np.array_equal(k0, k1) and np.array_equal(dv0, ctx.direct_visibility())
    assert np.array_equal(S0, S1.cpu().numpy())
    o = oracle.simulate(wl, curv=dict(budget=40_000))
    compare_paths(g1, o["rec"])
    assert np.array_equal(k1, o["cand_keep"])
    ctx.set_tune(stack_depth=0)
    with pytest.raises(st.SonotraceError):
        ctx.set_tune(stack_depth=129)


@pytest.mark.parametrize("case", ["clutter", "vegetation"])
def test_stage_overlap_gives_identical_results(st, case):
    """The diffraction stage (sampling, filters, line of sight, accumulation) and the direct path run on a
    side stream beside the trace (the default) or in order on the context's stream: path records,
    diffraction samples and filters, direct visibility, all three spectra and the gradients of a backward
    call are bit-identical either way, over consecutive calls.  The vegetation case has over a million
    triangles, so the hit-point and the candidate line-of-sight queues are both sorted, each stage with
    its own sort buffers."""
    import torch
    if case == "clutter":
        wl = small_clutter(target_tris=20_000, n_rays=20_000, bounces=4, n_mics=12, n_bins=196)
        curv = st.curv_params(sample_budget=200_000)
    else:
        wl = synth.vegetation(seed=303, target_tris=1_100_000, n_rays=200_000, bounces=3, n_bins=256)
        curv = None
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, curv)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    rng = np.random.default_rng(5)
    res = []
    for on in (True, False, True):
        ctx.set_stage_overlap(on)
        S, s = ctx.simulate(sc, p, stats=True)
        assert s.ms_trace > 0 and s.ms_diffraction > 0 and s.ms_accumulate > 0 and s.candidates_kept > 0
        r = dict(S=S.cpu().numpy(), paths=ctx.paths(wl.bounces), diff=ctx.diffraction(),
                 dvis=ctx.direct_visibility())
        if case == "clutter":
            G = torch.as_tensor(rng.standard_normal(S.shape) + 1j * rng.standard_normal(S.shape),
                                dtype=torch.complex64, device=S.device) if not res else res[0]["G"]
            r["G"] = G
            r["grad"] = [g.cpu().numpy() for g in ctx.backward(sc, G, wl.k_band.shape[0], wl.k_band.shape[1])]
        res.append(r)
    ref = res[1]
    assert np.abs(ref["S"][1]).max() > 0 and np.abs(ref["S"][0]).max() > 0
    for r in (res[0], res[2]):
        assert np.array_equal(r["S"], ref["S"])
        for k in ("tri", "p", "d", "r", "los"):
            assert np.array_equal(r["paths"][k], ref["paths"][k]), k
        for a, b in zip(r["diff"], ref["diff"]):
            assert np.array_equal(a, b)
        assert np.array_equal(r["dvis"], ref["dvis"])
        if case == "clutter":
            for a, b in zip(r["grad"], ref["grad"]):
                assert np.array_equal(a, b)
