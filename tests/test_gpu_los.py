"""Per-microphone receiver test (ST_LOS_PER_MIC) against the oracle: path records and the per-record
microphone masks bit for bit, spectra within the spectra tolerance, for the general accumulator (a spread
array whose microphones see different hit points), a plane wall between two microphone groups, and the
two-microphone accumulator with directivity tables; the gradients of the adjoint over masked records; and
the argument checks of the mode (the batched form's parity is in test_gpu_batch)."""
import dataclasses

import numpy as np
import pytest

import synth
from test_oracle_los import _wall_workload

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


def run_both(st, wl, curv_budget=None):
    import oracle
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=curv_budget) if curv_budget else None)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, los_mode=st.ST_LOS_PER_MIC)
    S, stats = ctx.simulate(sc, p, stats=True)
    o = oracle.simulate(wl, curv=dict(budget=curv_budget) if curv_budget else None, los_mode=1)
    return ctx, S.cpu().numpy(), stats, o


def check_paths_and_masks(ctx, wl, o):
    g = ctx.paths(wl.bounces)
    rec = o["rec"]
    assert np.array_equal(g["tri"], rec["tri"])
    hit = rec["tri"] >= 0
    assert np.array_equal(g["p"][hit], rec["p"][hit])
    assert np.array_equal(g["los"], rec["los"])
    m = ctx.receiver_masks(wl.bounces)
    assert np.array_equal(m, rec["mask"])
    return m, hit


def test_spread_array_masks_and_spectra(st):
    rng = np.random.default_rng(61)
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=20_000, bounces=4, n_mics=12, n_bins=96)
    mics = np.stack([rng.uniform(-8, 8, 12), rng.uniform(-8, 8, 12), rng.uniform(0.3, 2.0, 12)], 1)
    wl = dataclasses.replace(wl, mics=mics.astype(np.float32))
    ctx, S, stats, o = run_both(st, wl, curv_budget=100_000)
    m, hit = check_paths_and_masks(ctx, wl, o)
    full = np.uint64((1 << 12) - 1)
    partial = hit & (m != 0) & (m != full)
    assert partial.sum() > 1000  # hit points that some microphones see and others do not
    assert stats.shadow_queries >= 12 * stats.records
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))


def test_wall_between_microphone_groups(st):
    wl = _wall_workload()
    ctx, S, _, o = run_both(st, wl)
    m, hit = check_paths_and_masks(ctx, wl, o)
    assert np.any((m[hit] & np.uint64(0b11000)) == 0) and np.any((m[hit] & np.uint64(0b00111)) != 0)
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))


def test_two_ears_with_directivity(st):
    """The accumulator for one microphone pair, with emitter and receiver tables; ears 0.8 m apart so that
    nearby leaves hide a hit point from one ear only."""
    wl = synth.vegetation(seed=303, target_tris=40_000, n_rays=30_000, bounces=3, n_bins=96, leaves_per_mesh=64)
    wl = dataclasses.replace(wl, mics=np.array([[0.0, 0.4, 0.0], [0.0, -0.4, 0.0]], np.float32))
    ctx, S, _, o = run_both(st, wl, curv_budget=200_000)
    m, hit = check_paths_and_masks(ctx, wl, o)
    assert np.sum(hit & ((m == 1) | (m == 2))) > 20
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))


def test_single_microphone_equals_reference_point_test(st):
    # one microphone behind the wall: the wall's own hit points see it, the floor's in front of it do not
    wl = dataclasses.replace(_wall_workload(2000), mics=np.array([[-1.0, 0.0, 1.0]], np.float32))
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    S0 = ctx.simulate(sc, st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)).cpu().numpy()
    los0 = ctx.paths(wl.bounces)["los"]
    S1 = ctx.simulate(sc, st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance,
                                        los_mode=st.ST_LOS_PER_MIC)).cpu().numpy()
    assert np.array_equal(ctx.paths(wl.bounces)["los"], los0)
    assert np.array_equal(ctx.receiver_masks(wl.bounces), los0.astype(np.uint64))
    assert 0 < los0.sum() < (ctx.paths(wl.bounces)["tri"] >= 0).sum()
    assert np.array_equal(S1, S0)


def test_gradients_follow_the_masks(st):
    """st_backward after a per-microphone simulate: reflection, microphone, emitter (specular paths through
    their hit points, diffraction and direct paths) and lobe-width gradients against the oracle's float64
    analytic gradient over the same masked records, 1e-3 per block; a spread array in the clutter scene,
    so that many records reach some microphones and not others."""
    import oracle
    import torch
    rng = np.random.default_rng(62)
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=20_000, bounces=4, n_mics=6, n_bins=40)
    mics = np.stack([rng.uniform(-8, 8, 6), rng.uniform(-8, 8, 6), rng.uniform(0.3, 2.0, 6)], 1)
    wl = dataclasses.replace(wl, mics=mics.astype(np.float32))
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=100_000))
    S = ctx.simulate(sc, st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance,
                                       los_mode=st.ST_LOS_PER_MIC))
    m = ctx.receiver_masks(wl.bounces)
    full = np.uint64((1 << 6) - 1)
    assert np.sum((m != 0) & (m != full)) > 1000
    target = torch.as_tensor(rng.normal(size=S.shape) + 1j * rng.normal(size=S.shape), dtype=torch.complex64,
                             device=S.device) * S.abs().mean()
    G = 2.0 * (S - target)
    n_mat, n_bands = wl.k_band.shape
    gk, gm, ge = (x.cpu().numpy() for x in ctx.backward(sc, G, n_mat, n_bands))
    gb = ctx.backward_beta(sc, G, n_mat, n_bands).cpu().numpy()
    o = oracle.simulate(wl, curv=dict(budget=100_000), los_mode=1)
    assert np.array_equal(o["rec"]["mask"], m)
    dk, dmic, demit, dbeta = oracle.spectra_grad(
        o["params"], o["rec"], wl.dirs, wl.tri_mat, G.cpu().numpy().astype(np.complex128), o.get("cand_tri"),
        o.get("cand_p"), o.get("cand_keep"), o["direct_vis"], with_beta=True,
        tri_nrm=oracle.tri_normals(wl.verts, wl.tris))
    rel = lambda a, b: float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))
    for name, a, b in (("k", gk, dk), ("mic", gm, dmic), ("emitter", ge, demit), ("beta", gb, dbeta)):
        assert rel(a, b) <= 1e-3, (name, rel(a, b))


def test_mode_argument_checks(st):
    wl = synth.shoebox(seed=7, n_rays=64, bounces=2, n_mics=65, n_bins=8)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    with pytest.raises(st.SonotraceError):
        ctx.simulate(sc, st.sim_params(max_bounces=2, los_mode=st.ST_LOS_PER_MIC))
    with pytest.raises(st.SonotraceError):
        ctx.simulate(sc, st.sim_params(max_bounces=2, los_mode=2))
    ctx.set_receivers(wl.mics[:4])
    ctx.simulate(sc, st.sim_params(max_bounces=2))
    with pytest.raises(st.SonotraceError):  # masks exist only after a per-microphone simulate
        ctx.receiver_masks(2)
    ctx.simulate(sc, st.sim_params(max_bounces=2, los_mode=st.ST_LOS_PER_MIC))
    assert ctx.receiver_masks(2).shape == (64, 2)
    job = st.BatchJob(sc, wl.emitter, wl.emitter_quat, wl.dirs, wl.mics, 8, wl.f_lo, wl.f_hi, 2)
    with pytest.raises(st.SonotraceError):  # 65 microphones in a job
        ctx.simulate_batch([job], st.sim_params(los_mode=st.ST_LOS_PER_MIC))
    with pytest.raises(st.SonotraceError):
        ctx.simulate_batch([job], st.sim_params(los_mode=2))
