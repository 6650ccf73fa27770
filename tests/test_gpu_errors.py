"""Status codes of the C ABI through the binding: meshes the device validation rejects (ST_ERR_MESH),
calls out of order (ST_ERR_STATE) and arguments out of range (ST_ERR_ARG); after every error the
context still gives the same spectra, bit for bit, as before it.  Every case is turned into an error on
the host or by the device's validation pass, which runs before any kernel indexes with the mesh."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st_
    return st_


def status_of(st, fn, *a, **kw):
    with pytest.raises(st.SonotraceError) as e:
        fn(*a, **kw)
    return e.value.status


def new_scene(st, ctx, wl, verts=None, tris=None, mat=None, obj=None):
    sc = st.Scene(ctx, wl.verts if verts is None else verts, wl.tris if tris is None else tris,
                  wl.tri_mat if mat is None else mat, wl.tri_obj if obj is None else obj)
    sc.set_materials(wl.band_hz, wl.k_band, wl.beta_band, wl.diff_band)
    return sc


def test_mesh_errors_leave_the_context_usable(st):
    wl = synth.clutter(seed=31, target_tris=3000, n_rays=3000, bounces=3, n_mics=4, n_bins=32)
    ctx = st.Context(0)
    good = st.from_workload(ctx, wl, st.curv_params(sample_budget=20_000))
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    S_ref = ctx.simulate(good, p).cpu().numpy()
    assert np.abs(S_ref).sum() > 0

    T = wl.tris.copy()
    T[5, 1] = len(wl.verts)  # vertex index past the end
    assert status_of(st, new_scene(st, ctx, wl, tris=T).precompute) == st.ST_ERR_MESH
    T = wl.tris.copy()
    T[7, 2] = -1
    assert status_of(st, new_scene(st, ctx, wl, tris=T).precompute) == st.ST_ERR_MESH
    V = wl.verts.copy()
    V[3, 2] = np.nan
    assert status_of(st, new_scene(st, ctx, wl, verts=V).precompute) == st.ST_ERR_MESH
    V[3, 2] = np.inf
    assert status_of(st, new_scene(st, ctx, wl, verts=V).precompute) == st.ST_ERR_MESH
    M = wl.tri_mat.copy()
    M[0] = wl.k_band.shape[0]  # material past the table
    assert status_of(st, new_scene(st, ctx, wl, mat=M).precompute) == st.ST_ERR_MESH
    O = wl.tri_obj.copy()
    O[0] = -2
    assert status_of(st, st.Scene, ctx, wl.verts, wl.tris, wl.tri_mat, O) == st.ST_ERR_MESH
    # a scene that failed validation cannot be simulated
    T = wl.tris.copy()
    T[5, 1] = len(wl.verts)
    bad = new_scene(st, ctx, wl, tris=T)
    status_of(st, bad.precompute)
    assert status_of(st, ctx.simulate, bad, p) == st.ST_ERR_STATE
    # a refit to a non-finite vertex leaves the scene unbuilt; an update with the original positions
    # builds it in full again (same vertices, same parameters: the same spectra bit for bit)
    moved = st.from_workload(ctx, wl, st.curv_params(sample_budget=20_000))
    V = wl.verts.copy()
    V[10, 0] = np.inf
    assert status_of(st, moved.update_vertices, V) == st.ST_ERR_MESH
    assert status_of(st, ctx.simulate, moved, p) == st.ST_ERR_STATE
    moved.update_vertices(wl.verts)
    assert np.array_equal(ctx.simulate(moved, p).cpu().numpy(), S_ref)
    # the good scene, unchanged by the errors above: the same spectra bit for bit
    assert np.array_equal(ctx.simulate(good, p).cpu().numpy(), S_ref)
    # a scene never precomputed cannot be updated
    fresh = new_scene(st, ctx, wl)
    assert status_of(st, fresh.update_vertices, wl.verts) == st.ST_ERR_STATE


def test_order_and_argument_checks(st):
    wl = synth.shoebox(seed=7, n_rays=200, bounces=2, n_mics=3, n_bins=16)
    ctx = st.Context(0)
    sc = st.Scene(ctx, wl.verts, wl.tris, wl.tri_mat, wl.tri_obj)
    assert status_of(st, sc.precompute) == st.ST_ERR_STATE  # materials first
    sc.set_materials(wl.band_hz, wl.k_band, wl.beta_band, wl.diff_band)
    p = st.sim_params(max_bounces=2)
    import torch
    out = torch.empty((3, len(wl.mics), wl.n_bins), dtype=torch.complex64, device="cuda:0")
    assert status_of(st, ctx.simulate, sc, p, out) == st.ST_ERR_STATE  # not precomputed, no sensor
    sc.precompute()
    assert status_of(st, ctx.simulate, sc, p, out) == st.ST_ERR_STATE  # emitter, receivers, grid missing
    assert status_of(st, ctx.paths, 2) == st.ST_ERR_STATE  # no simulate yet
    assert status_of(st, sc.set_materials, wl.band_hz, wl.k_band, np.zeros_like(wl.beta_band),
                     wl.diff_band) == st.ST_ERR_ARG  # beta must be > 0
    if len(wl.band_hz) > 1:
        assert status_of(st, sc.set_materials, wl.band_hz[::-1].copy(), wl.k_band, wl.beta_band,
                         wl.diff_band) == st.ST_ERR_ARG  # band centres must ascend
    assert status_of(st, ctx.set_frequencies, 0, wl.f_lo, wl.f_hi) == st.ST_ERR_ARG
    assert status_of(st, ctx.set_frequencies, 8, wl.f_hi, wl.f_lo) == st.ST_ERR_ARG
    assert status_of(st, ctx.set_receivers, np.zeros((0, 3), np.float32)) == st.ST_ERR_ARG
    ctx.set_frequencies(wl.n_bins, wl.f_lo, wl.f_hi)
    ctx.set_emitter(wl.emitter, wl.emitter_quat, wl.dirs)
    ctx.set_receivers(wl.mics)
    for bounces in (0, 9):
        assert status_of(st, ctx.simulate, sc, st.sim_params(max_bounces=bounces)) == st.ST_ERR_ARG
    G = torch.ones((3, len(wl.mics), wl.n_bins), dtype=torch.complex64, device="cuda:0")
    assert status_of(st, ctx.backward, sc, G, *wl.k_band.shape) == st.ST_ERR_STATE  # no simulate yet
    S = ctx.simulate(sc, p)
    ctx.backward(sc, G, *wl.k_band.shape)
    sc.update_vertices(wl.verts)  # a refit: the path set of the last simulate no longer belongs to the scene
    assert status_of(st, ctx.backward, sc, G, *wl.k_band.shape) == st.ST_ERR_STATE
    assert np.array_equal(ctx.simulate(sc, p).cpu().numpy(), S.cpu().numpy())
