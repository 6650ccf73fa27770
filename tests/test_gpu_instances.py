"""Instanced scenes (st_scene_load_instances, st_scene_set_instance_transforms) against the oracle: the
world triangles the device expands equal the oracle's expansion bit for bit, the path set of a simulate
over them equals the oracle's on its expanded scene (spectra within 1e-4), and so they do again after the
instances have been moved and the scene refit; plus the argument checks of the instance calls."""
import dataclasses

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def st():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st_
    return st_


def flat(fo, xform):
    import oracle
    V, T, M, O = oracle.expand_instances(fo.protos, fo.inst_proto, xform)
    return dataclasses.replace(fo.base, verts=V, tris=T, tri_mat=M, tri_obj=O)


def check_geometry(sc, wl):
    V, T, M, O = sc.geometry()
    assert np.array_equal(V, wl.verts) and np.array_equal(T, wl.tris)
    assert np.array_equal(M, wl.tri_mat) and np.array_equal(O, wl.tri_obj)


def simulate_and_compare(st, ctx, sc, wl, budget):
    import oracle
    S, stats = ctx.simulate(sc, st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance), stats=True)
    S = S.cpu().numpy()
    o = oracle.simulate(wl, curv=dict(budget=budget))
    g, rec = ctx.paths(wl.bounces), o["rec"]
    assert np.array_equal(g["tri"], rec["tri"]) and np.array_equal(g["los"], rec["los"])
    hit = rec["tri"] >= 0
    assert np.array_equal(g["p"][hit], rec["p"][hit])
    _, _, keep = ctx.diffraction()
    assert np.array_equal(keep, o["cand_keep"]) and keep.sum() > 500
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))
    return S


def test_forest_expansion_and_parity_before_and_after_moving(st):
    fo = synth.instanced_forest(seed=606, n_inst=300, n_rays=20_000, bounces=3, n_mics=8, n_bins=64)
    b = fo.base
    ctx = st.Context(0)
    sc = st.Scene.from_instances(ctx, fo.protos, fo.inst_proto, fo.inst_xform)
    assert sc.n_tris == sum(len(fo.protos[q][1]) for q in fo.inst_proto)
    sc.set_materials(b.band_hz, b.k_band, b.beta_band, b.diff_band)
    sc.precompute(st.curv_params(sample_budget=100_000))
    ctx.set_frequencies(b.n_bins, b.f_lo, b.f_hi)
    ctx.set_emitter(b.emitter, b.emitter_quat, b.dirs, None, b.fov_half)
    ctx.set_receivers(b.mics)
    wl = flat(fo, fo.inst_xform)
    check_geometry(sc, wl)
    S0 = simulate_and_compare(st, ctx, sc, wl, 100_000)
    # move every third plant: a turn about the vertical and a shift, then a full refit
    rng = np.random.default_rng(7)
    X = fo.inst_xform.astype(np.float64).copy()
    for i in range(1, len(X), 3):
        a = rng.uniform(-0.5, 0.5)
        Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
        X[i, :, :3] = Rz @ X[i, :, :3]
        X[i, :2, 3] += rng.uniform(-0.4, 0.4, 2)
    X = X.astype(np.float32)
    sc.set_instance_transforms(X)
    wl2 = flat(fo, X)
    check_geometry(sc, wl2)
    S1 = simulate_and_compare(st, ctx, sc, wl2, 100_000)
    assert not np.array_equal(S0, S1)
    # the transforms from device memory give the same scene
    import torch
    sc.set_instance_transforms(torch.as_tensor(fo.inst_xform, device="cuda:0"))
    check_geometry(sc, wl)


def test_instance_argument_checks(st):
    fo = synth.instanced_forest(seed=607, n_inst=5, n_rays=64, n_mics=2, n_bins=8)
    ctx = st.Context(0)
    bad = fo.inst_proto.copy()
    bad[2] = len(fo.protos)  # no such prototype
    with pytest.raises(st.SonotraceError):
        st.Scene.from_instances(ctx, fo.protos, bad, fo.inst_xform)
    X = fo.inst_xform.copy()
    X[1, 0, 0] = np.inf
    with pytest.raises(st.SonotraceError):
        st.Scene.from_instances(ctx, fo.protos, fo.inst_proto, X)
    protos = list(fo.protos)
    v, t, m = protos[1]
    t = t.copy()
    t[0, 0] = len(v)  # local index past the prototype's vertices
    protos[1] = (v, t, m)
    with pytest.raises(st.SonotraceError):
        st.Scene.from_instances(ctx, protos, fo.inst_proto, fo.inst_xform)
    sc = st.Scene.from_instances(ctx, fo.protos, fo.inst_proto, fo.inst_xform)
    with pytest.raises(st.SonotraceError):  # not precomputed yet
        sc.set_instance_transforms(fo.inst_xform)
    flat_sc = st.Scene(ctx, *sc.geometry())
    with pytest.raises(st.SonotraceError):  # not an instanced scene
        flat_sc.n_inst = sc.n_inst
        flat_sc.set_instance_transforms(fo.inst_xform)
