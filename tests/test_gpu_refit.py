"""Dynamic scenes: new vertex positions refit into the LBVH topology of the first build.  The
results must equal the oracle on the moved scene exactly (path sets, curvature, samples) and within
the spectra tolerance: boxes stay conservative whatever the motion."""
import dataclasses
import math

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


def rot(axis, ang):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def move_meshes(wl, meshes, shift, ang):
    v = wl.verts.astype(np.float64).copy()
    for k, m in enumerate(meshes):
        idx = np.unique(wl.tris[wl.tri_obj == m])
        c = v[idx].mean(0)
        R = rot([0.3, 1.0, 0.2 * k], ang * (k + 1))
        v[idx] = (v[idx] - c) @ R.T + c + np.asarray(shift) * (k + 1)
    return v.astype(np.float32)


def compare(ctx, sc, S, wl, o):
    g = ctx.paths(wl.bounces)
    for k in ("tri", "los", "p", "d", "r"):
        a, b = g[k], o["rec"][k]
        assert np.array_equal(a, b), k
    G, C, ns = sc.curvature()
    assert np.array_equal(G, o["G"]) and np.array_equal(C, o["C"]) and np.array_equal(ns, o["cdf"]["n_samples"])
    ct, cp, keep = ctx.diffraction()
    assert np.array_equal(ct, o["cand_tri"]) and np.array_equal(cp, o["cand_p"]) and np.array_equal(keep, o["cand_keep"])
    for c in range(3):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL, (c, rel_l2(S[c], o["spectra"][c]))


def test_refit_rigid_and_large_motion_matches_oracle(st):
    import oracle
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=20_000, bounces=4, n_mics=6, n_bins=64)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=100_000))
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    ctx.simulate(sc, p)
    meshes = list(range(1, int(wl.tri_obj.max()) + 1, 3))
    for shift, ang in (((0.05, -0.02, 0.0), 0.2), ((2.0, 1.5, 0.3), 1.1)):  # small, then large motion
        v = move_meshes(wl, meshes, shift, ang)
        sc.update_vertices(v)
        wm = dataclasses.replace(wl, verts=v)
        S = ctx.simulate(sc, p).cpu().numpy()
        o = oracle.simulate(wm, curv=dict(budget=100_000))
        compare(ctx, sc, S, wm, o)


def test_refit_deformation_matches_fresh_build(st):
    """A smooth non-rigid deformation of every vertex: refit == a fresh precompute of the moved scene."""
    wl = synth.clutter(seed=7, target_tris=8_000, n_rays=8_000, bounces=3, n_mics=4, n_bins=32)
    v = wl.verts.astype(np.float64)
    v2 = (v + 0.05 * np.sin(v[:, [1, 2, 0]] * 1.3)).astype(np.float32)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    sc.update_vertices(v2)
    S1 = ctx.simulate(sc, p).cpu().numpy()
    g1 = ctx.paths(wl.bounces)
    d1 = ctx.diffraction()
    ctx2 = st.Context(0)
    sc2 = st.from_workload(ctx2, dataclasses.replace(wl, verts=v2))
    S2 = ctx2.simulate(sc2, p).cpu().numpy()
    g2 = ctx2.paths(wl.bounces)
    d2 = ctx2.diffraction()
    for k in g1:
        assert np.array_equal(g1[k], g2[k]), k
    for a, b in zip(d1, d2):
        assert np.array_equal(a, b)
    assert np.array_equal(S1[2], S2[2])  # direct path: same inputs, same kernels
    for c in (0, 1):
        assert rel_l2(S1[c], S2[c]) <= 1e-6


def test_refit_keep_curvature_rigid_translation(st):
    """Rigid motion with the curvature kept: specular and direct paths equal the oracle's."""
    import oracle
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=10_000, bounces=3, n_mics=4, n_bins=48)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    v = move_meshes(wl, [2, 5, 9], (0.5, 0.25, 0.0), 0.0)
    sc.update_vertices(v, keep_curvature=True)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance,
                      components=st.ST_COMP_SPECULAR | st.ST_COMP_DIRECT)
    S = ctx.simulate(sc, p).cpu().numpy()
    wm = dataclasses.replace(wl, verts=v, diffraction=False)
    o = oracle.simulate(wm, components=5)
    g = ctx.paths(wl.bounces)
    for k in ("tri", "los", "p", "d", "r"):
        assert np.array_equal(g[k], o["rec"][k]), k
    for c in (0, 2):
        assert rel_l2(S[c], o["spectra"][c]) <= TOL
