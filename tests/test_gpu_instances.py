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


# ---------------------------------------------------------------- two-level structure
# Per-prototype BVHs in object space under a BVH over the instances' world boxes.  Triangles are tested in
# world space with the expansion's vertices, so every result must equal the flat structure's bit for bit.

def _scene(st, ctx, fo, xform, two_level, budget=100_000):
    b = fo.base
    sc = st.Scene.from_instances(ctx, fo.protos, fo.inst_proto, xform)
    sc.set_materials(b.band_hz, b.k_band, b.beta_band, b.diff_band)
    if two_level:
        sc.set_structure(True)
    sc.precompute(st.curv_params(sample_budget=budget))
    return sc


def _run(st, ctx, sc, B, **kw):
    p = st.sim_params(max_bounces=B, max_distance=60.0, **kw)
    S, stats = ctx.simulate(sc, p, stats=True)
    out = dict(S=S.cpu().numpy(), paths=ctx.paths(B), keep=ctx.diffraction()[2], direct=ctx.direct_visibility(),
               restarts=stats.stack_restarts)
    if kw.get("los_mode") == st.ST_LOS_PER_MIC:
        out["masks"] = ctx.receiver_masks(B)
    return out


def _same(a, b):
    assert np.array_equal(a["S"], b["S"])
    for k in ("tri", "p", "d", "r", "los"):
        assert np.array_equal(a["paths"][k], b["paths"][k]), k
    assert np.array_equal(a["keep"], b["keep"]) and np.array_equal(a["direct"], b["direct"])
    if "masks" in a:
        assert np.array_equal(a["masks"], b["masks"])


def _sensor(ctx, b, dirs=None, emitter=None):
    ctx.set_frequencies(b.n_bins, b.f_lo, b.f_hi)
    ctx.set_emitter(b.emitter if emitter is None else emitter, b.emitter_quat, b.dirs if dirs is None else dirs, None,
                    b.fov_half)
    ctx.set_receivers(b.mics)


def test_two_level_equals_flat(st):
    """The 300-plant forest: path records, diffraction filters, direct visibility, per-microphone masks and
    spectra of the two-level structure equal the flat structure's bit for bit -- with the default stack,
    with stacks of 1-4 entries (restart walk across both levels), after a full and a curvature-keeping move,
    and after switching the structure of a precomputed scene either way (the flat structure's results are
    pinned to the oracle by the test above)."""
    fo = synth.instanced_forest(seed=606, n_inst=300, n_rays=20_000, bounces=3, n_mics=8, n_bins=64)
    b = fo.base
    ctx = st.Context(0)
    sf = _scene(st, ctx, fo, fo.inst_xform, False)
    stl = _scene(st, ctx, fo, fo.inst_xform, True)
    _sensor(ctx, b)
    ref = _run(st, ctx, sf, 3)
    assert (ref["paths"]["tri"] >= 0).sum() > 10_000 and ref["keep"].sum() > 500
    _same(_run(st, ctx, stl, 3), ref)
    _same(_run(st, ctx, stl, 3, los_mode=st.ST_LOS_PER_MIC), _run(st, ctx, sf, 3, los_mode=st.ST_LOS_PER_MIC))
    for depth in (1, 2, 4):
        ctx.set_tune(stack_depth=depth)
        r = _run(st, ctx, stl, 3)
        assert r["restarts"] > 0, depth
        _same(r, ref)
    ctx.set_tune()
    # move every third plant (full refit / rebuild of the top level), then move back keeping the curvature
    rng = np.random.default_rng(8)
    X = fo.inst_xform.astype(np.float64).copy()
    for i in range(1, len(X), 3):
        a = rng.uniform(-0.5, 0.5)
        Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
        X[i, :, :3] = Rz @ X[i, :, :3]
        X[i, :2, 3] += rng.uniform(-0.4, 0.4, 2)
    X = X.astype(np.float32)
    for sc in (sf, stl):
        sc.set_instance_transforms(X)
    moved = _run(st, ctx, sf, 3)
    assert not np.array_equal(moved["S"], ref["S"])
    _same(_run(st, ctx, stl, 3), moved)
    for sc in (sf, stl):
        sc.set_instance_transforms(fo.inst_xform, keep_curvature=True)
    kept = _run(st, ctx, sf, 3)
    _same(_run(st, ctx, stl, 3), kept)
    # switching a precomputed scene rebuilds it in full (curvature included) with its last precompute's
    # parameters: back at the first transforms, both give the first results
    sf.set_structure(True)
    stl.set_structure(False)
    _same(_run(st, ctx, sf, 3), ref)
    _same(_run(st, ctx, stl, 3), ref)


def _far_cluster(n_inst, seed, with_empty=False):
    """Tiny sheared, unevenly scaled plants (scale 0.01-0.03) packed in a 0.5 m cube 35 m from the
    emitter, over a ground quad: object-space ray origins are thousands of prototype sizes away, so the
    growth of the object-space boxes (not the prototypes' own padding) keeps the walk conservative.  An
    empty prototype (no triangles) can be instanced as well."""
    rng = np.random.default_rng(seed)
    base = synth.instanced_forest(seed=seed, n_inst=2, n_rays=16, n_mics=4, n_bins=32)
    protos = list(base.protos)
    ground = (np.array([[-5, -5, 0], [40, -5, 0], [40, 40, 0], [-5, 40, 0]], np.float32), protos[0][1], protos[0][2])
    protos[0] = ground
    if with_empty:
        protos.append((np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.int32)))
    C = np.array([25.0, 25.0, 3.0])
    kind, xf = [0], [np.concatenate([np.eye(3), np.zeros((3, 1))], 1)]
    while len(kind) < n_inst:
        q = len(protos) - 1 if (with_empty and len(kind) == 1) else int(rng.integers(1, 4))
        a, e = rng.uniform(0, 2 * np.pi, 2)
        R = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]]) @ \
            np.array([[1, 0, 0], [0, np.cos(e), -np.sin(e)], [0, np.sin(e), np.cos(e)]])
        Sh = np.array([[1, rng.uniform(-0.5, 0.5), 0], [0, 1, rng.uniform(-0.5, 0.5)], [0, 0, 1]])
        A = R @ np.diag(rng.uniform(0.01, 0.03, 3)) @ Sh
        xf.append(np.concatenate([A, (C + rng.uniform(-0.25, 0.25, 3))[:, None]], 1))
        kind.append(q)
    b = base.base
    emitter = np.array([0.0, 0.0, 1.0], np.float32)
    tgt = C + rng.uniform(-0.3, 0.3, (20_000, 3))
    dirs = (tgt - emitter) / np.linalg.norm(tgt - emitter, axis=1, keepdims=True)
    fo = synth.InstancedScene(protos=protos, inst_proto=np.array(kind, np.int32),
                              inst_xform=np.array(xf, np.float64).astype(np.float32),
                              base=dataclasses.replace(b, emitter=emitter, dirs=dirs.astype(np.float32),
                                                       mics=(b.mics - b.mics.mean(0) + np.array([0.5, 0, 1])).astype(np.float32)))
    return fo


@pytest.mark.parametrize("n_inst,with_empty", [(200, False), (3, True), (1, False)])
def test_two_level_far_sheared_instances_and_small_tops(st, n_inst, with_empty):
    """Far, tiny, sheared instances; top levels of one to three instances (a root node holding each
    instance as its own leaf) with an empty prototype among them: two-level results equal flat ones bit
    for bit, with the default and a 1-entry stack."""
    fo = _far_cluster(n_inst, seed=41 + n_inst, with_empty=with_empty)
    ctx = st.Context(0)
    sf = _scene(st, ctx, fo, fo.inst_xform, False, budget=50_000)
    stl = _scene(st, ctx, fo, fo.inst_xform, True, budget=50_000)
    _sensor(ctx, fo.base)
    ref = _run(st, ctx, sf, 3)
    if n_inst >= 100:
        hit_plants = np.isin(ref["paths"]["tri"][:, 0], np.arange(2, sf.n_tris))
        assert hit_plants.sum() > 1000, hit_plants.sum()
    _same(_run(st, ctx, stl, 3), ref)
    ctx.set_tune(stack_depth=1)
    _same(_run(st, ctx, stl, 3), ref)
    ctx.set_tune()


def test_two_level_argument_checks(st):
    fo = synth.instanced_forest(seed=608, n_inst=6, n_rays=256, n_mics=2, n_bins=8)
    b = fo.base
    ctx = st.Context(0)
    L = st.load()
    sc = st.Scene.from_instances(ctx, fo.protos, fo.inst_proto, fo.inst_xform)
    assert L.st_scene_set_structure(sc.h, 2) == st.ST_ERR_ARG
    flat_sc = st.Scene(ctx, *sc.geometry())
    assert L.st_scene_set_structure(flat_sc.h, 1) == st.ST_ERR_STATE
    assert L.st_scene_set_structure(flat_sc.h, 0) == 0
    # a singular map is refused when the two-level structure is built
    X = fo.inst_xform.copy()
    X[3, :, :3] = 0.0
    bad = _scene(st, ctx, fo, fo.inst_xform, True)
    with pytest.raises(st.SonotraceError) as e:
        bad.set_instance_transforms(X)
    assert e.value.status == st.ST_ERR_MESH
    bad.set_instance_transforms(fo.inst_xform)  # finite, invertible maps build it again
    good = _scene(st, ctx, fo, fo.inst_xform, True)
    with pytest.raises(st.SonotraceError) as e:
        good.update_vertices(good.geometry()[0])
    assert e.value.status == st.ST_ERR_STATE
    _sensor(ctx, b)
    job = st.BatchJob(good, b.emitter, b.emitter_quat, b.dirs, b.mics, b.n_bins, b.f_lo, b.f_hi, 2)
    with pytest.raises(st.SonotraceError) as e:
        ctx.simulate_batch([job], st.sim_params(max_distance=60.0))
    assert e.value.status == st.ST_ERR_ARG
    S = ctx.simulate(bad, st.sim_params(max_bounces=2, max_distance=60.0)).cpu().numpy()
    assert np.array_equal(S, ctx.simulate(good, st.sim_params(max_bounces=2, max_distance=60.0)).cpu().numpy())
