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


def test_frequency_grid_array(st):
    """Bins given as an ascending, uniformly spaced array give the spectra of the same grid given by its
    ends, bit for bit; a non-uniform, descending or empty array is rejected and the context keeps its
    grid."""
    wl = synth.clutter(seed=31, target_tris=3000, n_rays=2000, bounces=3, n_mics=4, n_bins=37)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=20_000))
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    S_ref = ctx.simulate(sc, p).cpu().numpy()
    f = np.linspace(wl.f_lo, wl.f_hi, wl.n_bins)
    ctx.set_frequency_grid(f.astype(np.float32))
    assert np.array_equal(ctx.simulate(sc, p).cpu().numpy(), S_ref)
    g = f.copy()
    g[5] += 0.3 * (f[1] - f[0])
    assert status_of(st, ctx.set_frequency_grid, g) == st.ST_ERR_ARG
    assert status_of(st, ctx.set_frequency_grid, f[::-1].copy()) == st.ST_ERR_ARG
    assert status_of(st, ctx.set_frequency_grid, np.zeros(0, np.float32)) == st.ST_ERR_ARG
    assert np.array_equal(ctx.simulate(sc, p).cpu().numpy(), S_ref)
    ctx.set_frequency_grid(np.array([wl.f_lo], np.float32))
    assert ctx.simulate(sc, p).shape == (3, len(wl.mics), 1)


def test_injected_allocation_failure(st):
    """A device allocation that fails (injected on the host: the allocator returns the out-of-memory
    error without allocating) makes the call that needs it return ST_ERR_OOM; the context then still
    works, and its spectra equal a fresh context's bit for bit."""
    L = st.load()
    wl = synth.clutter(seed=31, target_tris=3000, n_rays=3000, bounces=3, n_mics=4, n_bins=32)
    try:
        ctx = st.Context(0)
        sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=20_000))
        p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
        for after in (0, 1, 3, 7):
            L.st_inject_alloc_failure(after)
            ctx2 = st.Context(0)
            try:
                sc2 = st.from_workload(ctx2, wl, st.curv_params(sample_budget=20_000))
                code = status_of(st, ctx2.simulate, sc2, p)
            except st.SonotraceError as e:  # the failure hit the scene load or precompute
                code = e.status
            L.st_inject_alloc_failure(-1)
            assert code == st.ST_ERR_OOM, (after, code)
        # a simulate that needs larger buffers than the last one fails at its first allocation ...
        wl2 = synth.clutter(seed=31, target_tris=3000, n_rays=9000, bounces=3, n_mics=4, n_bins=32)
        ctx.set_emitter(wl2.emitter, wl2.emitter_quat, wl2.dirs)
        L.st_inject_alloc_failure(0)
        assert status_of(st, ctx.simulate, sc, p) == st.ST_ERR_OOM
        L.st_inject_alloc_failure(-1)
        # ... and the next one, with nothing injected, regrows them and gives the fresh context's spectra
        S = ctx.simulate(sc, p).cpu().numpy()
        fresh = st.Context(0)
        scf = st.from_workload(fresh, wl2, st.curv_params(sample_budget=20_000))
        assert np.array_equal(S, fresh.simulate(scf, p).cpu().numpy())
    finally:
        L.st_inject_alloc_failure(-1)


def test_log_levels(tmp_path):
    """ST_LOG=1 writes every error to stderr, ST_LOG=2 also one line per simulate and precompute; unset, the
    library writes nothing (checked in child processes: the level is read once per process)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "run.py"
    script.write_text(
        "import sys\n"
        f"sys.path[:0] = [{root!r}, {os.path.join(root, 'tests')!r}]\n"
        "import numpy as np, paper_2602_19652_gb300 as st, synth\n"
        "ctx = st.Context(0)\n"
        "wl = synth.shoebox(seed=101, n_rays=500)\n"
        "try:\n"
        "    ctx.simulate(st.Scene(ctx, wl.verts, wl.tris, wl.tri_mat, wl.tri_obj))\n"
        "except st.SonotraceError:\n"
        "    pass\n"
        "sc = st.from_workload(ctx, wl)\n"
        "ctx.simulate(sc)\n")
    out = {}
    for level in (None, "1", "2"):
        env = dict(os.environ)
        env.pop("ST_LOG", None)
        if level:
            env["ST_LOG"] = level
        r = subprocess.run([sys.executable, str(script)], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        out[level] = [l for l in r.stderr.splitlines() if l.startswith("sonotrace:")]
    assert out[None] == []
    assert any("error" in l and "simulate" in l for l in out["1"]) and not any("simulate: " in l and "rays" in l
                                                                              for l in out["1"])
    assert any("precompute:" in l for l in out["2"]) and any("rays x" in l for l in out["2"])


def test_scene_checkpoint_resume(st):
    """A precomputed scene serialised to a host blob and restored in another context (no precompute)
    gives the same path records, diffraction samples, curvature and spectra bit for bit; a truncated, a
    modified and a foreign blob are refused on the host; instanced and unprecomputed scenes are refused."""
    import ctypes as C
    wl = synth.clutter(seed=41, target_tris=6000, n_rays=4000, bounces=3, n_mics=8, n_bins=64)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, st.curv_params(sample_budget=30_000))
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    S0 = ctx.simulate(sc, p).cpu().numpy()
    P0, D0 = ctx.paths(wl.bounces), ctx.diffraction()
    G0 = sc.curvature()
    blob = sc.serialize()
    ctx2 = st.Context(0)
    sc2 = st.Scene.deserialize(ctx2, blob)
    ctx2.set_frequencies(wl.n_bins, wl.f_lo, wl.f_hi)
    ctx2.set_emitter(wl.emitter, wl.emitter_quat, wl.dirs, None, wl.fov_half)
    ctx2.set_receivers(wl.mics)
    S1 = ctx2.simulate(sc2, p).cpu().numpy()
    assert np.array_equal(S0, S1)
    P1, D1 = ctx2.paths(wl.bounces), ctx2.diffraction()
    for k in P0:
        assert np.array_equal(P0[k], P1[k]), k
    for a, b in zip(D0, D1):
        assert np.array_equal(a, b)
    for a, b in zip(G0, sc2.curvature()):
        assert np.array_equal(a, b)
    assert sc2.serialize() == blob
    # the restored scene refits like the original
    v = sc.geometry()[0] + np.float32(0.01)
    sc.update_vertices(v)
    sc2.update_vertices(v)
    assert np.array_equal(ctx.simulate(sc, p).cpu().numpy(), ctx2.simulate(sc2, p).cpu().numpy())
    L = st.load()
    h = C.c_void_p()
    bad = bytearray(blob)
    bad[len(bad) // 2] ^= 1
    for b in (blob[: len(blob) - 8], bytes(bad), b"XXXX" + blob[4:]):
        buf = C.create_string_buffer(bytes(b), len(b))
        assert L.st_scene_deserialize(ctx2.h, buf, len(b), C.byref(h)) == st.ST_ERR_ARG
    n = C.c_size_t(16)
    small = C.create_string_buffer(16)
    assert L.st_scene_serialize(sc.h, small, C.byref(n)) == st.ST_ERR_ARG and n.value == len(blob)
    raw = st.Scene(ctx, wl.verts, wl.tris, wl.tri_mat, wl.tri_obj)
    assert L.st_scene_serialize(raw.h, None, C.byref(n)) == st.ST_ERR_STATE
    fo = synth.instanced_forest(seed=609, n_inst=4, n_rays=64, n_mics=2, n_bins=8)
    inst = st.Scene.from_instances(ctx, fo.protos, fo.inst_proto, fo.inst_xform)
    inst.set_materials(fo.base.band_hz, fo.base.k_band, fo.base.beta_band, fo.base.diff_band)
    inst.precompute()
    assert L.st_scene_serialize(inst.h, None, C.byref(n)) == st.ST_ERR_STATE
