"""Parity at the benchmark's full size and launch configuration (the clutter workload: ~200k
triangles, 1M rays x 5 bounces, 4M diffraction samples, 32 mics x 512 bins).

The oracle traces every ray with its own BVH (multi-threaded) and draws and filters every
diffraction sample, so path sets and samples are compared in full, bit for bit; the spectra are
compared on a sample of (microphone, bin) outputs that the oracle evaluates one by one over all
paths."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2602_19652_gb300 as st
    wl = synth.clutter(seed=202)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    S, stats = ctx.simulate(sc, p, stats=True)
    S = S.cpu().numpy()
    g = ctx.paths(wl.bounces)
    gd = ctx.diffraction()
    gv = ctx.direct_visibility()
    # microphones across the pair and tile boundaries, bins at the edges of bin tiles and chain runs
    ms = np.array([0, 5, 13, 16, 17, 31], np.int32)
    ks = np.array([0, 1, 15, 16, 127, 128, 200, 255, 256, 377, 500, 511], np.int32)
    o = oracle.simulate(wl, ms=ms, ks=ks)
    return dict(wl=wl, S=S, stats=stats, g=g, gd=gd, gv=gv, o=o, ms=ms, ks=ks)


def test_full_path_set_bit_exact(run):
    g, o = run["g"], run["o"]["rec"]
    for k in ("tri", "los", "p", "d", "r"):
        a, b = g[k], o[k]
        bad = np.argwhere(~(a == b).reshape(len(a), -1).all(1)).ravel()
        assert len(bad) == 0, f"{k}: {len(bad)} of {len(a)} rays differ (first {bad[:5]})"
    assert run["stats"].visible_records == int(((o["tri"] >= 0) & (o["los"] == 1)).sum())


def test_full_diffraction_samples_bit_exact(run):
    ct, cp, keep = run["gd"]
    o = run["o"]
    assert len(ct) == len(o["cand_tri"]) > 1_000_000
    assert np.array_equal(ct, o["cand_tri"])
    assert np.array_equal(cp, o["cand_p"])
    assert np.array_equal(keep, o["cand_keep"])
    assert np.array_equal(run["gv"], o["direct_vis"])


def test_full_spectra_sampled_outputs(run):
    S, o, ms, ks = run["S"], run["o"]["spectra"], run["ms"], run["ks"]
    for c in range(3):
        a = S[c][np.ix_(ms, ks)]
        b = o[c]
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= TOL, (c, err)


@pytest.fixture(scope="module")
def veg():
    """The vegetation workload at full size: ~2M leaf triangles, 4M rays x 4 bounces, piston emitter
    table, two directional ears, 1024 bins 20-120 kHz, diffraction with the field-of-view filter."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2602_19652_gb300 as st
    wl = synth.vegetation(seed=303)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    S, stats = ctx.simulate(sc, p, stats=True)
    S = S.cpu().numpy()
    g = ctx.paths(wl.bounces)
    gd = ctx.diffraction()
    ms = np.array([0, 1], np.int32)
    ks = np.array([0, 1, 15, 16, 255, 256, 333, 511, 512, 700, 1000, 1023], np.int32)
    o = oracle.simulate(wl, ms=ms, ks=ks)
    return dict(wl=wl, S=S, stats=stats, g=g, gd=gd, o=o, ms=ms, ks=ks)


def test_vegetation_full_path_set_and_samples_bit_exact(veg):
    g, o = veg["g"], veg["o"]["rec"]
    assert veg["wl"].n_tris > 1_900_000 and len(g["tri"]) == 4_000_000
    for k in ("tri", "los", "p", "d", "r"):
        a, b = g[k], o[k]
        bad = np.argwhere(~(a == b).reshape(len(a), -1).all(1)).ravel()
        assert len(bad) == 0, f"{k}: {len(bad)} of {len(a)} rays differ (first {bad[:5]})"
    ct, cp, keep = veg["gd"]
    assert np.array_equal(ct, veg["o"]["cand_tri"])
    assert np.array_equal(cp, veg["o"]["cand_p"])
    assert np.array_equal(keep, veg["o"]["cand_keep"])
    assert 0 < keep.sum() < len(keep)


def test_vegetation_full_spectra_sampled_outputs(veg):
    S, o, ms, ks = veg["S"], veg["o"]["spectra"], veg["ms"], veg["ks"]
    for c in range(3):
        a = S[c][np.ix_(ms, ks)]
        b = o[c]
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= TOL, (c, err)
