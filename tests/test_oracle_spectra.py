"""Pins for the oracle's spectrum synthesis (Eq. 2-4, 7-8, 11-12) and its analytic gradient.

Expected values below are derived by hand from the construction (distances of 3-4-5 style
geometry, angles of 0 and 45 degrees, absorption chosen to give a factor 0.1, band values that
interpolate to round numbers), not by re-running the oracle's formulas."""
import math

import numpy as np
import pytest

import oracle
import synth

C_SOUND = 343.0


def _slab_workload(k_floor, k_ceil, band_hz, beta, F, f_lo, f_hi, mics, emitter=(0.0, 0.0, 3.0)):
    """Floor z=0 (material 0) and ceiling z=5 (material 1), 40 x 40 m."""
    V = np.array([[-20, -20, 0], [20, -20, 0], [20, 20, 0], [-20, 20, 0],
                  [-20, -20, 5], [20, -20, 5], [20, 20, 5], [-20, 20, 5]], np.float32)
    T = np.array([[0, 1, 2], [0, 2, 3], [4, 6, 5], [4, 7, 6]], np.int32)
    nb = len(band_hz)
    return synth.Workload(
        name="slab", verts=V, tris=T, tri_mat=np.array([0, 0, 1, 1], np.int32), tri_obj=np.zeros(4, np.int32),
        band_hz=np.asarray(band_hz, np.float32),
        k_band=np.array([k_floor, k_ceil], np.float32),
        beta_band=np.full((2, nb), beta, np.float32), diff_band=np.full((2, nb), 0.05, np.float32),
        emitter=np.asarray(emitter, np.float32), emitter_quat=np.array([1, 0, 0, 0], np.float32),
        dirs=np.array([[0, 0, -1]], np.float32), mics=np.asarray(mics, np.float32),
        n_bins=F, f_lo=f_lo, f_hi=f_hi, bounces=2)


def test_single_path_closed_form_and_band_interpolation():
    band = [20e3, 40e3, 80e3]
    wl = _slab_workload([0.25, 0.5, 1.0], [0.5, 0.5, 0.5], band, math.pi / 4, 9, 10e3, 90e3,
                        mics=[[0.0, 0.0, 1.0]])
    wl.bounces = 1
    out = oracle.simulate(wl, a0=5.0, a1_per_khz=0.0, components=1)
    S = out["spectra"][0, 0]
    f = 10e3 + 10e3 * np.arange(9)
    k_expect = np.array([0.25, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 1.0, 1.0])  # clamped / linear between centres
    r = 4.0                                   # 3 m down, 1 m up to the microphone; gamma = 0
    expect = k_expect / 16.0 * 0.1 * np.exp(1j * 2 * np.pi * f * r / C_SOUND)   # 10^(-5*4/20) = 0.1
    assert np.allclose(S, expect, rtol=1e-12, atol=0)


def test_lobe_angle_45_degrees():
    wl = _slab_workload([1.0], [1.0], [40e3], math.pi / 4, 3, 20e3, 60e3, mics=[[1.0, 0.0, 1.0]])
    wl.bounces = 1
    out = oracle.simulate(wl, a0=0.0, a1_per_khz=0.0, components=1)
    S = out["spectra"][0, 0]
    f = np.array([20e3, 40e3, 60e3])
    r = 3.0 + math.sqrt(2.0)
    beta32 = float(np.float32(math.pi / 4))   # the band table is float32
    lobe = math.exp(-(math.pi / 4) ** 2 / (2 * beta32 ** 2))   # gamma = 45 degrees
    expect = lobe / r ** 2 * np.exp(1j * 2 * np.pi * f * r / C_SOUND)
    assert np.allclose(S, expect, rtol=1e-12, atol=0)


@pytest.mark.parametrize("mode", [0, 1])
def test_two_bounces_cumulative_reflection(mode):
    wl = _slab_workload([0.5], [0.75], [40e3], 0.3, 2, 30e3, 50e3, mics=[[0.0, 0.0, 1.0]])
    out = oracle.simulate(wl, a0=0.0, a1_per_khz=0.0, components=1, reflection_mode=mode)
    rec = out["rec"]
    assert list(rec["tri"][0] >= 0) == [True, True]
    assert list(rec["r"][0]) == [3.0, 8.0]
    S = out["spectra"][0, 0]
    f = np.array([30e3, 50e3])
    k2 = 0.5 * 0.75 if mode == 0 else 0.75
    expect = 0.5 / 16.0 * np.exp(2j * np.pi * f * 4.0 / C_SOUND) + k2 / 144.0 * np.exp(2j * np.pi * f * 12.0 / C_SOUND)
    assert np.allclose(S, expect, rtol=1e-12, atol=0)


def test_direct_path_closed_form_and_occlusion():
    wl = _slab_workload([1.0], [1.0], [40e3], 0.3, 4, 20e3, 80e3,
                        mics=[[3.0, 4.0, 3.0], [0.0, 0.0, 7.0]], emitter=(0.0, 0.0, 3.0))
    out = oracle.simulate(wl, a0=2.0, a1_per_khz=0.1, components=4, direct_gain=2.0)
    S = out["spectra"][2]
    f = 20e3 + 20e3 * np.arange(4)
    alpha = 2.0 + 0.1 * f / 1000.0
    r = 5.0
    expect = 2.0 / 25.0 * 10 ** (-alpha * r / 20) * np.exp(2j * np.pi * f * r / C_SOUND)
    assert np.allclose(S[0], expect, rtol=1e-12)
    assert np.all(S[1] == 0)                  # behind the ceiling: occluded


def test_diffraction_reciprocity():
    """Swapping emitter and a single microphone leaves the diffraction spectrum unchanged
    (r = |s - o| + |o - m| is symmetric) when both see the same candidates."""
    wl = synth.clutter(seed=21, target_tris=4000, n_rays=1, n_mics=1, n_bins=32)
    wl.mics = np.array([[8.0, 9.0, 1.5]], np.float32)
    G = oracle.curvature(wl.verts, wl.tris)
    Cm = oracle.tri_metric(wl.verts, wl.tris, G)
    cd = oracle.diffraction_cdf(wl.verts, wl.tris, Cm, wl.tri_obj, seed=3)
    ct, cp = oracle.diffraction_samples(wl.verts, wl.tris, cd, seed=4)
    sc = oracle.Scene(wl.verts, wl.tris)
    k1 = oracle.diffraction_filter(sc, wl.emitter, wl.emitter_quat, ct, cp, cos_inc=0.0)
    k2 = oracle.diffraction_filter(sc, wl.mics[0], wl.emitter_quat, ct, cp, cos_inc=0.0)
    keep = (k1 & k2).astype(np.uint8)
    assert keep.sum() > 50
    empty = dict(tri=np.full((1, 1), -1, np.int32), p=np.zeros((1, 1, 3), np.float32),
                 d=np.zeros((1, 1, 3), np.float32), r=np.zeros((1, 1)), los=np.zeros((1, 1), np.uint8))
    pa = oracle.spec_params(wl)
    Sa = oracle.spectra(pa, empty, wl.dirs, wl.tri_mat, ct, cp, keep)
    pb = oracle.spec_params(wl, mics=wl.emitter[None, :], emitter=wl.mics[0])
    Sb = oracle.spectra(pb, empty, wl.dirs, wl.tri_mat, ct, cp, keep)
    assert np.abs(Sa[1]).max() > 0
    assert np.allclose(Sa[1], Sb[1], rtol=1e-12, atol=1e-12 * np.abs(Sa[1]).max())


def test_zero_absorption_invariants():
    """k = 1, no air absorption, a closed room: every ray yields B visible records and the
    specular spectrum at any bin is bounded by sum 1/r^2 (each term has |lobe| <= 1)."""
    wl = synth.shoebox(seed=5, n_rays=400, bounces=4, absorption=0.0, beta_deg=1e4)
    out = oracle.simulate(wl, a0=0.0, a1_per_khz=0.0, components=1)
    rec = out["rec"]
    assert (rec["tri"] >= 0).all() and (rec["los"] == 1).all()
    r = rec["r"] + np.linalg.norm(rec["p"].astype(np.float64) - wl.mics[0].astype(np.float64), axis=-1)
    bound = np.sum(1.0 / r ** 2)
    S = out["spectra"][0, 0]
    assert np.all(np.abs(S) <= bound * (1 + 1e-12))
    # with beta -> infinity the lobe is 1: at f -> 0 every term is 1/r^2 in phase
    assert abs(np.abs(S[0]) - bound) / bound < 1.0


def _grad_problem(n_rays=300, F=12):
    wl = synth.gradient_problem(seed=404, n_rays=n_rays)
    wl.n_bins = F
    out = oracle.simulate(wl, components=5)
    # a few diffraction candidates on the walls, kept
    rng = np.random.default_rng(0)
    ct = rng.integers(0, 12, 20).astype(np.int32)
    V, T = wl.verts, wl.tris
    a, b = rng.uniform(0, 0.5, 20), rng.uniform(0, 0.5, 20)
    cp = (V[T[ct, 0]] + a[:, None] * (V[T[ct, 1]] - V[T[ct, 0]]) + b[:, None] * (V[T[ct, 2]] - V[T[ct, 0]])).astype(np.float32)
    keep = np.ones(20, np.uint8)
    return wl, out, ct, cp, keep


def test_gradient_matches_central_differences():
    """Analytic float64 gradient vs central differences with Richardson extrapolation on 20 random
    directions.  The base point and every perturbed point are exactly representable in float32
    (the interface precision), so the differences are exact float64 evaluations."""
    wl, out, ct, cp, keep = _grad_problem()
    rec, dv = out["rec"], out["direct_vis"]
    q = lambda x, e: np.round(np.asarray(x, np.float64) * 2.0 ** e) / 2.0 ** e
    k0, m0, s0 = q(wl.k_band, 12), q(wl.mics, 12), q(wl.emitter, 12)
    rng = np.random.default_rng(404)

    def spectra_at(k, m, s):
        for a in (k, m, s):
            assert np.array_equal(a.astype(np.float32).astype(np.float64), a)
        p = oracle.spec_params(wl, mics=m.astype(np.float32), k_band=k.astype(np.float32), emitter=s.astype(np.float32))
        return oracle.spectra(p, rec, wl.dirs, wl.tri_mat, ct, cp, keep, dv)

    S0 = spectra_at(k0, m0, s0)
    St = spectra_at(q(k0 * 0.9, 12), m0 + 2.0 ** -7, s0 - 2.0 ** -7)
    G = 2.0 * (S0 - St)
    p = oracle.spec_params(wl, mics=m0.astype(np.float32), k_band=k0.astype(np.float32), emitter=s0.astype(np.float32))
    dk, dmic, demit = oracle.spectra_grad(p, rec, wl.dirs, wl.tri_mat, G, ct, cp, keep, dv)
    assert np.abs(dk).max() > 0 and np.abs(dmic).max() > 0 and np.abs(demit).max() > 0

    def loss(k, m, s):
        return float(np.sum(np.abs(spectra_at(k, m, s) - St) ** 2))

    for _ in range(20):
        vk = q(rng.uniform(-1, 1, k0.shape), 5)
        vm = q(rng.uniform(-1, 1, m0.shape), 5)
        vs = q(rng.uniform(-1, 1, 3), 5)

        def D(h_k, h_x):
            return (loss(k0 + h_k * vk, m0 + h_x * vm, s0 + h_x * vs)
                    - loss(k0 - h_k * vk, m0 - h_x * vm, s0 - h_x * vs)) / 2.0

        hk, hx = 2.0 ** -10, 2.0 ** -16
        # D(t w) = t grad.w + c t^3 + O(t^5)  =>  (8 D(w/2) - D(w)) / 3 = grad.w + O(|w|^5)
        fd = (8.0 * D(hk / 2, hx / 2) - D(hk, hx)) / 3.0
        terms = np.concatenate([(dk * hk * vk).ravel(), (dmic * hx * vm).ravel(), demit * hx * vs])
        an = terms.sum()
        assert abs(fd - an) <= 1e-6 * np.abs(terms).sum(), (fd, an)


def test_gradient_with_microphone_masks_matches_central_differences():
    """The per-microphone receiver test: records with random microphone masks (each record reaches only
    the microphones whose bit is set, in the spectra and in the gradient).  The reflection, microphone and
    lobe-width gradients against central differences of the masked spectra, the emitter gradient through
    the hit points against those of the masked frozen-chain restatement, Richardson extrapolated; a
    gradient that ignored the masks would differ from them."""
    wl, out, _, _, _ = _grad_problem()
    rec = dict(out["rec"])
    M = len(wl.mics)
    rng = np.random.default_rng(406)
    hit_vis = (rec["tri"] >= 0) & (rec["los"] != 0)
    mask = np.where(hit_vis, rng.integers(0, 1 << M, rec["tri"].shape, dtype=np.uint64), 0).astype(np.uint64)
    rec["mask"], rec["los"] = mask, (mask != 0).astype(np.uint8)
    full = np.uint64((1 << M) - 1)
    assert np.sum((mask != 0) & (mask != full)) > 100
    nrm = oracle.tri_normals(wl.verts, wl.tris)
    q = lambda x, e: np.round(np.asarray(x, np.float64) * 2.0 ** e) / 2.0 ** e
    k0, m0, s0, b0 = q(wl.k_band, 12), q(wl.mics, 12), q(wl.emitter, 12), q(wl.beta_band, 14)

    def spectra_at(k, m, s, b):
        for a in (k, m, s, b):
            assert np.array_equal(a.astype(np.float32).astype(np.float64), a)
        p = oracle.spec_params(wl, mics=m.astype(np.float32), k_band=k.astype(np.float32),
                               emitter=s.astype(np.float32), beta_band=b.astype(np.float32))
        return oracle.spectra(p, rec, wl.dirs, wl.tri_mat)

    # the masks change the spectra (a mask-blind sum would differ)
    full_rec = dict(rec, mask=np.where(mask != 0, full, np.uint64(0)).astype(np.uint64))
    p0 = oracle.spec_params(wl)
    assert not np.allclose(oracle.spectra(p0, rec, wl.dirs, wl.tri_mat)[0],
                           oracle.spectra(p0, full_rec, wl.dirs, wl.tri_mat)[0])
    S0 = spectra_at(k0, m0, s0, b0)
    St = spectra_at(q(k0 * 0.9, 12), m0 + 2.0 ** -7, s0 - 2.0 ** -7, q(b0 * 1.2, 14))
    G = 2.0 * (S0 - St)
    p = oracle.spec_params(wl, mics=m0.astype(np.float32), k_band=k0.astype(np.float32),
                           emitter=s0.astype(np.float32), beta_band=b0.astype(np.float32))
    dk, dmic, _, dbeta = oracle.spectra_grad(p, rec, wl.dirs, wl.tri_mat, G, with_beta=True)
    assert np.abs(dk).max() > 0 and np.abs(dmic).max() > 0 and np.abs(dbeta).max() > 0

    def loss(k, m, s, b):
        return float(np.sum(np.abs(spectra_at(k, m, s, b) - St) ** 2))

    for _ in range(6):
        vk = q(rng.uniform(-1, 1, k0.shape), 5)
        vm = q(rng.uniform(-1, 1, m0.shape), 5)
        vb = q(rng.uniform(-1, 1, b0.shape), 5)

        def D(h_k, h_x, h_b):
            return (loss(k0 + h_k * vk, m0 + h_x * vm, s0, b0 + h_b * vb)
                    - loss(k0 - h_k * vk, m0 - h_x * vm, s0, b0 - h_b * vb)) / 2.0

        hk, hx, hb = 2.0 ** -10, 2.0 ** -16, 2.0 ** -12
        fd = (8.0 * D(hk / 2, hx / 2, hb / 2) - D(hk, hx, hb)) / 3.0
        terms = np.concatenate([(dk * hk * vk).ravel(), (dmic * hx * vm).ravel(), (dbeta * hb * vb).ravel()])
        assert abs(fd - terms.sum()) <= 1e-6 * np.abs(terms).sum(), (fd, terms.sum())
    # the emitter through the hit points: central differences of the masked frozen-chain restatement, which
    # at the stored emitter reproduces the oracle's masked spectra
    se = wl.emitter.astype(np.float64)
    spec = lambda s_: _frozen_chain_spectra(wl, rec, s_, s_ref=se)
    Se = spec(se)
    Sref = oracle.spectra(oracle.spec_params(wl), rec, wl.dirs, wl.tri_mat)[0]
    assert np.linalg.norm(Se - Sref) <= 1e-9 * np.linalg.norm(Sref)
    Ste = spec(se + np.array([0.01, -0.02, 0.015]))
    Ge = np.zeros((3,) + Se.shape, np.complex128)
    Ge[0] = 2.0 * (Se - Ste)
    _, _, demit_s = oracle.spectra_grad(oracle.spec_params(wl), rec, wl.dirs, wl.tri_mat, Ge, tri_nrm=nrm)
    assert np.abs(demit_s).max() > 0
    for _ in range(3):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)

        def Ds(h):
            return (np.sum(np.abs(spec(se + h * v) - Ste) ** 2) - np.sum(np.abs(spec(se - h * v) - Ste) ** 2)) / 2.0

        h = 1e-4
        fd = (8.0 * Ds(h / 2) - Ds(h)) / 3.0
        an = float(demit_s @ (h * v))
        assert abs(fd - an) <= 1e-4 * np.abs(demit_s * h * v).sum() + 1e-12, (fd, an)


def test_beta_gradient_matches_central_differences():
    """Lobe-width gradient (specular paths, the last hit's material) vs central differences with
    Richardson extrapolation; beta values and steps exactly representable in float32."""
    wl, out, ct, cp, keep = _grad_problem()
    rec = out["rec"]
    q = lambda x, e: np.round(np.asarray(x, np.float64) * 2.0 ** e) / 2.0 ** e
    b0 = q(wl.beta_band, 14)
    rng = np.random.default_rng(405)

    def spectra_at(b):
        assert np.array_equal(b.astype(np.float32).astype(np.float64), b)
        p = oracle.spec_params(wl, beta_band=b.astype(np.float32))
        return oracle.spectra(p, rec, wl.dirs, wl.tri_mat)

    S0 = spectra_at(b0)
    St = spectra_at(q(b0 * 1.2, 14))
    G = 2.0 * (S0 - St)
    p = oracle.spec_params(wl, beta_band=b0.astype(np.float32))
    _, _, _, dbeta = oracle.spectra_grad(p, rec, wl.dirs, wl.tri_mat, G, with_beta=True)
    assert np.abs(dbeta).max() > 0

    def loss(b):
        return float(np.sum(np.abs(spectra_at(b) - St) ** 2))

    for _ in range(10):
        v = q(rng.uniform(-1, 1, b0.shape), 5)

        def D(h):
            return (loss(b0 + h * v) - loss(b0 - h * v)) / 2.0

        h = 2.0 ** -12
        fd = (8.0 * D(h / 2) - D(h)) / 3.0
        terms = (dbeta * h * v).ravel()
        assert abs(fd - terms.sum()) <= 1e-6 * np.abs(terms).sum(), (fd, terms.sum())


def _rot32(q, v):
    """q applied to v in float32 with the tracing's operation order (no fused products)."""
    f = np.float32
    q = [f(x) for x in q]
    v = [f(x) for x in v]
    t = [f(2.0) * (q[2] * v[2] - q[3] * v[1]), f(2.0) * (q[3] * v[0] - q[1] * v[2]), f(2.0) * (q[1] * v[1] - q[2] * v[0])]
    c = [q[2] * t[2] - q[3] * t[1], q[3] * t[0] - q[1] * t[2], q[1] * t[1] - q[2] * t[0]]
    return np.array([(v[k] + q[0] * t[k]) + c[k] for k in range(3)], np.float64)


def _frozen_chain_spectra(wl, rec, s, a1_per_khz=0.033, c=343.0, s_ref=None):
    """Specular spectra in float64 with every record's triangle chain and ray direction frozen and its
    hit points re-intersected from the emitter position s (the plain formula of Eq. 2-4, reflection
    product over the chain, lobe of the last hit).  With s_ref, hit points and lengths are the stored
    records' plus the float64 displacement between the intersections from s and from s_ref (the
    records are float32: at s_ref this reproduces them exactly)."""
    F = wl.n_bins
    f = wl.f_lo + np.arange(F) * ((wl.f_hi - wl.f_lo) / (F - 1))
    band = wl.band_hz.astype(np.float64)
    b0 = np.clip(np.searchsorted(band, f, side="right") - 1, 0, len(band) - 2)
    w = np.clip((f - band[b0]) / (band[b0 + 1] - band[b0]), 0.0, 1.0)
    kb, bb = wl.k_band.astype(np.float64), wl.beta_band.astype(np.float64)
    kf = (1 - w) * kb[:, b0] + w * kb[:, b0 + 1]                       # [n_mat][F]
    gf = (1 - w) / (2 * bb[:, b0] ** 2) + w / (2 * bb[:, b0 + 1] ** 2)
    alpha = a1_per_khz * f / 1000.0
    V = wl.verts.astype(np.float64)
    nrm = oracle.tri_normals(wl.verts, wl.tris).astype(np.float64)
    M = len(wl.mics)
    S = np.zeros((M, F), np.complex128)
    N, B = rec["tri"].shape
    for i in range(N):
        Pq = np.asarray(s, np.float64)
        Pb = np.asarray(s if s_ref is None else s_ref, np.float64)
        d = _rot32(wl.emitter_quat, wl.dirs[i])
        r, rb, chain = 0.0, 0.0, []
        for j in range(B):
            tri = rec["tri"][i, j]
            if tri < 0:
                break
            n = nrm[tri]
            t = n @ (V[wl.tris[tri, 0]] - Pq) / (n @ d)
            tb = n @ (V[wl.tris[tri, 0]] - Pb) / (n @ d)
            Pq, Pb = Pq + t * d, Pb + tb * d
            r, rb = r + t, rb + tb
            chain.append(wl.tri_mat[tri])
            d = rec["d"][i, j].astype(np.float64)
            if not rec["los"][i, j]:
                continue
            kprod = np.prod(kf[chain], axis=0)
            Pu, ru = Pq, r
            if s_ref is not None:
                Pu = rec["p"][i, j].astype(np.float64) + (Pq - Pb)
                ru = float(rec["r"][i, j]) + (r - rb)
            for m in range(M):
                if "mask" in rec and not (int(rec["mask"][i, j]) >> m) & 1:
                    continue  # per-microphone receiver test: microphone m does not see this hit
                v = wl.mics[m].astype(np.float64) - Pu
                dist = np.linalg.norm(v)
                u = v / dist
                gm = math.atan2(np.linalg.norm(np.cross(d, u)), d @ u)
                rr = ru + dist
                A = np.exp(-gm * gm * gf[chain[-1]]) * kprod * 10.0 ** (-alpha * rr / 20.0) / rr ** 2
                S[m] += A * np.exp(2j * np.pi * f * rr / c)
    return S


def test_specular_emitter_gradient_matches_central_differences():
    """Emitter-position gradient through the specular hit points (chains and directions frozen)
    against central differences of a float64 frozen-chain restatement, Richardson extrapolated."""
    wl, out, _, _, _ = _grad_problem(n_rays=200, F=10)
    rec = out["rec"]
    s0 = wl.emitter.astype(np.float64)
    spec = lambda s: _frozen_chain_spectra(wl, rec, s, s_ref=s0)
    S0 = spec(s0)
    # at s0 the restatement reproduces the oracle's spectra from the stored records
    Sref = oracle.spectra(oracle.spec_params(wl), rec, wl.dirs, wl.tri_mat)[0]
    assert np.linalg.norm(S0 - Sref) <= 1e-9 * np.linalg.norm(Sref)
    # the re-intersection from s0 itself lands on the stored hit points (float32 rounding apart)
    S_raw = _frozen_chain_spectra(wl, rec, s0)
    assert np.linalg.norm(S_raw - Sref) <= 1e-3 * np.linalg.norm(Sref)
    St = spec(s0 + np.array([0.01, -0.02, 0.015]))
    G = np.zeros((3,) + S0.shape, np.complex128)
    G[0] = 2.0 * (S0 - St)
    nrm = oracle.tri_normals(wl.verts, wl.tris)
    _, _, demit = oracle.spectra_grad(oracle.spec_params(wl), rec, wl.dirs, wl.tri_mat, G, tri_nrm=nrm)
    assert np.abs(demit).max() > 0

    def loss(s):
        return float(np.sum(np.abs(spec(s) - St) ** 2))

    rng = np.random.default_rng(406)
    for _ in range(3):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)

        def D(h):
            return (loss(s0 + h * v) - loss(s0 - h * v)) / 2.0

        h = 1e-4
        fd = (8.0 * D(h / 2) - D(h)) / 3.0
        an = float(demit @ (h * v))
        assert abs(fd - an) <= 1e-4 * np.abs(demit * h * v).sum() + 1e-12, (fd, an)
