"""The allocation-free accumulation entry point, for callers that cannot allocate device memory
(fixed arenas owned by another allocator, real-time loops, callbacks where allocation is not
allowed).  It must give the specular spectrum of st_simulate, from the same path records, within
the parity tolerance, on consecutive calls that share its fixed scratch -- at the largest chain
length it accepts and in both reflection modes -- and the oracle's specular spectrum as well.
Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("bounces,reflection_mode", [(3, 0), (3, 1), (8, 0), (8, 1)])
def test_noalloc_matches_simulate_and_oracle_on_two_calls(bounces, reflection_mode):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st
    L = st.load()
    # the differentiation workload's room (four wall materials, 32-mic disc, 128 bins)
    wl = synth.shoebox(seed=404, n_rays=2000, bounces=bounces, n_bins=128, n_mics=32, four_materials=True)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, components=st.ST_COMP_SPECULAR,
                      reflection_mode=reflection_mode)
    ref = ctx.simulate(sc, p)[0].cpu().numpy()
    torch.cuda.synchronize()
    ora = oracle.simulate(wl, reflection_mode=reflection_mode, components=1)["spectra"][0]
    N, B, M, F = len(wl.dirs), wl.bounces, len(wl.mics), wl.n_bins
    dev = torch.device("cuda", 0)
    tri = torch.empty((N, B), dtype=torch.int32, device=dev)
    pt = torch.empty((N, B, 3), dtype=torch.float32, device=dev)
    dr = torch.empty((N, B, 3), dtype=torch.float32, device=dev)
    r = torch.empty((N, B), dtype=torch.float64, device=dev)
    los = torch.empty((N, B), dtype=torch.uint8, device=dev)
    vp = lambda t: C.c_void_p(t.data_ptr())
    st.check(L.st_get_paths(ctx.h, vp(tri), vp(pt), vp(dr), vp(r), vp(los), st.ST_MEM_DEVICE), ctx.h)
    assert int((tri[:, B - 1] >= 0).sum()) > 0, "no path reaches the last bounce"
    tri_mat = torch.as_tensor(wl.tri_mat, dtype=torch.int32, device=dev)
    T = wl.n_tris
    mics = torch.as_tensor(wl.mics, dtype=torch.float32, device=dev)
    band = np.ascontiguousarray(wl.band_hz, np.float32)
    kb = np.ascontiguousarray(wl.k_band, np.float32)
    beta = np.ascontiguousarray(wl.beta_band, np.float32)
    hp = lambda a: a.ctypes.data_as(C.c_void_p)
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def call(tm, los_t, out, n_bins=F):
        return L.st_accumulate_specular_noalloc(vp(tri), vp(pt), vp(dr), vp(r), vp(los_t), N, B, vp(tm), T,
                                                vp(mics), M, n_bins, wl.f_lo, wl.f_hi, kb.shape[0], kb.shape[1],
                                                hp(band), hp(kb), hp(beta), C.byref(p), vp(out), stream)

    outs = []
    for _ in range(2):
        out = torch.full((M, F), float("nan"), dtype=torch.complex64, device=dev)
        rc = call(tri_mat, los, out)
        torch.cuda.synchronize()
        assert rc == 0
        a = out.cpu().numpy()
        assert _rel(a, ref) <= TOL, _rel(a, ref)
        assert _rel(a, ora) <= TOL, _rel(a, ora)
        outs.append(a)
    assert np.array_equal(outs[0], outs[1])

    # a material id out of range drops the chains through that triangle, exactly as if their records
    # were not visible (nothing is read outside the tables)
    bad_tri = int(tri[0, 0].item()) if int(tri[0, 0].item()) >= 0 else 0
    tm_bad = tri_mat.clone()
    tm_bad[bad_tri] = kb.shape[0]
    through = (tri == bad_tri).to(torch.int32).cumsum(1) > 0
    los_cut = torch.where(through, torch.zeros_like(los), los)
    out_bad = torch.empty((M, F), dtype=torch.complex64, device=dev)
    out_cut = torch.empty((M, F), dtype=torch.complex64, device=dev)
    assert call(tm_bad, los, out_bad) == 0
    assert call(tri_mat, los_cut, out_cut) == 0
    torch.cuda.synchronize()
    assert np.array_equal(out_bad.cpu().numpy(), out_cut.cpu().numpy())
    assert not np.array_equal(out_bad.cpu().numpy(), outs[0])

    # sizes beyond the fixed scratch are rejected
    assert call(tri_mat, los, out, n_bins=1 << 16) == -1
