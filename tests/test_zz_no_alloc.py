"""The allocation-free accumulation entry point, for callers that cannot allocate device memory
(fixed arenas owned by another allocator, real-time loops, callbacks where allocation is not
allowed).  It must give the specular spectrum of st_simulate, from the same path records, within
the parity tolerance, on consecutive calls that share its fixed scratch.  Kept in its own file,
collected last."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def test_noalloc_matches_simulate_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st
    L = st.load()
    wl = synth.gradient_problem(n_rays=4000)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, components=st.ST_COMP_SPECULAR)
    ref = ctx.simulate(sc, p)[0].clone()
    torch.cuda.synchronize()
    N, B, M, F = len(wl.dirs), wl.bounces, len(wl.mics), wl.n_bins
    dev = torch.device("cuda", 0)
    tri = torch.empty((N, B), dtype=torch.int32, device=dev)
    pt = torch.empty((N, B, 3), dtype=torch.float32, device=dev)
    dr = torch.empty((N, B, 3), dtype=torch.float32, device=dev)
    r = torch.empty((N, B), dtype=torch.float64, device=dev)
    los = torch.empty((N, B), dtype=torch.uint8, device=dev)
    vp = lambda t: C.c_void_p(t.data_ptr())
    st.check(L.st_get_paths(ctx.h, vp(tri), vp(pt), vp(dr), vp(r), vp(los), st.ST_MEM_DEVICE), ctx.h)
    tri_mat = torch.as_tensor(wl.tri_mat, dtype=torch.int32, device=dev)
    mics = torch.as_tensor(wl.mics, dtype=torch.float32, device=dev)
    band = np.ascontiguousarray(wl.band_hz, np.float32)
    kb = np.ascontiguousarray(wl.k_band, np.float32)
    beta = np.ascontiguousarray(wl.beta_band, np.float32)
    hp = lambda a: a.ctypes.data_as(C.c_void_p)
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    outs = []
    for _ in range(2):
        out = torch.full((M, F), float("nan"), dtype=torch.complex64, device=dev)
        rc = L.st_accumulate_specular_noalloc(vp(tri), vp(pt), vp(dr), vp(r), vp(los), N, B, vp(tri_mat), vp(mics),
                                              M, F, wl.f_lo, wl.f_hi, kb.shape[0], kb.shape[1], hp(band), hp(kb),
                                              hp(beta), C.byref(p), vp(out), stream)
        torch.cuda.synchronize()
        assert rc == 0
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= TOL, err
        outs.append(a)
    assert np.array_equal(outs[0], outs[1])
    # sizes beyond the fixed scratch are rejected
    rc = L.st_accumulate_specular_noalloc(vp(tri), vp(pt), vp(dr), vp(r), vp(los), N, B, vp(tri_mat), vp(mics),
                                          M, 1 << 16, wl.f_lo, wl.f_hi, kb.shape[0], kb.shape[1], hp(band), hp(kb),
                                          hp(beta), C.byref(p), vp(out), stream)
    assert rc == -1
