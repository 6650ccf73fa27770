"""Impulse responses and received signals on the GPU against the oracle's float64 restatement, on
spectra the GPU simulated (both sides take the same complex64 spectra as input)."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=20_000, bounces=4, n_mics=5, n_bins=96)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    S = ctx.simulate(sc, st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance))
    return dict(torch=torch, st=st, ctx=ctx, sc=sc, wl=wl, S=S)


def chirp(f0, f1, dur, fs):
    t = np.arange(int(dur * fs)) / fs
    k = (f1 - f0) / dur
    return (np.sin(2 * np.pi * (f0 * t + 0.5 * k * t * t)) * np.hanning(len(t))).astype(np.float32)


def test_impulse_response_sum_of_components(env):
    from oracle import signal
    wl, S = env["wl"], env["S"]
    fs, N = 200e3, 3001
    y = env["ctx"].impulse_response(S, wl.f_lo, wl.f_hi, fs, N).cpu().numpy()
    ref = signal.impulse_response(S.cpu().numpy().astype(np.complex128), wl.f_lo, wl.f_hi, fs, N)
    assert y.shape == ref.shape == (5, N)
    assert rel_l2(y, ref) <= TOL, rel_l2(y, ref)


def test_received_signal_per_component_with_window_and_call(env):
    from oracle import signal
    torch, wl, S = env["torch"], env["wl"], env["S"]
    fs, N = 250e3, 20000
    call = chirp(80e3, 20e3, 1e-3, fs)
    w = np.hanning(wl.n_bins).astype(np.float32)
    y = env["ctx"].impulse_response(S, wl.f_lo, wl.f_hi, fs, N, window=torch.from_numpy(w),
                                    call=torch.from_numpy(call), per_component=True).cpu().numpy()
    ref = signal.impulse_response(S.cpu().numpy().astype(np.complex128), wl.f_lo, wl.f_hi, fs, N, call=call,
                                  window=w, sum_components=False)
    assert y.shape == ref.shape == (3, 5, N)
    for c in range(3):
        assert rel_l2(y[c], ref[c]) <= TOL, (c, rel_l2(y[c], ref[c]))


def test_long_response_many_bins(env):
    """512 bins, 40,000 samples: phases of up to 10^4 cycles reduced in float64."""
    from oracle import signal
    torch = env["torch"]
    rng = np.random.default_rng(7)
    S = (rng.normal(size=(1, 2, 512)) + 1j * rng.normal(size=(1, 2, 512))).astype(np.complex64)
    y = env["ctx"].impulse_response(torch.from_numpy(S).cuda(), 20e3, 80e3, 200e3, 40000).cpu().numpy()
    ref = signal.impulse_response(S.astype(np.complex128), 20e3, 80e3, 200e3, 40000)
    assert rel_l2(y, ref) <= TOL, rel_l2(y, ref)


def test_single_bin_single_mic(env):
    from oracle import signal
    torch = env["torch"]
    S = np.array([[[0.3 - 0.4j]]], np.complex64)
    y = env["ctx"].impulse_response(torch.from_numpy(S).cuda(), 40e3, 40e3, 192e3, 77).cpu().numpy()
    ref = signal.impulse_response(S.astype(np.complex128), 40e3, 40e3, 192e3, 77)
    assert rel_l2(y, ref) <= TOL


def test_direct_path_echo_times():
    """Direct component of the shoebox: each microphone's response peaks at t = |s - m| / c, modulo the
    period 1 / df of a response computed from a spectrum sampled every df."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st
    wl = synth.shoebox(seed=101)
    wl.mics = np.array([[1.0, 1.0, 1.2], [3.1, 2.2, 0.7], [0.4, 2.5, 2.0]], np.float32)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    S = ctx.simulate(sc, st.sim_params(max_bounces=wl.bounces, components=st.ST_COMP_DIRECT))
    fs = 400e3
    y = ctx.impulse_response(S, wl.f_lo, wl.f_hi, fs, 8000).cpu().numpy()
    period = (wl.n_bins - 1) / (wl.f_hi - wl.f_lo)
    for m in range(3):
        tau = float(np.linalg.norm(wl.mics[m].astype(np.float64) - wl.emitter)) / 343.0
        expect = (tau % period) * fs
        one = np.abs(y[m][:int(period * fs)])  # one period: the copies beyond it are equal
        got = int(np.argmax(one))
        assert min(abs(got - expect), abs(got - expect + period * fs), abs(got - expect - period * fs)) <= 2.0, \
            (m, got, expect)
