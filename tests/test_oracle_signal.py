"""Pins of the oracle's signal stage (impulse responses and received signals) against the mathematics:
a single path's closed-form geometric sum, numpy's FFT in the special case of a grid starting at 0
Hz with df = fs / N, a unit impulse call, a delayed impulse (time shift) and linearity."""
import numpy as np

from oracle import signal


def single_path(F, f_lo, f_hi, tau, amp=1.0):
    f = signal.freq_grid(F, f_lo, f_hi)
    return amp * np.exp(2j * np.pi * f * tau)


def test_single_path_closed_form():
    F, f_lo, f_hi, fs, N = 257, 20e3, 80e3, 400e3, 600
    tau = 0.6123e-3
    S = single_path(F, f_lo, f_hi, tau, 0.7)[None, None]
    h = signal.impulse_response(S, f_lo, f_hi, fs, N)[0]
    df = (f_hi - f_lo) / (F - 1)
    x = tau - np.arange(N) / fs
    # sum_k e^{j 2 pi (f_lo + k df) x} = e^{j 2 pi f_lo x} (1 - q^F) / (1 - q), q = e^{j 2 pi df x}
    q = np.exp(2j * np.pi * df * x)
    geo = np.where(np.abs(1 - q) < 1e-12, F, (1 - q ** F) / np.where(np.abs(1 - q) < 1e-12, 1, 1 - q))
    ref = 2 * df * 0.7 * np.real(np.exp(2j * np.pi * f_lo * x) * geo)
    assert np.max(np.abs(h - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert abs(np.argmax(np.abs(h)) - tau * fs) <= 1.0  # the echo sits at t = r / c


def test_matches_numpy_fft_special_case():
    rng = np.random.default_rng(1)
    Nfft, fs = 512, 1000.0
    F = 200
    df = fs / Nfft
    S = rng.normal(size=(3, 4, F)) + 1j * rng.normal(size=(3, 4, F))
    h = signal.impulse_response(S, 0.0, df * (F - 1), fs, Nfft, sum_components=False)
    pad = np.zeros((3, 4, Nfft), np.complex128)
    pad[..., :F] = S
    ref = 2 * df * np.real(np.fft.fft(pad, axis=-1))  # sum_k S_k e^{-j 2 pi k n / N}
    assert np.allclose(h, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_unit_and_delayed_impulse_call():
    rng = np.random.default_rng(2)
    F, f_lo, f_hi, fs, N = 64, 20e3, 60e3, 200e3, 300
    S = rng.normal(size=(2, F)) + 1j * rng.normal(size=(2, F))
    h = signal.impulse_response(S, f_lo, f_hi, fs, N)
    unit = np.zeros(5)
    unit[0] = fs  # (1/fs) * fs * e^0 = 1 at every bin
    assert np.allclose(signal.impulse_response(S, f_lo, f_hi, fs, N, call=unit), h, atol=1e-12 * np.abs(h).max())
    d = 17
    delayed = np.zeros(d + 1)
    delayed[d] = fs
    y = signal.impulse_response(S, f_lo, f_hi, fs, N, call=delayed)
    assert np.allclose(y[:, d:], h[:, :N - d], atol=1e-9 * np.abs(h).max())


def test_linearity_over_components():
    rng = np.random.default_rng(3)
    S = rng.normal(size=(3, 2, 40)) + 1j * rng.normal(size=(3, 2, 40))
    per = signal.impulse_response(S, 1e3, 5e3, 20e3, 100, sum_components=False)
    tot = signal.impulse_response(S, 1e3, 5e3, 20e3, 100)
    assert np.allclose(per.sum(0), tot, atol=1e-12 * np.abs(tot).max())
