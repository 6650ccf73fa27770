"""Impulse responses and receiver signals on the CPU (float64) -- TEST INFRASTRUCTURE ONLY.

Only `tests/` and the CPU leg of `bench.py` may import this module.  It restates the signal stage of
the method (Sec. III-C to III-F): every path's transfer function is M(f) e^{+j 2 pi f r / c}; its
impulse response is the inverse Fourier transform, summed over paths (Eq. 5-6 specular, 9-10
diffraction, 13 direct); the components add into the scene's impulse response, and the received
signal is its convolution with the emitted call.  By linearity the sum over paths is the inverse
transform of the accumulated spectrum S[c][m][k] on the uniform grid f_k = f_lo + k df.

Reading (the paper names F^{-1} without its convention): the delay term e^{+j 2 pi f r / c} puts an
echo at t = r / c when the inverse transform takes the kernel e^{-j 2 pi f t} (time dependence
e^{-j omega t}), and the spectra hold the positive frequencies of a real signal, so

    h[m][n] = 2 df Re sum_k w_k S[m][k] E_k e^{-j 2 pi f_k n / fs},   t_n = n / fs,
    E_k     = (1 / fs) sum_i call[i] e^{+j 2 pi f_k i / fs}      (E = 1 without a call),

which is the band-limited impulse response (or received signal) sampled at fs; w is an optional
per-bin window.  Pinned by: the closed-form geometric sum of a single path, the special case that
equals numpy's FFT, a unit impulse call (E = 1) and a delayed impulse (a time shift).
"""
from __future__ import annotations

import numpy as np


def freq_grid(n_bins: int, f_lo: float, f_hi: float) -> np.ndarray:
    """f_k = f_lo + k (f_hi - f_lo) / (F - 1); a single bin sits at f_lo."""
    if n_bins == 1:
        return np.array([f_lo], np.float64)
    return f_lo + np.arange(n_bins, dtype=np.float64) * ((f_hi - f_lo) / (n_bins - 1))


def call_spectrum(call, f: np.ndarray, fs: float) -> np.ndarray:
    """E_k = (1/fs) sum_i call[i] e^{+j 2 pi f_k i / fs} (float64)."""
    call = np.asarray(call, np.float64)
    i = np.arange(len(call), dtype=np.float64)
    ph = np.outer(f, i) / fs
    return (np.exp(2j * np.pi * ph) @ call) / fs


def impulse_response(S, f_lo: float, f_hi: float, fs: float, n_samples: int, call=None, window=None,
                     sum_components: bool = True) -> np.ndarray:
    """S: complex [C][M][F] (or [M][F]).  Returns float64 [M][n] (components summed) or [C][M][n]."""
    S = np.asarray(S, np.complex128)
    if S.ndim == 2:
        S = S[None]
    Cn, M, F = S.shape
    f = freq_grid(F, f_lo, f_hi)
    df = (f_hi - f_lo) / (F - 1) if F > 1 else 1.0
    g = np.ones(F, np.complex128)
    if window is not None:
        g = g * np.asarray(window, np.float64)
    if call is not None:
        g = g * call_spectrum(call, f, fs)
    if sum_components:
        S = S.sum(axis=0, keepdims=True)
    n = np.arange(n_samples, dtype=np.float64)
    kern = np.exp(-2j * np.pi * np.outer(f, n) / fs)  # [F][N]
    out = 2.0 * df * np.real((S * g) @ kern)
    return out[0] if sum_components else out
