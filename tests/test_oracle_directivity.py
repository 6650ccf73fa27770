"""Pins for the oracle's directivity (Sec. III-F: emission pattern and receiver transfer, applied per
path in the spectra).  The emitter table is sampled over the angle theta between the emitter's forward
axis (its quaternion applied to +x) and a path's departure direction, on theta_i = i pi / (n_theta - 1),
linear in theta.  A receiver table is sampled over azimuth and elevation of the arrival direction (from
the microphone towards the path's last point) in the microphone's frame (the world direction turned by
the conjugate of the microphone's quaternion): az_i = -pi + 2 pi i / n_az (periodic), el_j = -pi / 2 +
j pi / (n_el - 1), bilinear in (az, el) and linear between band centres.

Every expected value here comes from the geometry and from the fact that linear interpolation
reproduces a linear function: constant tables scale the spectra exactly; a table linear in theta,
elevation or azimuth returns that line at off-grid angles that the test places by hand; a single-cell
peak follows a quarter turn of the microphone by a quarter of the azimuth grid.  The spectra are
divided by those of the same paths with omni tables, which removes every other factor."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth

F = 8
N_BANDS = 4


def _rot(axis, ang):
    """Rotation matrix about `axis` by `ang` (Rodrigues)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _quat(axis, ang):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    return np.array([math.cos(ang / 2), *(math.sin(ang / 2) * a)], np.float32)


def _workload(emitter, mics, emitter_quat=None, emitter_table=None, mic_tables=None, mic_quats=None):
    v = np.array([[50, 50, 50], [51, 50, 50], [50, 51, 50]], np.float32)  # one triangle, out of the way
    M = len(mics)
    return synth.Workload(
        name="directivity", verts=v, tris=np.array([[0, 1, 2]], np.int32), tri_mat=np.zeros(1, np.int32),
        tri_obj=np.zeros(1, np.int32), band_hz=np.linspace(25e3, 75e3, N_BANDS).astype(np.float32),
        k_band=np.full((1, N_BANDS), 0.8, np.float32), beta_band=np.full((1, N_BANDS), 0.3, np.float32),
        diff_band=np.full((1, N_BANDS), 0.05, np.float32), emitter=np.asarray(emitter, np.float32),
        emitter_quat=np.array([1, 0, 0, 0], np.float32) if emitter_quat is None else emitter_quat,
        dirs=np.zeros((0, 3), np.float32), mics=np.asarray(mics, np.float32).reshape(M, 3), n_bins=F,
        f_lo=20e3, f_hi=80e3, bounces=1, emitter_table=emitter_table, mic_tables=mic_tables, mic_quats=mic_quats)


def _direct(wl):
    """Direct-path spectra [M][F] of a workload whose every microphone is visible."""
    P = oracle.spec_params(wl)
    rec = dict(tri=np.zeros((0, 1), np.int32), p=np.zeros((0, 1, 3), np.float32),
               d=np.zeros((0, 1, 3), np.float32), r=np.zeros((0, 1)), los=np.zeros((0, 1), np.uint8))
    return oracle.spectra(P, rec, wl.dirs, wl.tri_mat, direct_vis=np.ones(len(wl.mics), np.uint8))[2]


def _omni(wl):
    return dataclasses.replace(wl, emitter_table=None, mic_tables=None, mic_quats=None)


def _ratio(wl):
    return _direct(wl) / _direct(_omni(wl))


def _angle(u, v):
    u, v = np.asarray(u, np.float64), np.asarray(v, np.float64)
    return math.atan2(np.linalg.norm(np.cross(u, v)), float(np.dot(u, v)))


def test_constant_tables_scale_every_component():
    """Constant emitter (0.7) and receiver (1.3) tables scale the specular, diffraction and direct
    spectra by exactly 0.91 (their float32 values' product), for paths leaving and arriving in all directions."""
    rng = np.random.default_rng(1)
    M, N, B, K = 5, 40, 2, 30
    mics = rng.uniform(-2, 2, (M, 3)).astype(np.float32)
    q = _quat([1, 2, 3], 0.8)
    mq = np.stack([_quat(rng.normal(size=3), rng.uniform(0, 6)) for _ in range(M)])
    wl = _workload([0.1, 0.2, 0.3], mics, emitter_quat=q, emitter_table=np.full((19, F), 0.7, np.float32),
                   mic_tables=np.full((M, 13, 24, N_BANDS), 1.3, np.float32), mic_quats=mq)
    wl = dataclasses.replace(wl, dirs=synth.fibonacci_directions(N))
    rec = dict(tri=np.zeros((N, B), np.int32), p=rng.uniform(-3, 3, (N, B, 3)).astype(np.float32),
               d=synth.fibonacci_directions(N * B)[rng.permutation(N * B)].reshape(N, B, 3),
               r=rng.uniform(1, 5, (N, B)), los=(rng.uniform(size=(N, B)) < 0.8).astype(np.uint8))
    ct, cp = np.zeros(K, np.int32), rng.uniform(-3, 3, (K, 3)).astype(np.float32)
    keep = np.ones(K, np.uint8)
    dv = np.ones(M, np.uint8)
    S = oracle.spectra(oracle.spec_params(wl), rec, wl.dirs, wl.tri_mat, ct, cp, keep, dv)
    S0 = oracle.spectra(oracle.spec_params(_omni(wl)), rec, wl.dirs, wl.tri_mat, ct, cp, keep, dv)
    for c in range(3):
        assert np.abs(S0[c]).min() > 0
        want = float(np.float32(0.7)) * float(np.float32(1.3))   # the tables hold float32 values
        assert np.allclose(S[c], want * S0[c], rtol=1e-12, atol=0), c


def test_emitter_table_linear_in_theta_at_off_grid_angles():
    """An emitter table a_k + b_k theta_i returns a_k + b_k theta at any theta, where theta is the angle
    between the emitter's forward axis and the departure direction.  The emitter is turned a quarter
    turn about z (forward = +y), so a table read about +x, or on a grid of pi / n_theta, fails."""
    n_theta = 19
    th_grid = np.arange(n_theta) * math.pi / (n_theta - 1)
    a = np.linspace(0.5, 1.5, F)
    b = np.linspace(-0.3, 0.2, F)
    table = (a[None, :] + b[None, :] * th_grid[:, None]).astype(np.float32)
    s = np.array([0.5, -0.25, 0.125], np.float32)
    fwd = np.array([0.0, 1.0, 0.0])
    want_th = [0.1, 0.65, 1.234, 2.0, 2.9]
    mics = []
    for i, th in enumerate(want_th):
        side = _rot(fwd, 0.7 * i) @ np.array([0.0, 0.0, 1.0])       # any direction normal to forward
        mics.append(s + 2.0 * (math.cos(th) * fwd + math.sin(th) * side))
    mics = np.array(mics, np.float32)
    wl = _workload(s, mics, emitter_quat=_quat([0, 0, 1], math.pi / 2), emitter_table=table)
    R = _ratio(wl)
    for m in range(len(mics)):
        th = _angle(fwd, mics[m].astype(np.float64) - s)           # the float32 positions' angle
        assert abs(th - want_th[m]) < 1e-6
        assert np.allclose(R[m].real, a + b * th, rtol=1e-6, atol=1e-6), (m, R[m].real, a + b * th)  # float32 table
        assert np.allclose(R[m].imag, 0, atol=1e-12)


def test_emitter_table_on_specular_paths_uses_the_ray_direction():
    """A specular path leaves along its ray's direction (in the emitter frame): with forward = +x in that
    frame, theta is the angle of the ray direction from +x, whatever the emitter's quaternion."""
    n_theta = 37
    th_grid = np.arange(n_theta) * math.pi / (n_theta - 1)
    table = np.repeat((0.25 + 0.5 * th_grid)[:, None], F, 1).astype(np.float32)
    want_th = np.array([0.05, 0.8, 1.7, 2.6, 3.1])
    dirs = np.stack([np.cos(want_th), np.sin(want_th) * 0.6, np.sin(want_th) * 0.8], 1).astype(np.float32)
    N = len(dirs)
    wl = _workload([0, 0, 0], [[1.0, 0.5, 0.2]], emitter_quat=_quat([1, -2, 0.5], 1.1), emitter_table=table)
    wl = dataclasses.replace(wl, dirs=dirs)
    rec = dict(tri=np.zeros((N, 1), np.int32), p=np.tile(np.array([3.0, -1.0, 2.0], np.float32), (N, 1, 1)),
               d=np.tile(np.array([0.0, 0.0, 1.0], np.float32), (N, 1, 1)), r=np.full((N, 1), 2.0),
               los=np.ones((N, 1), np.uint8))
    for i in range(N):
        one = {k: v[i:i + 1] for k, v in rec.items()}
        S = oracle.spectra(oracle.spec_params(wl), one, dirs[i:i + 1], wl.tri_mat)[0]
        S0 = oracle.spectra(oracle.spec_params(_omni(wl)), one, dirs[i:i + 1], wl.tri_mat)[0]
        th = _angle([1.0, 0.0, 0.0], dirs[i])
        assert np.allclose(S / S0, 0.25 + 0.5 * th, rtol=1e-6), (i, (S / S0)[0, 0], 0.25 + 0.5 * th)


def _mic_table(fun, n_el=91, n_az=180):
    el = -math.pi / 2 + np.arange(n_el) * math.pi / (n_el - 1)
    az = -math.pi + np.arange(n_az) * 2 * math.pi / n_az
    E, A = np.meshgrid(el, az, indexing="ij")
    return np.repeat(fun(A, E)[:, :, None], N_BANDS, 2).astype(np.float32)


def _source_at(mic, R, az, el, dist=1.5):
    """Emitter position whose arrival direction at `mic` has azimuth az and elevation el in the frame R
    (columns = the microphone's axes in the world)."""
    local = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return (np.asarray(mic, np.float64) + dist * (R @ local)).astype(np.float32)


@pytest.mark.parametrize("which", ["elevation", "azimuth"])
def test_receiver_table_linear_in_one_angle(which):
    """A receiver table linear in elevation (or in azimuth, away from the cell that wraps around)
    returns that line at hand-placed off-grid arrival directions, for a microphone turned by a general
    rotation: an azimuth/elevation swap, a missing conjugate or a grid off by one cell fails."""
    fun = (lambda A, E: 1.0 + 0.4 * E) if which == "elevation" else (lambda A, E: 1.0 + 0.2 * A)
    table = _mic_table(fun)[None]
    mic = np.array([0.3, -0.2, 0.1], np.float32)
    Rm = _rot([0.3, -1.0, 0.6], 2.1)
    mq = _quat([0.3, -1.0, 0.6], 2.1)[None]
    for az, el in [(-2.5, 0.3), (-0.77, -1.1), (0.41, 0.93), (1.9, -0.2), (3.0, 0.05)]:
        s = _source_at(mic, Rm, az, el)
        wl = _workload(s, mic[None], mic_tables=table, mic_quats=mq)
        loc = Rm.T @ (s.astype(np.float64) - mic)                   # the float32 positions' angles
        az_t = math.atan2(loc[1], loc[0])
        el_t = math.asin(loc[2] / np.linalg.norm(loc))
        assert abs(az_t - az) < 1e-5 and abs(el_t - el) < 1e-5
        want = fun(az_t, el_t)
        assert np.allclose(_ratio(wl)[0].real, want, rtol=1e-5), (az, el, _ratio(wl)[0].real, want)


def test_receiver_table_linear_between_bands():
    """Band values u + v f_b (f_b the band centres) give u + v f at every bin inside the band range and
    the end values outside it."""
    table = np.zeros((1, 7, 12, N_BANDS), np.float32)
    band = np.linspace(25e3, 75e3, N_BANDS)
    table[:] = (0.6 + 0.8 * band / 1e5).astype(np.float32)
    mic = np.zeros(3, np.float32)
    wl = _workload([1.0, 0.7, -0.4], mic[None], mic_tables=table)
    f = np.linspace(20e3, 80e3, F)
    want = 0.6 + 0.8 * np.clip(f, band[0], band[-1]) / 1e5
    assert np.allclose(_ratio(wl)[0].real, want, rtol=1e-6)


def test_quarter_turn_moves_a_single_cell_peak_by_a_quarter_of_the_azimuth_grid():
    """A table that is 1 at one cell (az_30 = -120 deg, el_55 = 20 deg) and 0 elsewhere: with the
    identity quaternion an arrival from that cell's direction reads 1; after a quarter turn of the
    microphone about z the peak is met a quarter of the grid (45 cells) further in world azimuth, and
    the original direction reads 0 (a missing conjugate would move it the other way)."""
    n_el, n_az = 91, 180
    table = np.zeros((1, n_el, n_az, N_BANDS), np.float32)
    i0, j0 = 30, 55
    table[0, j0, i0, :] = 1.0
    az0 = -math.pi + i0 * 2 * math.pi / n_az
    el0 = -math.pi / 2 + j0 * math.pi / (n_el - 1)
    mic = np.array([0.25, 0.5, -0.125], np.float32)
    quarter = _quat([0, 0, 1], math.pi / 2)[None]
    I = np.eye(3)
    step = 2 * math.pi / n_az

    def read(az, q):
        s = _source_at(mic, I, az, el0, dist=2.0)
        return _ratio(_workload(s, mic[None], mic_tables=table, mic_quats=q))[0].real

    ident = np.array([[1, 0, 0, 0]], np.float32)
    assert np.allclose(read(az0, ident), 1.0, atol=1e-5)
    assert np.allclose(read(az0 + step, ident), 0.0, atol=1e-5)
    assert np.allclose(read(az0 + 45 * step, quarter), 1.0, atol=1e-5)
    assert np.allclose(read(az0, quarter), 0.0, atol=1e-5)
    assert np.allclose(read(az0 - 45 * step, quarter), 0.0, atol=1e-5)
    # halfway between two cells in azimuth and in elevation: a quarter of the peak (bilinear)
    s = _source_at(mic, I, az0 + 45 * step + step / 2, el0 + math.pi / (n_el - 1) / 2, dist=2.0)
    assert np.allclose(_ratio(_workload(s, mic[None], mic_tables=table, mic_quats=quarter))[0].real, 0.25,
                       atol=1e-4)
