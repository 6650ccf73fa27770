"""Pins for the oracle's per-microphone receiver test (the variant of the receiver connection with one
visibility ray per microphone instead of one towards the array's reference point).

The expectations come from the geometry, not from the oracle's visibility code: in an empty convex room
every hit point on a wall sees every interior point, and a plane wall separates the half-spaces on its two
sides."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth


def test_convex_room_every_microphone_visible_and_spectra_unchanged():
    wl = synth.shoebox(seed=7, n_rays=600, bounces=3, n_mics=6, n_bins=24)
    o0 = oracle.simulate(wl, components=1)
    o1 = oracle.simulate(wl, components=1, los_mode=1)
    rec = o1["rec"]
    hit = rec["tri"] >= 0
    full = np.uint64((1 << len(wl.mics)) - 1)
    assert hit.sum() > 1000
    assert np.all(rec["mask"][hit] == full)
    assert np.all(rec["mask"][~hit] == 0)
    assert np.array_equal(rec["los"], hit.astype(np.uint8))
    assert np.array_equal(o0["rec"]["los"], rec["los"])
    # the same (record, microphone) terms: identical sums
    assert np.array_equal(o1["spectra"], o0["spectra"])


def test_single_microphone_equals_reference_point_test():
    """With one microphone the reference point is the microphone itself: both tests cast the same rays.
    One microphone behind the wall: the wall's own hit points see it, the floor's in front of it do not."""
    wl = dataclasses.replace(_wall_workload(2000), mics=np.array([[-1.0, 0.0, 1.0]], np.float32))
    o0 = oracle.simulate(wl, components=1)
    o1 = oracle.simulate(wl, components=1, los_mode=1)
    assert np.array_equal(o1["rec"]["los"], o0["rec"]["los"])
    assert np.array_equal(o1["rec"]["mask"], o0["rec"]["los"].astype(np.uint64))
    assert 0 < o0["rec"]["los"].sum() < (o0["rec"]["tri"] >= 0).sum()
    assert np.array_equal(o1["spectra"], o0["spectra"])


def _wall_workload(n_rays=4000):
    """Floor z = 0 over x in [-10, 10] (material 0) and a wall x = 0 over |y|, z <= 10 (material 1); the
    emitter and microphones 0-2 in front of the wall (x > 0), microphones 3-4 behind it (x < 0)."""
    V = np.array([[-10, -10, 0], [10, -10, 0], [10, 10, 0], [-10, 10, 0],
                  [0, -10, 0], [0, 10, 0], [0, 10, 10], [0, -10, 10]], np.float32)
    T = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    nb = 4
    mics = np.array([[1.0, -0.3, 1.0], [1.2, 0.2, 0.8], [0.9, 0.1, 1.3], [-1.0, 0.0, 1.0], [-1.5, 0.4, 0.7]],
                    np.float32)
    return synth.Workload(
        name="wall", verts=V, tris=T, tri_mat=np.array([0, 0, 1, 1], np.int32), tri_obj=np.zeros(4, np.int32),
        band_hz=np.linspace(20e3, 80e3, nb).astype(np.float32), k_band=np.full((2, nb), 0.8, np.float32),
        beta_band=np.full((2, nb), math.radians(20.0), np.float32), diff_band=np.full((2, nb), 0.05, np.float32),
        emitter=np.array([2.0, 0.0, 1.0], np.float32), emitter_quat=np.array([1, 0, 0, 0], np.float32),
        dirs=synth.fibonacci_directions(n_rays), mics=mics, n_bins=16, f_lo=20e3, f_hi=80e3, bounces=3,
        max_distance=100.0)


def test_wall_separates_microphone_groups():
    wl = _wall_workload()
    o = oracle.simulate(wl, components=1, los_mode=1)
    rec = o["rec"]
    hit = rec["tri"] >= 0
    P = rec["p"]
    front, back = np.uint64(0b00111), np.uint64(0b11000)
    # hit points on the floor clearly in front of the wall: every front microphone visible, none behind
    floor_front = hit & (np.abs(P[..., 2]) < 1e-4) & (P[..., 0] > 0.05)
    assert floor_front.sum() > 300
    assert np.all((rec["mask"][floor_front] & front) == front)
    assert np.all((rec["mask"][floor_front] & back) == 0)
    # no ray reaches the far side of the wall (the emitter is in front, both surfaces reflect back)
    assert not np.any(hit & (P[..., 0] < -1e-4))
    # the microphones behind the wall receive specular paths only from hit points on the wall itself
    # (the hit triangle is excluded from its own visibility ray)
    any_back = hit & ((rec["mask"] & back) != 0)
    assert np.all(np.abs(P[..., 0][any_back]) < 1e-4)
    S = o["spectra"][0]
    assert np.abs(S[:3]).sum() > 0
    o_floor = oracle.simulate(dict_free_wall(wl), components=1, los_mode=1)
    # without the wall's records (wall made non-reflecting by moving it away) the back microphones see
    # floor points and so receive specular energy: the mask is what removes it above
    assert np.all((o_floor["rec"]["mask"][(o_floor["rec"]["tri"] >= 0)] & back) == back)


def dict_free_wall(wl):
    """The same scene with the wall moved far behind the back microphones (x = -50)."""
    import dataclasses
    V = wl.verts.copy()
    V[4:, 0] = -50.0
    return dataclasses.replace(wl, verts=V)


def test_per_microphone_test_needs_at_most_64_microphones():
    wl = synth.shoebox(seed=7, n_rays=10, bounces=1, n_mics=65, n_bins=4)
    with pytest.raises(ValueError):
        oracle.simulate(wl, components=1, los_mode=1)
