"""Pins for the oracle's geometry: Philox known answers, normals, the watertight test,
brute force == BVH, and the shoebox unfolding closed form (Algorithm 1 on a box)."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(oracle_lib):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_normals_known():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 2]], dtype=np.float32)
    T = np.array([[0, 1, 2], [0, 2, 1], [0, 3, 1]], dtype=np.int32)
    n = oracle.tri_normals(V, T)
    assert np.array_equal(n[0], [0, 0, 1])
    assert np.array_equal(n[1], [0, 0, -1])
    assert np.array_equal(n[2], [0, 1, 0])
    # degenerate triangle -> zero normal
    n = oracle.tri_normals(V, np.array([[0, 1, 1]], dtype=np.int32))
    assert np.array_equal(n[0], [0, 0, 0])


def test_intersection_special_cases():
    # unit right triangle in z = 0; rays straight down
    V = np.array([[0, 0, 0], [2, 0, 0], [0, 2, 0]], dtype=np.float32)
    T = np.array([[0, 1, 2]], dtype=np.int32)
    sc = oracle.Scene(V, T, use_bvh=False)
    tri, t = sc.closest_hit([0.5, 0.5, 3.0], [0, 0, -1])
    assert tri == 0 and t == 3.0
    tri, t = sc.closest_hit([0.5, 0.5, -1.5], [0, 0, 1])          # two-sided
    assert tri == 0 and t == 1.5
    assert sc.closest_hit([1.5, 1.5, 3.0], [0, 0, -1])[0] == -1     # outside the hypotenuse
    assert sc.closest_hit([0.5, 0.5, 3.0], [0, 0, 1])[0] == -1      # behind the origin
    assert sc.closest_hit([0.5, 0.5, 3.0], [0, 0, -1], exclude=0)[0] == -1
    assert sc.closest_hit([0.5, 0.5, 1e-6], [0, 0, -1], t_min=1e-5)[0] == -1  # t <= t_min
    # parallel ray in the plane: no hit
    assert sc.closest_hit([-1, 0.5, 0], [1, 0, 0])[0] == -1


def test_watertight_shared_edge():
    """A square split along its diagonal: rays through the shared edge and the shared vertices
    must hit (never fall through the crack); ties in t resolve to the lower triangle index."""
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float32)
    T = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    sc = oracle.Scene(V, T, use_bvh=False)
    for s in np.linspace(0.0, 1.0, 33, dtype=np.float32):
        tri, t = sc.closest_hit([s, s, 1.0], [0, 0, -1])
        assert tri == 0 and t == 1.0, (s, tri, t)
    rng = np.random.default_rng(1)
    for _ in range(2000):  # oblique rays aimed at points on the diagonal
        s = np.float32(rng.uniform(0.01, 0.99))
        d = rng.normal(size=3)
        d[2] = -abs(d[2]) - 0.2
        d = (d / np.linalg.norm(d)).astype(np.float32)
        o = (np.array([s, s, 0.0]) - 2.0 * d.astype(np.float64)).astype(np.float32)
        tri, _ = sc.closest_hit(o, d)
        assert tri in (0, 1)


def test_bvh_equals_brute_force():
    wl = synth.clutter(seed=7, target_tris=6000, n_rays=1, diffraction=False)
    bf = oracle.Scene(wl.verts, wl.tris, use_bvh=False)
    bv = oracle.Scene(wl.verts, wl.tris, use_bvh=True)
    rng = np.random.default_rng(3)
    n_hit = 0
    for _ in range(600):
        o = np.array([rng.uniform(0, 20), rng.uniform(0, 20), rng.uniform(0.01, 5)], dtype=np.float32)
        d = rng.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        a = bf.closest_hit(o, d)
        b = bv.closest_hit(o, d)
        assert a == b
        n_hit += a[0] >= 0
        tgt = np.array([rng.uniform(0, 20), rng.uniform(0, 20), rng.uniform(0.01, 5)], dtype=np.float32)
        assert bf.visible(o, tgt) == bv.visible(o, tgt)
    assert n_hit > 150
    # whole-trace equality on the same scene
    dirs = synth.fibonacci_directions(2000)
    s = np.array([10.0, 10.0, 1.0], dtype=np.float32)
    q = np.array([1, 0, 0, 0], dtype=np.float32)
    R = np.array([10.0, 10.05, 1.0], dtype=np.float32)
    ra = oracle.trace(bf, s, q, dirs, 4, R=R)
    rb = oracle.trace(bv, s, q, dirs, 4, R=R)
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k


def _unfold(o, d, L, nb):
    """Crossings of the straight line o + t d with the lattice planes x_k = n L_k, in order:
    returns [(t, axis, wall_id)], wall parity mapped to the box's wall numbering."""
    ev = []
    wall_of = {0: (2, 3), 1: (4, 5), 2: (0, 1)}
    for k in range(3):
        if d[k] == 0:
            continue
        n = 1 if d[k] > 0 else 0
        for _ in range(nb + 1):
            t = (n * L[k] - o[k]) / d[k]
            ev.append((t, k, wall_of[k][n % 2]))
            n += 1 if d[k] > 0 else -1
    ev.sort()
    return ev[:nb + 1]


def _fold(x, L):
    u = np.mod(x, 2 * L)
    return np.where(u <= L, u, 2 * L - u)


def test_shoebox_unfolding_closed_form():
    """Specular paths in a box are straight lines in the mirrored lattice: hit j is the j-th plane
    crossing, its wall the plane family + parity, r_j the crossing time, P_j the folded point."""
    wl = synth.shoebox(seed=101, n_rays=3000, bounces=6)
    L = wl.extra["room"].astype(np.float64)
    wall = wl.extra["wall"]
    sc = oracle.Scene(wl.verts, wl.tris, use_bvh=False)
    rec = oracle.trace(sc, wl.emitter, wl.emitter_quat, wl.dirs, wl.bounces, R=wl.mics[0])
    checked = 0
    for i in range(len(wl.dirs)):
        o = wl.emitter.astype(np.float64)
        d = wl.dirs[i].astype(np.float64)
        d /= np.linalg.norm(d)
        ev = _unfold(o, d, L, wl.bounces)
        for j in range(wl.bounces):
            t, _, w = ev[j]
            if abs(ev[j + 1][0] - t) < 1e-4 * t or (j > 0 and abs(t - ev[j - 1][0]) < 1e-4 * t):
                break  # too close to an edge or corner of the room
            assert rec["tri"][i, j] >= 0
            assert wall[rec["tri"][i, j]] == w, (i, j)
            assert abs(rec["r"][i, j] - t) <= 1e-5 * t
            p = _fold(o + t * d, L)
            assert np.allclose(rec["p"][i, j], p, atol=2e-5 * L.max())
            checked += 1
    assert checked > 0.9 * len(wl.dirs) * wl.bounces
    # closed convex room: every ray makes every bounce and sees the receiver point
    assert (rec["tri"] >= 0).all() and (rec["los"] == 1).all()


def test_trace_terminates_at_max_distance():
    wl = synth.shoebox(seed=101, n_rays=500, bounces=8)
    sc = oracle.Scene(wl.verts, wl.tris, use_bvh=False)
    rec = oracle.trace(sc, wl.emitter, wl.emitter_quat, wl.dirs, wl.bounces, r_max=6.0, R=wl.mics[0])
    for i in range(len(wl.dirs)):
        n = int((rec["tri"][i] >= 0).sum())
        assert (rec["tri"][i, :n] >= 0).all() and (rec["tri"][i, n:] < 0).all()
        if n < wl.bounces:
            assert rec["r"][i, n - 1] >= 6.0 and (n == 1 or rec["r"][i, n - 2] < 6.0)
        assert np.all(np.diff(rec["r"][i, :n]) > 0)


def test_reflection_mirror():
    """One bounce off the floor: the reflected direction mirrors z and keeps x, y exactly."""
    V = np.array([[-10, -10, 0], [10, -10, 0], [10, 10, 0], [-10, 10, 0]], dtype=np.float32)
    T = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    sc = oracle.Scene(V, T, use_bvh=False)
    d = np.array([[0.6, 0.0, -0.8]], dtype=np.float32)
    rec = oracle.trace(sc, [0, 0, 4], [1, 0, 0, 0], d, 2, R=np.array([0, 0, 5], np.float32))
    assert rec["tri"][0, 0] >= 0 and rec["tri"][0, 1] == -1
    assert np.allclose(rec["d"][0, 0], [0.6, 0.0, 0.8], atol=1e-7)
    assert np.allclose(rec["p"][0, 0], [3.0, 0.0, 0.0], atol=1e-6)
    assert abs(rec["r"][0, 0] - 5.0) < 1e-6
