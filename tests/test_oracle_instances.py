"""Pins for the oracle's expansion of instanced scenes (shared meshes placed by affine maps x -> A x + b).

The expectations come from geometry, not from the expansion code: identity maps reproduce the prototypes,
translations on a coarse grid and quarter turns are exact in float32, a rotation with a uniform scale
keeps edge-length ratios and the facing of every triangle, and the world triangles of instance i index
its own vertices, which follow those of instance i-1."""
import math

import numpy as np

import oracle
import synth


def _grid_protos(rng):
    """Two small prototypes whose coordinates lie on a 2^-8 grid within (-4, 4) (exact under the maps below)."""
    out = []
    for nv, nt, mat in ((5, 4, 1), (7, 6, 2)):
        v = (rng.integers(-1000, 1000, (nv, 3)) / 256.0).astype(np.float32)
        t = rng.integers(0, nv, (nt, 3)).astype(np.int32)
        out.append((v, t, np.full(nt, mat, np.int32)))
    return out


def _xf(A, b):
    return np.concatenate([np.asarray(A, np.float64), np.asarray(b, np.float64)[:, None]], 1).astype(np.float32)


def test_identity_maps_reproduce_the_prototypes_in_instance_order():
    rng = np.random.default_rng(1)
    protos = _grid_protos(rng)
    inst = np.array([1, 0, 1, 1, 0], np.int32)
    V, T, M, O = oracle.expand_instances(protos, inst, [_xf(np.eye(3), np.zeros(3))] * len(inst))
    vb = 0
    tb = 0
    for i, q in enumerate(inst):
        pv, pt, pm = protos[q]
        assert np.array_equal(V[vb:vb + len(pv)], pv)
        assert np.array_equal(T[tb:tb + len(pt)], pt + vb)  # local indices offset by the instance's first vertex
        assert np.all(M[tb:tb + len(pt)] == pm) and np.all(O[tb:tb + len(pt)] == i)
        vb += len(pv)
        tb += len(pt)
    assert vb == len(V) and tb == len(T)


def test_translations_and_quarter_turns_are_exact():
    rng = np.random.default_rng(2)
    protos = _grid_protos(rng)
    pv = protos[0][0].astype(np.float64)
    b = np.array([7.0, -3.0, 12.0])
    Rz90 = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]  # (x, y, z) -> (-y, x, z); its transpose would give (y, -x, z)
    Rx90 = [[1, 0, 0], [0, 0, -1], [0, 1, 0]]  # (x, y, z) -> (x, -z, y)
    cases = [(np.eye(3), b, pv + b),
             (Rz90, np.zeros(3), np.stack([-pv[:, 1], pv[:, 0], pv[:, 2]], 1)),
             (Rx90, b, np.stack([pv[:, 0], -pv[:, 2], pv[:, 1]], 1) + b),
             (2.0 * np.eye(3), np.zeros(3), 2.0 * pv)]
    for A, bb, want in cases:
        V, _, _, _ = oracle.expand_instances(protos, [0], [_xf(A, bb)])
        assert np.array_equal(V.astype(np.float64), want)


def test_rotation_with_uniform_scale_keeps_shape_and_facing():
    rng = np.random.default_rng(3)
    v, f = synth.icosphere(2)
    protos = [(v.astype(np.float32), f.astype(np.int32), np.zeros(len(f), np.int32))]
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    s = 1.7
    V, T, _, _ = oracle.expand_instances(protos, [0], [_xf(s * R, [3.0, -2.0, 0.5])])
    P = protos[0][0].astype(np.float64)
    W = V.astype(np.float64)
    e0 = np.linalg.norm(P[f[:, 1]] - P[f[:, 0]], axis=1)
    e1 = np.linalg.norm(W[T[:, 1]] - W[T[:, 0]], axis=1)
    assert np.max(np.abs(e1 / e0 - s)) < 1e-5
    n0 = np.cross(P[f[:, 1]] - P[f[:, 0]], P[f[:, 2]] - P[f[:, 0]])
    n1 = np.cross(W[T[:, 1]] - W[T[:, 0]], W[T[:, 2]] - W[T[:, 0]])
    n0 = (R @ n0.T).T / np.linalg.norm(n0, axis=1, keepdims=True)
    n1 /= np.linalg.norm(n1, axis=1, keepdims=True)
    assert np.min(np.sum(n0 * n1, 1)) > 0.9999  # each triangle still faces the rotated way
    # the centre of the unit sphere lands on b
    assert np.allclose(W.mean(0), [3.0, -2.0, 0.5], atol=1e-5)


def test_forest_expands_and_runs_through_the_oracle():
    fo = synth.instanced_forest(n_inst=40, n_rays=2000, n_mics=4, n_bins=16)
    V, T, M, O = oracle.expand_instances(fo.protos, fo.inst_proto, fo.inst_xform)
    assert O.max() == 39 and len(T) == sum(len(fo.protos[q][1]) for q in fo.inst_proto)
    wl = type(fo.base)(**{**fo.base.__dict__, "verts": V, "tris": T, "tri_mat": M, "tri_obj": O})
    o = oracle.simulate(wl, curv=dict(budget=20_000))
    assert (o["rec"]["tri"] >= 0).sum() > 1000
    assert o["cand_keep"].sum() > 0
    assert np.abs(o["spectra"][0]).sum() > 0
    # the ground (instance 0) and the plants are hit
    hit_obj = O[o["rec"]["tri"][o["rec"]["tri"] >= 0]]
    assert np.any(hit_obj == 0) and np.any(hit_obj > 0)
    assert math.isfinite(float(np.abs(o["spectra"]).sum()))
