"""CPU oracle for the acoustic path-tracing hot path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import this
package.  It is a plain restatement of the method (float32 geometry in the GPU's precision and
operation order, float64 for everything after geometry) in `sonotrace_oracle.c`, wrapped with
ctypes and numpy.  It shares no code with the CUDA library.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  philox4x32_10      published known-answer vectors of Random123
  tri_normals        axis-aligned and rotated triangles with known normals
  curvature, metric  sphere (G ~ 1/R), cylinder side (G ~ 1/(2R)), plane (G = 0)
  diffraction_cdf    exact integer prefix sums; sample histogram chi-square vs weights
  trace              brute force == BVH bit for bit; shoebox unfolding closed form
  diffraction_filter hand-placed candidates: field of view, incidence limit, line of sight, orientation
  los_per_mic        empty convex room: every microphone visible and spectra equal to the reference-point
                     test; a plane wall between two microphone groups: the half-space each group is in;
                     one microphone: identical to the reference-point test
  spectra            single-path closed forms; direct path closed form; reciprocity
  spectra_grad       float64 central finite differences (also over records with microphone masks)
  expand_instances   identity maps, exact translations and quarter turns, rotations that keep edge-length
                     ratios and every triangle's facing
  (absolute scale of spectra against measurements: parity unpinned -- the paper has no data)
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


P = C.c_void_p
I32, I64, U32, U64, F32, F64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_float, C.c_double


class SpecParams(C.Structure):
    _fields_ = [
        ("F", I32), ("f_lo", F64), ("f_hi", F64), ("c", F64), ("a0", F64), ("a1_per_khz", F64),
        ("n_mat", I32), ("n_bands", I32), ("band_hz", P), ("k_band", P), ("beta_band", P), ("diff_band", P),
        ("M", I32), ("mics", P), ("mic_quats", P), ("mic_tables", P), ("n_az", I32), ("n_el", I32),
        ("s", P), ("q", P), ("emit_table", P), ("n_theta", I32), ("reflection_mode", I32),
        ("direct_gain", F64),
    ]


def _declare(L):
    L.ora_philox4x32_10.argtypes = [P, P, P]
    L.ora_tri_normals.argtypes = [I64, P, P, P]
    L.ora_weld.argtypes = [I64, P, P]
    L.ora_weld.restype = C.c_int
    L.ora_curvature.argtypes = [I64, P, I64, P, P]
    L.ora_curvature.restype = C.c_int
    L.ora_curvature_mixed.argtypes = [I64, P, I64, P, P, P]
    L.ora_curvature_mixed.restype = C.c_int
    L.ora_tri_metric.argtypes = [I64, P, I64, P, P, F32, F32, P]
    L.ora_diffraction_cdf.argtypes = [I64, P, I64, P, P, P, I32, F64, U64, F32, I32, I64, P, P, P, P]
    L.ora_diffraction_cdf.restype = C.c_int
    L.ora_diffraction_samples.argtypes = [P, P, I32, P, P, P, P, U64, U32, P, P]
    L.ora_diffraction_samples.restype = I64
    L.ora_scene_new.argtypes = [I64, P, I64, P, C.c_int]
    L.ora_scene_new.restype = P
    L.ora_scene_free.argtypes = [P]
    L.ora_closest_hit.argtypes = [P, P, P, I32, F32, P]
    L.ora_closest_hit.restype = I32
    L.ora_visible.argtypes = [P, P, P, I32, F32, F32]
    L.ora_visible.restype = C.c_int
    L.ora_mic_centroid.argtypes = [I32, P, P]
    L.ora_trace.argtypes = [P, P, P, P, I64, P, I32, F64, F32, F32, P, P, P, P, P, P, I32]
    L.ora_trace.restype = C.c_int
    L.ora_diffraction_filter.argtypes = [P, P, P, P, I64, P, P, F32, F32, F32, F32, P, I32]
    L.ora_direct_visibility.argtypes = [P, P, I32, P, F32, F32, P]
    L.ora_spectra.argtypes = [C.POINTER(SpecParams), I64, I32, P, P, P, P, P, P, P, I64, P, P, P, P,
                              I32, P, I32, P, I32, P, P]
    L.ora_los_per_mic.argtypes = [P, I64, P, P, I32, P, F32, F32, P, P, I32]
    L.ora_los_per_mic.restype = C.c_int
    L.ora_spectra.restype = C.c_int
    L.ora_spectra_grad.argtypes = [C.POINTER(SpecParams), I64, I32, P, P, P, P, P, P, P, I64, P, P, P, P,
                                   P, P, P, P, P, P, P, P]
    L.ora_spectra_grad.restype = C.c_int


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------------------------ RNG
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(_p(c), _p(k), _p(out))
    return out


# ------------------------------------------------------------------------------------ geometry
def tri_normals(verts, tris):
    v, t = _c(verts, np.float32), _c(tris, np.int32)
    n = np.zeros((len(t), 3), dtype=np.float32)
    lib().ora_tri_normals(len(t), _p(v), _p(t), _p(n))
    return n


def weld(verts):
    v = _c(verts, np.float32)
    out = np.zeros(len(v), dtype=np.int32)
    lib().ora_weld(len(v), _p(v), _p(out))
    return out


def curvature(verts, tris, mixed_area=False):
    """G_v per input vertex; with mixed_area, also each vertex's mixed area A_mixed (Meyer et al.)."""
    v, t = _c(verts, np.float32), _c(tris, np.int32)
    G = np.zeros(len(v), dtype=np.float32)
    A = np.zeros(len(v), dtype=np.float32) if mixed_area else None
    if lib().ora_curvature_mixed(len(v), _p(v), len(t), _p(t), _p(G), _p(A)) != 0:
        raise MemoryError("oracle curvature")
    return (G, A) if mixed_area else G


def tri_metric(verts, tris, G, eta=1.0, area_ref=1e-4):
    v, t, g = _c(verts, np.float32), _c(tris, np.int32), _c(G, np.float32)
    Cc = np.zeros(len(t), dtype=np.float32)
    lib().ora_tri_metric(len(v), _p(v), len(t), _p(t), _p(g), eta, area_ref, _p(Cc))
    return Cc


def diffraction_cdf(verts, tris, Cm, tri_obj, dither=1e-3, seed=0, hc_frac=0.25, samples_per_vertex=64,
                    budget=4_000_000):
    v, t, cm, ob = _c(verts, np.float32), _c(tris, np.int32), _c(Cm, np.float32), _c(tri_obj, np.int32)
    n_obj = int(ob.max()) + 1 if len(ob) else 0
    mesh_tris = np.zeros(len(t), dtype=np.int32)
    mesh_off = np.zeros(n_obj + 1, dtype=np.int64)
    cdf = np.zeros(len(t), dtype=np.uint64)
    ns = np.zeros(max(n_obj, 1), dtype=np.int64)
    lib().ora_diffraction_cdf(len(v), _p(v), len(t), _p(t), _p(cm), _p(ob), n_obj, dither, seed, hc_frac,
                              samples_per_vertex, budget, _p(mesh_tris), _p(mesh_off), _p(cdf), _p(ns))
    return dict(mesh_tris=mesh_tris, mesh_off=mesh_off, cdf=cdf, n_samples=ns[:n_obj], n_obj=n_obj)


def diffraction_samples(verts, tris, cdfd, seed=0, pose=0):
    v, t = _c(verts, np.float32), _c(tris, np.int32)
    K = int(cdfd["n_samples"].sum())
    ct = np.zeros(max(K, 1), dtype=np.int32)
    cp = np.zeros((max(K, 1), 3), dtype=np.float32)
    k = lib().ora_diffraction_samples(_p(v), _p(t), cdfd["n_obj"], _p(cdfd["mesh_tris"]), _p(cdfd["mesh_off"]),
                                      _p(cdfd["cdf"]), _p(cdfd["n_samples"]), seed, pose, _p(ct), _p(cp))
    assert k == K
    return ct[:K], cp[:K]


class Scene:
    """Triangle scene for the oracle's intersection queries (brute force or median-split BVH)."""

    def __init__(self, verts, tris, use_bvh=None):
        self.verts = _c(verts, np.float32)
        self.tris = _c(tris, np.int32)
        if use_bvh is None:
            use_bvh = len(self.tris) > 64
        self.h = lib().ora_scene_new(len(self.tris), _p(self.verts), len(self.verts), _p(self.tris), int(use_bvh))
        self.nrm = tri_normals(self.verts, self.tris)

    def __del__(self):
        try:
            if self.h:
                lib().ora_scene_free(self.h)
        except Exception:
            pass

    def closest_hit(self, o, d, exclude=-1, t_min=1e-5):
        o, d = _c(o, np.float32), _c(d, np.float32)
        t = np.zeros(1, dtype=np.float32)
        tri = lib().ora_closest_hit(self.h, _p(o), _p(d), exclude, t_min, _p(t))
        return int(tri), float(t[0])

    def visible(self, o, target, exclude=-1, t_min=1e-5, eps=1e-4):
        o, g = _c(o, np.float32), _c(target, np.float32)
        return bool(lib().ora_visible(self.h, _p(o), _p(g), exclude, t_min, eps))


def expand_instances(protos, inst_proto, inst_xform):
    """World triangles of a scene given as instances of shared meshes (Sec. III-B registers objects; a
    forest repeats plant meshes): instance i, in order, is prototype inst_proto[i] = (verts, tris with
    local indices, tri_mat) under x -> A x + b, inst_xform[i] = [A | b] (3 x 4).  Each world coordinate
    is ((A_r0 x + A_r1 y) + A_r2 z) + b_r with every product and sum rounded to float32 (numpy float32
    arithmetic), instance i's vertices and triangles follow instance i-1's, and instance i is object i.
    Returns (verts f32 [V][3], tris i32 [T][3], tri_mat i32 [T], tri_obj i32 [T])."""
    V, T, Mt, O = [], [], [], []
    base = 0
    for i, (q, X) in enumerate(zip(np.asarray(inst_proto), np.asarray(inst_xform, np.float32).reshape(-1, 3, 4))):
        pv, pt, pm = protos[int(q)]
        pv = np.asarray(pv, np.float32).reshape(-1, 3)
        x, y, z = pv[:, 0], pv[:, 1], pv[:, 2]
        w = np.empty_like(pv)
        for r in range(3):
            w[:, r] = ((X[r, 0] * x + X[r, 1] * y) + X[r, 2] * z) + X[r, 3]
        V.append(w)
        T.append(np.asarray(pt, np.int64).reshape(-1, 3) + base)
        Mt.append(np.asarray(pm, np.int32).reshape(-1))
        O.append(np.full(len(Mt[-1]), i, np.int32))
        base += len(pv)
    return (np.concatenate(V).astype(np.float32), np.concatenate(T).astype(np.int32), np.concatenate(Mt),
            np.concatenate(O))


def mic_centroid(mics):
    m = _c(mics, np.float32)
    R = np.zeros(3, dtype=np.float32)
    lib().ora_mic_centroid(len(m), _p(m), _p(R))
    return R


def trace(scene: Scene, s, q, dirs, B, r_max=1e9, t_min=1e-5, los_eps=1e-4, R=None, nthreads=0):
    s, q, dirs = _c(s, np.float32), _c(q, np.float32), _c(dirs, np.float32)
    N = len(dirs)
    R = _c(R, np.float32)
    rec = dict(tri=np.zeros((N, B), np.int32), p=np.zeros((N, B, 3), np.float32), d=np.zeros((N, B, 3), np.float32),
               r=np.zeros((N, B), np.float64), los=np.zeros((N, B), np.uint8))
    lib().ora_trace(scene.h, _p(scene.nrm), _p(s), _p(q), N, _p(dirs), B, r_max, t_min, los_eps, _p(R),
                    _p(rec["tri"]), _p(rec["p"]), _p(rec["d"]), _p(rec["r"]), _p(rec["los"]), nthreads)
    return rec


def diffraction_filter(scene: Scene, s, q, cand_tri, cand_p, fov_half=math.pi, cos_inc=None, theta_inc_deg=80.0,
                       t_min=1e-5, los_eps=1e-4, nthreads=0):
    s, q = _c(s, np.float32), _c(q, np.float32)
    ct, cp = _c(cand_tri, np.int32), _c(cand_p, np.float32)
    # the angles are float32 parameters of the interface: cos is taken of the float32 value
    f32 = lambda x: float(np.float32(x))
    cos_fov = np.float32(-2.0) if f32(fov_half) >= f32(math.pi) else np.float32(math.cos(f32(fov_half)))
    if cos_inc is None:
        cos_inc = np.float32(math.cos(f32(math.radians(theta_inc_deg))))
    keep = np.zeros(len(ct), dtype=np.uint8)
    lib().ora_diffraction_filter(scene.h, _p(scene.nrm), _p(s), _p(q), len(ct), _p(ct), _p(cp), float(cos_fov),
                                 float(cos_inc), t_min, los_eps, _p(keep), nthreads)
    return keep


def los_per_mic(scene: Scene, rec, mics, t_min=1e-5, los_eps=1e-4, nthreads=0):
    """Receiver test per microphone (Algorithm 1 leaves the receiver test unstated; the default casts one
    visibility ray per hit towards the microphones' centroid, this variant one ray per microphone):
    returns rec with 'mask' (uint64 [N][B], bit m = microphone m visible from the hit point) and 'los'
    (any microphone visible).  M <= 64."""
    m = _c(mics, np.float32)
    if not 1 <= len(m) <= 64:
        raise ValueError("per-microphone receiver test: 1 <= M <= 64")
    N, B = rec["tri"].shape
    mask = np.zeros((N, B), np.uint64)
    los = np.zeros((N, B), np.uint8)
    lib().ora_los_per_mic(scene.h, N * B, _p(_c(rec["tri"], np.int32)), _p(_c(rec["p"], np.float32)), len(m), _p(m),
                          t_min, los_eps, _p(mask), _p(los), nthreads)
    return dict(rec, mask=mask, los=los)


def direct_visibility(scene: Scene, s, mics, t_min=1e-5, los_eps=1e-4):
    s, m = _c(s, np.float32), _c(mics, np.float32)
    vis = np.zeros(len(m), dtype=np.uint8)
    lib().ora_direct_visibility(scene.h, _p(s), len(m), _p(m), t_min, los_eps, _p(vis))
    return vis


# ------------------------------------------------------------------------------------ spectra
class _Keep:
    """keeps numpy buffers alive while a SpecParams points into them"""


def spec_params(wl, mics=None, k_band=None, emitter=None, c=343.0, a0=0.0, a1_per_khz=0.033,
                reflection_mode=0, direct_gain=1.0, beta_band=None):
    keep = _Keep()
    keep.band = _c(wl.band_hz, np.float32)
    keep.k = _c(wl.k_band if k_band is None else k_band, np.float32)
    keep.beta = _c(wl.beta_band if beta_band is None else beta_band, np.float32)
    keep.diff = _c(wl.diff_band, np.float32)
    keep.mics = _c(wl.mics if mics is None else mics, np.float32)
    keep.s = _c(wl.emitter if emitter is None else emitter, np.float32)
    keep.q = _c(wl.emitter_quat, np.float32)
    keep.et = _c(wl.emitter_table, np.float32)
    keep.mt = _c(wl.mic_tables, np.float32)
    keep.mq = _c(wl.mic_quats, np.float32)
    P_ = SpecParams()
    P_.F, P_.f_lo, P_.f_hi, P_.c, P_.a0, P_.a1_per_khz = wl.n_bins, wl.f_lo, wl.f_hi, c, a0, a1_per_khz
    P_.n_mat, P_.n_bands = keep.k.shape
    P_.band_hz, P_.k_band, P_.beta_band, P_.diff_band = _p(keep.band), _p(keep.k), _p(keep.beta), _p(keep.diff)
    P_.M = len(keep.mics)
    P_.mics, P_.mic_quats, P_.mic_tables = _p(keep.mics), _p(keep.mq), _p(keep.mt)
    if keep.mt is not None:
        P_.n_el, P_.n_az = keep.mt.shape[1], keep.mt.shape[2]
    P_.s, P_.q, P_.emit_table = _p(keep.s), _p(keep.q), _p(keep.et)
    P_.n_theta = 0 if keep.et is None else keep.et.shape[0]
    P_.reflection_mode, P_.direct_gain = reflection_mode, direct_gain
    keep.P = P_
    return keep


def spectra(params, rec, dirs, tri_mat, cand_tri=None, cand_p=None, cand_keep=None, direct_vis=None,
            ms=None, ks=None, nthreads=0):
    """Returns complex128 [3][n_m][n_k] (specular, diffraction, direct)."""
    P_ = params.P
    N, B = rec["tri"].shape
    dirs, tm = _c(dirs, np.float32), _c(tri_mat, np.int32)
    ct, cp, ck = _c(cand_tri, np.int32), _c(cand_p, np.float32), _c(cand_keep, np.uint8)
    dv = _c(direct_vis, np.uint8)
    K = 0 if ct is None else len(ct)
    msa, ksa = _c(ms, np.int32), _c(ks, np.int32)
    nm = P_.M if msa is None else len(msa)
    nk = P_.F if ksa is None else len(ksa)
    out = np.zeros((3, nm, nk, 2), dtype=np.float64)
    lib().ora_spectra(C.byref(P_), N, B, _p(rec["tri"]), _p(rec["p"]), _p(rec["d"]), _p(rec["r"]), _p(rec["los"]),
                      _p(dirs), _p(tm), K, _p(ct), _p(cp), _p(ck), _p(dv), nm, _p(msa), nk, _p(ksa), nthreads,
                      _p(_c(rec.get("mask"), np.uint64)), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def spectra_grad(params, rec, dirs, tri_mat, G, cand_tri=None, cand_p=None, cand_keep=None, direct_vis=None,
                 with_beta=False, tri_nrm=None):
    """G: complex [3][M][F] = dL/dRe S + j dL/dIm S.  Returns (dk [n_mat][n_bands], dmic [M][3], demit [3]),
    and dbeta [n_mat][n_bands] (lobe widths, specular paths) as a fourth item when with_beta.  demit holds
    the diffraction and direct paths; given the triangle normals tri_nrm [T][3], it also holds the
    specular paths through their hit points (ray directions and triangle chains frozen).  Records carrying
    'mask' (the per-microphone receiver test) reach only the microphones whose bit is set."""
    P_ = params.P
    N, B = rec["tri"].shape
    dirs, tm = _c(dirs, np.float32), _c(tri_mat, np.int32)
    ct, cp, ck = _c(cand_tri, np.int32), _c(cand_p, np.float32), _c(cand_keep, np.uint8)
    dv = _c(direct_vis, np.uint8)
    K = 0 if ct is None else len(ct)
    Gr = np.ascontiguousarray(np.stack([np.real(G), np.imag(G)], -1), dtype=np.float64)
    dk = np.zeros((P_.n_mat, P_.n_bands), np.float64)
    dmic = np.zeros((P_.M, 3), np.float64)
    demit = np.zeros(3, np.float64)
    dbeta = np.zeros((P_.n_mat, P_.n_bands), np.float64) if with_beta else None
    nrm = _c(tri_nrm, np.float32)
    dspec = np.zeros(3, np.float64) if nrm is not None else None
    rc = lib().ora_spectra_grad(C.byref(P_), N, B, _p(rec["tri"]), _p(rec["p"]), _p(rec["d"]), _p(rec["r"]),
                                _p(rec["los"]), _p(dirs), _p(tm), K, _p(ct), _p(cp), _p(ck), _p(dv), _p(Gr),
                                _p(dk), _p(dmic), _p(demit), _p(dbeta), _p(nrm), _p(dspec),
                                _p(_c(rec.get("mask"), np.uint64)))
    if rc != 0:
        raise ValueError("oracle gradient needs omni emitter and microphones")
    if dspec is not None:
        demit = demit + dspec
    return (dk, dmic, demit, dbeta) if with_beta else (dk, dmic, demit)


# ------------------------------------------------------------------------------------ pipeline
def simulate(wl, *, c=343.0, a0=0.0, a1_per_khz=0.033, t_min=1e-5, los_eps=1e-4, reflection_mode=0,
             direct_gain=1.0, theta_inc_deg=80.0, curv=None, seed=0, pose=0, components=7, use_bvh=None,
             ms=None, ks=None, nthreads=0, ray_subset=None, los_mode=0):
    """The whole hot path on the CPU for one workload.  Returns a dict with the path records,
    diffraction candidates and spectra (complex128 [3][M][F]).  los_mode 1: the receiver test of each record
    is made per microphone (records then carry 'mask')."""
    curv = dict(eta=1.0, area_ref=1e-4, dither=1e-3, hc_frac=0.25, samples_per_vertex=64, budget=4_000_000,
                seed=0) | (curv or {})
    scene = Scene(wl.verts, wl.tris, use_bvh=use_bvh)
    R = mic_centroid(wl.mics)
    dirs = wl.dirs if ray_subset is None else wl.dirs[ray_subset]
    rec = trace(scene, wl.emitter, wl.emitter_quat, dirs, wl.bounces, r_max=wl.max_distance, t_min=t_min,
                los_eps=los_eps, R=R, nthreads=nthreads)
    if los_mode == 1:
        rec = los_per_mic(scene, rec, wl.mics, t_min, los_eps, nthreads)
    out = dict(rec=rec, R=R, scene=scene)
    cand_tri = cand_p = keep = None
    if wl.diffraction and (components & 2):
        G = curvature(wl.verts, wl.tris)
        Cm = tri_metric(wl.verts, wl.tris, G, curv["eta"], curv["area_ref"])
        cd = diffraction_cdf(wl.verts, wl.tris, Cm, wl.tri_obj, curv["dither"], curv["seed"], curv["hc_frac"],
                             curv["samples_per_vertex"], curv["budget"])
        cand_tri, cand_p = diffraction_samples(wl.verts, wl.tris, cd, seed=seed, pose=pose)
        keep = diffraction_filter(scene, wl.emitter, wl.emitter_quat, cand_tri, cand_p, fov_half=wl.fov_half,
                                  theta_inc_deg=theta_inc_deg, t_min=t_min, los_eps=los_eps, nthreads=nthreads)
        out.update(G=G, C=Cm, cdf=cd, cand_tri=cand_tri, cand_p=cand_p, cand_keep=keep)
    dvis = direct_visibility(scene, wl.emitter, wl.mics, t_min, los_eps) if (components & 4) else None
    out["direct_vis"] = dvis
    params = spec_params(wl, c=c, a0=a0, a1_per_khz=a1_per_khz, reflection_mode=reflection_mode,
                         direct_gain=direct_gain)
    recs = rec if (components & 1) else dict(rec, tri=np.full_like(rec["tri"], -1))
    out["params"] = params
    out["spectra"] = spectra(params, recs, dirs, wl.tri_mat, cand_tri, cand_p, keep, dvis, ms=ms, ks=ks,
                             nthreads=nthreads)
    return out
