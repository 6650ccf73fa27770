"""Seeded synthetic inputs for the acoustic path-tracing hot path.

This module only *makes inputs*: triangle meshes, sensor poses, microphone arrays,
per-band material curves, ray-direction sets and directivity tables.  It holds none
of the simulator's arithmetic (no intersection, reflection, curvature, sampling or
spectrum synthesis), so that the CUDA path and the CPU oracle can both read the
same inputs while sharing no code.

Workload shapes follow the paper's experiments (Sec. IV-A bioacoustics: 64-mic
array, ~600k rays, 3 hits; Sec. IV-B robotics: 32-mic array, 80k rays, 3 hits;
Sec. IV-C scaling sweeps).  The paper's own scenes (scorpion/pebbles, office
lobby, forest) are not available, so procedural scenes of the same kind stand in.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

F32 = np.float32


# --------------------------------------------------------------------------- rays
def fibonacci_directions(n: int) -> np.ndarray:
    """Fibonacci-sphere unit directions, computed in float64 and rounded to float32.

    The ray-angle set is an input of Algorithm 1 ("Ray Angles"); the paper's own
    set is a zonal equal-area partition, the workloads here use the Fibonacci
    lattice: z_i = 1 - (2i+1)/n, phi_i = i * pi * (3 - sqrt 5).
    """
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    d = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    return d.astype(F32)


# --------------------------------------------------------------------------- meshes
def _box_tris(lo, hi):
    """12 triangles of an axis-aligned box, two per wall.  Returns verts, tris, wall id per tri
    (0: z=lo floor, 1: z=hi ceiling, 2: x=lo, 3: x=hi, 4: y=lo, 5: y=hi)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=F32)
    quads = [(0, 1, 2, 3, 0), (4, 7, 6, 5, 1), (0, 3, 7, 4, 2), (1, 5, 6, 2, 3),
             (0, 4, 5, 1, 4), (3, 2, 6, 7, 5)]
    tris, wall = [], []
    for a, b, c, d, w in quads:
        tris += [[a, b, c], [a, c, d]]
        wall += [w, w]
    return v, np.array(tris, dtype=np.int32), np.array(wall, dtype=np.int32)


def icosphere(subdiv: int):
    """Unit icosphere with shared vertices (each edge midpoint created once)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    for _ in range(subdiv):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e = np.sort(e, axis=1)
        ue, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = v[ue[:, 0]] + v[ue[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        base = len(v)
        v = np.concatenate([v, mid], axis=0)
        nf = len(f)
        m01 = base + inv[0:nf]
        m12 = base + inv[nf:2 * nf]
        m20 = base + inv[2 * nf:3 * nf]
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], 1), np.stack([f[:, 1], m12, m01], 1),
            np.stack([f[:, 2], m20, m12], 1), np.stack([m01, m12, m20], 1)], axis=0)
    return v, f


def uv_sphere(n_lat: int, n_lon: int):
    """Unit latitude-longitude sphere: two pole vertices, n_lat - 1 rings of n_lon vertices, each quad
    between rings split along one diagonal, pole fans (about half of its triangles are obtuse)."""
    V = [[0.0, 0.0, 1.0]]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2.0 * math.pi * j / n_lon
            V.append([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    V.append([0.0, 0.0, -1.0])
    south = len(V) - 1
    F = [[0, 1 + j, 1 + (j + 1) % n_lon] for j in range(n_lon)]
    for i in range(n_lat - 2):
        for j in range(n_lon):
            a, b = 1 + i * n_lon + j, 1 + i * n_lon + (j + 1) % n_lon
            F += [[a, a + n_lon, b + n_lon], [a, b + n_lon, b]]
    last = 1 + (n_lat - 2) * n_lon
    F += [[last + j, south, last + (j + 1) % n_lon] for j in range(n_lon)]
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int64)


def cylinder(radius: float, height: float, seg: int):
    """Closed vertical cylinder (side quads + two cap fans), base at z=0."""
    a = np.arange(seg) * (2.0 * math.pi / seg)
    ring = np.stack([radius * np.cos(a), radius * np.sin(a)], 1)
    bot = np.concatenate([ring, np.zeros((seg, 1))], 1)
    top = np.concatenate([ring, np.full((seg, 1), height)], 1)
    v = np.concatenate([bot, top, [[0, 0, 0]], [[0, 0, height]]], 0)
    cb, ct = 2 * seg, 2 * seg + 1
    i = np.arange(seg)
    j = (i + 1) % seg
    side1 = np.stack([i, j, seg + j], 1)
    side2 = np.stack([i, seg + j, seg + i], 1)
    capb = np.stack([np.full(seg, cb), j, i], 1)
    capt = np.stack([np.full(seg, ct), seg + i, seg + j], 1)
    return v, np.concatenate([side1, side2, capb, capt], 0)


def leaf_disc(seg: int = 8):
    """Flat unit disc in the xy plane as a triangle fan (centre + seg rim vertices)."""
    a = np.arange(seg) * (2.0 * math.pi / seg)
    v = np.concatenate([[[0.0, 0.0, 0.0]], np.stack([np.cos(a), np.sin(a), np.zeros(seg)], 1)], 0)
    i = np.arange(seg)
    f = np.stack([np.zeros(seg, dtype=np.int64), 1 + i, 1 + (i + 1) % seg], 1)
    return v, f


def _random_rotations(rng, n):
    """Uniform random rotation matrices (from random unit quaternions)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], 1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], 1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], 1)], 1)


# --------------------------------------------------------------------------- materials
def smooth_band_curves(rng, n_mat: int, n_bands: int, lo: float, hi: float) -> np.ndarray:
    """Per-material smooth random curves over the bands: a sum of three random cosines,
    mapped affinely into [lo, hi]."""
    x = np.linspace(0.0, 1.0, n_bands)
    out = np.empty((n_mat, n_bands), dtype=np.float64)
    for m in range(n_mat):
        s = np.zeros(n_bands)
        for _ in range(3):
            s += rng.uniform(0.3, 1.0) * np.cos(2 * math.pi * rng.uniform(0.2, 1.5) * x + rng.uniform(0, 2 * math.pi))
        s = (s - s.min()) / max(s.max() - s.min(), 1e-12)
        out[m] = lo + (hi - lo) * s
    return out.astype(F32)


# --------------------------------------------------------------------------- arrays
def planar_disc_array(rng, n: int, radius: float, centre, normal_axis: int = 0) -> np.ndarray:
    """n microphone positions uniform in a disc of the given radius, in the plane
    perpendicular to coordinate axis `normal_axis`, centred at `centre`."""
    r = radius * np.sqrt(rng.uniform(0, 1, n))
    a = rng.uniform(0, 2 * math.pi, n)
    u, w = [ax for ax in range(3) if ax != normal_axis]
    p = np.tile(np.asarray(centre, dtype=np.float64), (n, 1))
    p[:, u] += r * np.cos(a)
    p[:, w] += r * np.sin(a)
    return p.astype(F32)


# --------------------------------------------------------------------------- directivity
def piston_table(radius_m: float, freqs_hz: np.ndarray, c: float = 343.0, n_theta: int = 1801) -> np.ndarray:
    """Emitter directivity table [n_theta][F] of a baffled circular piston,
    |2 J1(ka sin th) / (ka sin th)|, th uniform on [0, pi].  Evaluated with SciPy's J1."""
    from scipy.special import j1
    th = np.linspace(0.0, math.pi, n_theta)
    k = 2 * math.pi * np.asarray(freqs_hz, dtype=np.float64) / c
    x = np.outer(np.sin(th), k * radius_m)
    with np.errstate(invalid="ignore", divide="ignore"):
        d = np.where(x > 1e-12, 2 * j1(x) / np.where(x > 1e-12, x, 1.0), 1.0)
    return np.abs(d).astype(F32)


def ear_table(rng, n_az: int = 180, n_el: int = 91, n_bands: int = 16) -> np.ndarray:
    """Smooth random receiver directivity on a 2-degree (az, el) grid x bands, values in [0.05, 1].
    Layout [n_el][n_az][n_bands]; az = -180 + 2*i degrees, el = -90 + 2*j degrees."""
    az = np.deg2rad(-180.0 + 360.0 * np.arange(n_az) / n_az)
    el = np.deg2rad(np.linspace(-90.0, 90.0, n_el))
    E, A = np.meshgrid(el, az, indexing="ij")
    dirs = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1)
    out = np.empty((n_el, n_az, n_bands))
    lobe = rng.normal(size=3)
    lobe /= np.linalg.norm(lobe)
    lobe = 0.5 * lobe + np.array([0.8, 0.0, 0.0])
    lobe /= np.linalg.norm(lobe)
    for b in range(n_bands):
        sharp = 1.0 + 4.0 * b / max(n_bands - 1, 1)
        v = np.exp(sharp * (dirs @ lobe - 1.0))
        for _ in range(3):
            w = rng.normal(size=3)
            w /= np.linalg.norm(w)
            v *= 1.0 + 0.15 * np.cos(3.0 * (dirs @ w) + rng.uniform(0, 2 * math.pi))
        out[:, :, b] = v
    out = 0.05 + 0.95 * (out - out.min()) / (out.max() - out.min())
    return out.astype(F32)


# --------------------------------------------------------------------------- workloads
@dataclass
class Workload:
    """One simulation problem: scene + materials + sensor + frequency grid + tracing parameters."""
    name: str
    verts: np.ndarray            # [V][3] f32
    tris: np.ndarray             # [T][3] i32
    tri_mat: np.ndarray          # [T] i32
    tri_obj: np.ndarray          # [T] i32 (mesh id; diffraction CDFs are per mesh)
    band_hz: np.ndarray          # [n_bands] f32 ascending
    k_band: np.ndarray           # [n_mat][n_bands] f32 reflection magnitude
    beta_band: np.ndarray        # [n_mat][n_bands] f32 lobe opening angle (rad)
    diff_band: np.ndarray        # [n_mat][n_bands] f32 diffraction coefficient
    emitter: np.ndarray          # [3] f32
    emitter_quat: np.ndarray     # [4] f32 (w, x, y, z); forward = rotated +x
    dirs: np.ndarray             # [N][3] f32 local ray directions
    mics: np.ndarray             # [M][3] f32
    n_bins: int
    f_lo: float
    f_hi: float
    bounces: int
    max_distance: float = 100.0
    diffraction: bool = False
    fov_half: float = math.pi
    emitter_table: np.ndarray | None = None   # [n_theta][F] f32 or None (omni)
    mic_tables: np.ndarray | None = None      # [M][n_el][n_az][n_bands] f32 or None (omni)
    mic_quats: np.ndarray | None = None       # [M][4] f32 or None (identity)
    extra: dict = field(default_factory=dict)

    @property
    def n_tris(self):
        return int(self.tris.shape[0])


def _identity_quat():
    return np.array([1.0, 0.0, 0.0, 0.0], dtype=F32)


def shoebox(seed: int = 101, n_rays: int = 10_000, bounces: int = 3, n_bins: int = 128,
            n_mics: int = 1, four_materials: bool = False, absorption: float = 0.1,
            beta_deg: float = 10.0) -> Workload:
    """4 x 3 x 2.5 m shoebox room, 12 triangles, one omni emitter, omni microphone(s)
    at seeded uniform positions (0.1 m margin), Fibonacci rays, 20-80 kHz.

    With four_materials the walls get four materials (floor, ceiling, x walls, y walls)
    with smooth random band curves, and the microphones form a 32-mic 12 cm disc array."""
    rng = np.random.default_rng(seed)
    L = np.array([4.0, 3.0, 2.5])
    v, t, wall = _box_tris((0.0, 0.0, 0.0), tuple(L))
    margin = 0.1
    s = rng.uniform(margin, L - margin).astype(F32)
    n_bands = 16
    band = np.linspace(20e3, 80e3, n_bands).astype(F32)
    if four_materials:
        mat = np.array([0, 1, 2, 2, 3, 3], dtype=np.int32)[wall]
        k = smooth_band_curves(rng, 4, n_bands, 0.3, 0.95)
        beta = np.deg2rad(smooth_band_curves(rng, 4, n_bands, 5.0, 30.0)).astype(F32)
        diff = np.full((4, n_bands), 0.05, dtype=F32)
        centre = np.clip(rng.uniform(margin + 0.1, L - margin - 0.1), 0.2, None)
        mics = planar_disc_array(rng, n_mics if n_mics > 1 else 32, 0.06, centre, 0)
    else:
        mat = np.zeros(12, dtype=np.int32)
        k = np.full((1, n_bands), 1.0 - absorption, dtype=F32)
        beta = np.full((1, n_bands), math.radians(beta_deg), dtype=F32)
        diff = np.full((1, n_bands), 0.05, dtype=F32)
        mics = rng.uniform(margin, L - margin, size=(n_mics, 3)).astype(F32)
    return Workload(
        name="shoebox", verts=v, tris=t, tri_mat=mat, tri_obj=np.zeros(12, dtype=np.int32),
        band_hz=band, k_band=k.astype(F32), beta_band=beta.astype(F32), diff_band=diff,
        emitter=s, emitter_quat=_identity_quat(), dirs=fibonacci_directions(n_rays), mics=mics,
        n_bins=n_bins, f_lo=20e3, f_hi=80e3, bounces=bounces, max_distance=1e9,
        extra={"room": L.astype(F32), "wall": wall})


def clutter(seed: int = 202, target_tris: int = 200_000, n_rays: int = 1_000_000, bounces: int = 5,
            n_mics: int = 32, n_bins: int = 512, diffraction: bool = True) -> Workload:
    """Procedural clutter in a 20 x 20 x 5 m volume: a ground plane plus subdivided icospheres
    (radius log-uniform 0.05-0.5 m) and closed cylinders (r 0.02-0.2 m, h 0.2-3 m, 16-32
    segments) until ~target_tris triangles; 4 materials with smooth random band curves;
    a sensor (omni emitter + 32-mic 12 cm planar disc array facing +x) 1 m above the ground."""
    rng = np.random.default_rng(seed)
    sensor = np.array([10.0, 10.0, 1.0])
    V = [np.array([[0, 0, 0], [20, 0, 0], [20, 20, 0], [0, 20, 0]], dtype=np.float64)]
    Fc = [np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int64)]
    mats = [np.zeros(2, dtype=np.int32)]
    objs = [np.zeros(2, dtype=np.int32)]
    n_t, base, obj = 2, 4, 1
    ico_cache = {s: icosphere(s) for s in (2, 3, 4)}
    while n_t < target_tris:
        if rng.uniform() < 0.5:
            r = math.exp(rng.uniform(math.log(0.05), math.log(0.5)))
            sub = 2 if r < 0.12 else (3 if r < 0.25 else 4)
            c = np.array([rng.uniform(r, 20 - r), rng.uniform(r, 20 - r), rng.uniform(r, 5 - r)])
            if np.linalg.norm(c - sensor) < r + 0.6:
                continue
            v, f = ico_cache[sub]
            v = v * r + c
        else:
            r = rng.uniform(0.02, 0.2)
            h = rng.uniform(0.2, 3.0)
            seg = int(rng.integers(16, 33))
            c = np.array([rng.uniform(1, 19), rng.uniform(1, 19), 0.0])
            if np.linalg.norm((c - sensor)[:2]) < r + 0.6:
                continue
            v, f = cylinder(r, h, seg)
            v = v + c
        V.append(v)
        Fc.append(f + base)
        m = int(rng.integers(0, 4))
        mats.append(np.full(len(f), m, dtype=np.int32))
        objs.append(np.full(len(f), obj, dtype=np.int32))
        base += len(v)
        n_t += len(f)
        obj += 1
    n_bands = 16
    band = np.linspace(20e3, 80e3, n_bands).astype(F32)
    k = smooth_band_curves(rng, 4, n_bands, 0.3, 0.95)
    beta = np.deg2rad(smooth_band_curves(rng, 4, n_bands, 5.0, 30.0)).astype(F32)
    diff = smooth_band_curves(rng, 4, n_bands, 0.02, 0.08)
    mics = planar_disc_array(rng, n_mics, 0.06, sensor, 0)
    emitter = (sensor + np.array([0.01, 0.0, 0.0])).astype(F32)
    return Workload(
        name="clutter", verts=np.concatenate(V).astype(F32), tris=np.concatenate(Fc).astype(np.int32),
        tri_mat=np.concatenate(mats), tri_obj=np.concatenate(objs), band_hz=band, k_band=k,
        beta_band=beta, diff_band=diff, emitter=emitter, emitter_quat=_identity_quat(),
        dirs=fibonacci_directions(n_rays), mics=mics, n_bins=n_bins, f_lo=20e3, f_hi=80e3,
        bounces=bounces, max_distance=60.0, diffraction=diffraction)


def vegetation(seed: int = 303, target_tris: int = 2_000_000, n_rays: int = 4_000_000, bounces: int = 4,
               n_bins: int = 1024, leaves_per_mesh: int = 256, diffraction: bool = True) -> Workload:
    """Bat-like vegetation: leaf discs (8-triangle fans, radius 2-5 cm, uniform random
    orientation) placed by a homogeneous Poisson process in a 6 m sphere (a 0.3 m ball around
    the bat is kept clear); a piston emitter (a = 2 mm) facing +x at the centre and two ears at
    +-1 cm with smooth random directivity on a 2-degree grid; 20-120 kHz."""
    rng = np.random.default_rng(seed)
    n_leaves = target_tris // 8
    u = rng.normal(size=(n_leaves, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    rad = 6.0 * np.cbrt(rng.uniform((0.3 / 6.0) ** 3, 1.0, n_leaves))
    centres = u * rad[:, None]
    radii = rng.uniform(0.02, 0.05, n_leaves)
    R = _random_rotations(rng, n_leaves)
    lv, lf = leaf_disc(8)
    verts = np.einsum("nij,kj->nki", R, lv) * radii[:, None, None] + centres[:, None, :]
    tris = lf[None, :, :] + (np.arange(n_leaves) * len(lv))[:, None, None]
    n_bands = 16
    band = np.linspace(20e3, 120e3, n_bands).astype(F32)
    n_mat = 2
    k = smooth_band_curves(rng, n_mat, n_bands, 0.3, 0.9)
    beta = np.deg2rad(smooth_band_curves(rng, n_mat, n_bands, 5.0, 30.0)).astype(F32)
    diff = smooth_band_curves(rng, n_mat, n_bands, 0.02, 0.08)
    leaf_mat = rng.integers(0, n_mat, n_leaves).astype(np.int32)
    leaf_obj = (np.arange(n_leaves) // leaves_per_mesh).astype(np.int32)
    freqs = np.linspace(20e3, 120e3, n_bins)
    mics = np.array([[0.0, 0.01, 0.0], [0.0, -0.01, 0.0]], dtype=F32)
    tables = np.stack([ear_table(rng), ear_table(rng)[:, ::-1, :].copy()])
    return Workload(
        name="vegetation", verts=verts.reshape(-1, 3).astype(F32), tris=tris.reshape(-1, 3).astype(np.int32),
        tri_mat=np.repeat(leaf_mat, 8), tri_obj=np.repeat(leaf_obj, 8), band_hz=band, k_band=k,
        beta_band=beta, diff_band=diff, emitter=np.zeros(3, dtype=F32), emitter_quat=_identity_quat(),
        dirs=fibonacci_directions(n_rays), mics=mics, n_bins=n_bins, f_lo=20e3, f_hi=120e3,
        bounces=bounces, max_distance=30.0, diffraction=diffraction, fov_half=math.pi / 2,
        emitter_table=piston_table(0.002, freqs), mic_tables=tables,
        mic_quats=np.tile(_identity_quat(), (2, 1)))


@dataclass
class InstancedScene:
    """Shared meshes and their instances (the scene's world triangles are made by the code under test)."""
    protos: list                 # [(verts f32 [v][3], tris i32 [t][3] local indices, tri_mat i32 [t]), ...]
    inst_proto: np.ndarray       # [n_inst] i32 prototype of each instance
    inst_xform: np.ndarray       # [n_inst][3][4] f32 row-major [A | b]: x -> A x + b
    base: Workload               # sensor, materials, rays, grid; its own geometry arrays are empty


def _plant_protos():
    """Plant meshes with their base at the origin: a trunk (closed cylinder) under an icosphere crown, a
    bush (icosphere resting on the ground), a rock (box)."""
    tv, tf = cylinder(0.08, 2.0, 12)
    cv, cf = icosphere(2)
    cv = cv * 0.7 + np.array([0.0, 0.0, 2.5])
    tree_v = np.concatenate([tv, cv])
    tree_f = np.concatenate([tf, cf + len(tv)])
    tree_m = np.concatenate([np.full(len(tf), 1), np.full(len(cf), 2)])
    bv, bf = icosphere(3)
    bv = bv * 0.45 + np.array([0.0, 0.0, 0.45])
    rv, rf, _ = _box_tris((-0.3, -0.2, 0.0), (0.3, 0.2, 0.25))
    return [(tree_v.astype(F32), tree_f.astype(np.int32), tree_m.astype(np.int32)),
            (bv.astype(F32), bf.astype(np.int32), np.full(len(bf), 2, np.int32)),
            (rv.astype(F32), rf.astype(np.int32), np.full(len(rf), 3, np.int32))]


def instanced_forest(seed: int = 606, n_inst: int = 400, n_rays: int = 100_000, bounces: int = 3, n_mics: int = 8,
                     n_bins: int = 128, diffraction: bool = True) -> InstancedScene:
    """A forest floor as instances of a few shared meshes (the paper's forest repeats plant models):
    prototype 0 a 20 x 20 m ground quad (one instance, identity), prototypes 1-3 a tree, a bush and a
    rock placed uniformly in the area outside a 1.5 m clearing around the sensor, each rotated about the
    vertical by a uniform angle and scaled uniformly by 0.6-1.4 (rocks also tilted by up to 30 degrees
    about a horizontal axis); 4 materials; a 12 cm disc array of n_mics microphones with an omni emitter
    1 m above the centre."""
    rng = np.random.default_rng(seed)
    ground = (np.array([[0, 0, 0], [20, 0, 0], [20, 20, 0], [0, 20, 0]], F32), np.array([[0, 1, 2], [0, 2, 3]], np.int32),
              np.zeros(2, np.int32))
    protos = [ground] + _plant_protos()
    sensor = np.array([10.0, 10.0, 1.0])
    xf = [np.concatenate([np.eye(3), np.zeros((3, 1))], 1)]
    kind = [0]
    while len(kind) < n_inst:
        c = np.array([rng.uniform(0.5, 19.5), rng.uniform(0.5, 19.5), 0.0])
        if np.linalg.norm((c - sensor)[:2]) < 1.5:
            continue
        q = int(rng.integers(1, 4))
        a = rng.uniform(0, 2 * math.pi)
        Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
        if q == 3:
            t = rng.uniform(0, math.radians(30))
            Rz = Rz @ np.array([[1, 0, 0], [0, math.cos(t), -math.sin(t)], [0, math.sin(t), math.cos(t)]])
        xf.append(np.concatenate([Rz * rng.uniform(0.6, 1.4), c[:, None]], 1))
        kind.append(q)
    n_bands = 16
    band = np.linspace(20e3, 80e3, n_bands).astype(F32)
    empty = np.zeros((0, 3), F32)
    base = Workload(
        name="instanced_forest", verts=empty, tris=np.zeros((0, 3), np.int32), tri_mat=np.zeros(0, np.int32),
        tri_obj=np.zeros(0, np.int32), band_hz=band, k_band=smooth_band_curves(rng, 4, n_bands, 0.3, 0.95),
        beta_band=np.deg2rad(smooth_band_curves(rng, 4, n_bands, 5.0, 30.0)).astype(F32),
        diff_band=smooth_band_curves(rng, 4, n_bands, 0.02, 0.08),
        emitter=(sensor + np.array([0.01, 0.0, 0.0])).astype(F32), emitter_quat=_identity_quat(),
        dirs=fibonacci_directions(n_rays), mics=planar_disc_array(rng, n_mics, 0.06, sensor, 0), n_bins=n_bins,
        f_lo=20e3, f_hi=80e3, bounces=bounces, max_distance=60.0, diffraction=diffraction)
    return InstancedScene(protos=protos, inst_proto=np.array(kind, np.int32),
                          inst_xform=np.array(xf, np.float64).astype(F32), base=base)


def gradient_problem(seed: int = 404, n_rays: int = 10_000) -> Workload:
    """Shoebox geometry with four wall materials, a 32-mic disc array and 128 bins
    (the differentiation workload)."""
    return shoebox(seed=seed, n_rays=n_rays, bounces=3, n_bins=128, n_mics=32, four_materials=True)


def batched_poses(seed: int = 505, n_scenes: int = 16, poses_per_scene: int = 16,
                  tri_lo: float = 1e4, tri_hi: float = 2e6, scale: float = 1.0):
    """Job list for the batched form: n_scenes procedural scenes (triangle counts log-uniform
    in [tri_lo, tri_hi], 1-4 materials) with poses_per_scene sensor poses each; per pose the mic
    count is uniform in 2..64, bins in 256..2048, bounces in 1..5."""
    rng = np.random.default_rng(seed)
    jobs = []
    scenes = []
    for s in range(n_scenes):
        T = int(math.exp(rng.uniform(math.log(tri_lo), math.log(tri_hi))) * scale)
        wl = clutter(seed=int(rng.integers(1 << 30)), target_tris=max(T, 100), n_rays=1, n_mics=2, n_bins=256)
        n_mat = int(rng.integers(1, 5))
        wl.tri_mat = (wl.tri_mat % n_mat).astype(np.int32)
        wl.k_band = wl.k_band[:n_mat].copy()
        wl.beta_band = wl.beta_band[:n_mat].copy()
        wl.diff_band = wl.diff_band[:n_mat].copy()
        scenes.append(wl)
        for p in range(poses_per_scene):
            M = int(rng.integers(2, 65))
            F = int(rng.integers(256, 2049))
            B = int(rng.integers(1, 6))
            centre = np.array([rng.uniform(8, 12), rng.uniform(8, 12), rng.uniform(0.5, 1.5)])
            jobs.append(dict(scene=s, n_mics=M, n_bins=F, bounces=B,
                             mics=planar_disc_array(rng, M, 0.06, centre, 0),
                             emitter=(centre + np.array([0.01, 0, 0])).astype(F32),
                             pose_index=p))
    return scenes, jobs
