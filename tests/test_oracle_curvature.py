"""Pins for the oracle's pre-processing (Sec. III-B, Eq. 1) and diffraction sampling (Sec. III-D):
Meyer mean curvature on surfaces with known curvature, welding, the metric's high-pass behaviour,
exact integer CDFs, sample-count rule and the sampled distribution."""
import math

import numpy as np
import pytest

import oracle
import synth


def _sphere(R, sub):
    v, f = synth.icosphere(sub)
    return (v * R).astype(np.float32), f.astype(np.int32)


@pytest.mark.parametrize("R", [0.3, 2.0])
def test_sphere_curvature(R):
    v, f = _sphere(R, 4)            # 2562 vertices
    G = oracle.curvature(v, f)
    assert np.allclose(G, 1.0 / R, rtol=0.02)


def _tube(r, h, seg, rings):
    a = np.arange(seg) * 2 * math.pi / seg
    V, F = [], []
    for j in range(rings):
        z = h * j / (rings - 1)
        V += [[r * math.cos(t), r * math.sin(t), z] for t in a]
    for j in range(rings - 1):
        for i in range(seg):
            i2 = (i + 1) % seg
            p, q, s_, t_ = j * seg + i, j * seg + i2, (j + 1) * seg + i2, (j + 1) * seg + i
            F += [[p, q, s_], [p, s_, t_]]
    return np.array(V, np.float32), np.array(F, np.int32)


def test_cylinder_curvature():
    r = 0.5
    v, f = _tube(r, 1.0, 96, 41)
    G = oracle.curvature(v, f)
    inner = G[96:-96]                       # skip the two open boundary rings
    assert np.allclose(inner, 1.0 / (2 * r), rtol=0.03)


def test_plane_curvature_zero_and_metric():
    n = 12
    xs, ys = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n), indexing="ij")
    v = np.stack([xs.ravel(), ys.ravel(), np.zeros(n * n)], 1).astype(np.float32)
    F = []
    for i in range(n - 1):
        for j in range(n - 1):
            a, b, c, d = i * n + j, (i + 1) * n + j, (i + 1) * n + j + 1, i * n + j + 1
            F += [[a, b, c], [a, c, d]]
    f = np.array(F, np.int32)
    G = oracle.curvature(v, f)
    interior = [i * n + j for i in range(1, n - 1) for j in range(1, n - 1)]
    assert np.max(np.abs(G[interior])) <= 1e-6
    C = oracle.tri_metric(v, f, G, 1.0, 1e-4)
    assert np.all(C >= 0)


def test_weld_and_duplicated_vertices():
    """A sphere whose triangles each own private vertex copies welds back to the shared mesh."""
    v, f = _sphere(1.0, 3)
    G0 = oracle.curvature(v, f)
    v2 = v[f.reshape(-1)]                    # 3 private copies per triangle
    f2 = np.arange(len(v2), dtype=np.int32).reshape(-1, 3)
    w = oracle.weld(v2)
    assert np.array_equal(v2[w], v2)
    assert len(np.unique(w)) == len(v)
    G2 = oracle.curvature(v2, f2)
    assert np.array_equal(G2, G0[f.reshape(-1)])


def test_metric_high_pass():
    """C_i vanishes on a smooth closed sphere and is large at a cylinder's cap rim (Eq. 1)."""
    v, f = _sphere(0.5, 3)
    G = oracle.curvature(v, f)
    C = oracle.tri_metric(v, f, G)
    cv, cf = synth.cylinder(0.1, 1.0, 24)
    cv = cv.astype(np.float32)
    cf = cf.astype(np.int32)
    Gc = oracle.curvature(cv, cf)
    Cc = oracle.tri_metric(cv, cf, Gc)
    assert C.max() < 0.05 * Cc.max()


def test_cdf_integer_and_counts():
    wl = synth.clutter(seed=11, target_tris=3000, n_rays=1)
    G = oracle.curvature(wl.verts, wl.tris)
    C = oracle.tri_metric(wl.verts, wl.tris, G)
    cd = oracle.diffraction_cdf(wl.verts, wl.tris, C, wl.tri_obj, dither=1e-3, seed=5, budget=-1)
    off, cdf, mt = cd["mesh_off"], cd["cdf"], cd["mesh_tris"]
    for m in range(cd["n_obj"]):
        tri = mt[off[m]:off[m + 1]]
        assert np.all(np.diff(tri) > 0) and np.all(wl.tri_obj[tri] == m)
        seg = cdf[off[m]:off[m + 1]].astype(np.int64)
        q = np.diff(np.concatenate([[0], seg]))
        assert np.all(q >= 0)
        cmax = C[tri].max()
        if cmax > 0:
            Q = np.floor((C[tri] / cmax).astype(np.float32) * np.float32(2 ** 24)).astype(np.int64)
            assert np.all(q >= Q)                          # dither only adds
            assert np.all(q - Q <= 1e-3 * Q.mean() + 1)    # and stays below delta * mean
        # sample count rule: 64 per distinct welded vertex of high-curvature triangles
        canon = oracle.weld(wl.verts)
        hc = tri[(C[tri] > 0) & (C[tri] >= np.float32(0.25) * cmax)]
        nv = len(np.unique(canon[wl.tris[hc].reshape(-1)])) if len(hc) else 0
        assert cd["n_samples"][m] == (64 * nv if seg[-1] > 0 else 0)
    # budget scaling
    tot = int(cd["n_samples"].sum())
    cd2 = oracle.diffraction_cdf(wl.verts, wl.tris, C, wl.tri_obj, dither=1e-3, seed=5, budget=tot // 3)
    assert np.array_equal(cd2["n_samples"], (cd["n_samples"] * (tot // 3)) // tot)


def test_sampling_distribution_and_points():
    """Samples land on triangles with probability q_i / W (chi-square) and inside them."""
    rng = np.random.default_rng(2)
    T = 40
    v = rng.uniform(0, 1, size=(3 * T, 3)).astype(np.float32)
    f = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    C = rng.uniform(0, 1, T).astype(np.float32)
    C[::7] = 0
    obj = np.zeros(T, np.int32)
    cd = oracle.diffraction_cdf(v, f, C, obj, dither=0.0, seed=1, hc_frac=0.0, samples_per_vertex=2000, budget=-1)
    n = int(cd["n_samples"][0])
    assert n == 2000 * 3 * int((C > 0).sum())
    ct, cp = oracle.diffraction_samples(v, f, cd, seed=9, pose=3)
    q = np.diff(np.concatenate([[0], cd["cdf"].astype(np.int64)]))
    p = q / q.sum()
    cnt = np.bincount(ct, minlength=T)
    assert np.all(cnt[p == 0] == 0)
    nz = p > 0
    chi2 = np.sum((cnt[nz] - n * p[nz]) ** 2 / (n * p[nz]))
    dof = int(nz.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)
    # barycentric coordinates of each point w.r.t. its triangle are in [0, 1]
    A = v[f[ct, 0]].astype(np.float64)
    e1 = v[f[ct, 1]] - A
    e2 = v[f[ct, 2]] - A
    M = np.stack([e1, e2], -1)
    ab = np.linalg.lstsq(M[0], (cp[0] - A[0]), rcond=None)[0]
    sol = np.array([np.linalg.lstsq(M[i], cp[i] - A[i], rcond=None)[0] for i in range(0, len(ct), 97)])
    assert np.all(sol > -1e-4) and np.all(sol.sum(1) < 1 + 1e-4)
    # different pose -> different samples; same pose -> same
    ct2, _ = oracle.diffraction_samples(v, f, cd, seed=9, pose=4)
    ct3, _ = oracle.diffraction_samples(v, f, cd, seed=9, pose=3)
    assert not np.array_equal(ct, ct2) and np.array_equal(ct, ct3)


def test_curvature_rigid_invariance_and_inverse_length_scaling():
    """Mean curvature is a geometric invariant: a rotation and translation leave G unchanged and a uniform
    scale by s divides it by s, on an irregular mesh (a randomly perturbed icosphere, so that no symmetry
    hides a wrong weight).  The scales are powers of two, so the scaled vertices are exact and only the
    operator's own float32 rounding differs; a turn and a shift round the moved vertices, so they are
    compared within a tolerance well above that rounding and far below any wrong weight."""
    rng = np.random.default_rng(5)
    v, f = synth.icosphere(3)
    v = v * (1.0 + 0.15 * rng.uniform(-1, 1, (len(v), 1)))  # bumpy: curvature varies over the mesh
    v = v.astype(np.float32)
    f = f.astype(np.int32)
    G = oracle.curvature(v, f).astype(np.float64)
    assert G.std() > 0.2 * np.abs(G).mean()  # far from constant
    for s in (0.25, 4.0):
        Gs = oracle.curvature((v * np.float32(s)).astype(np.float32), f).astype(np.float64)
        assert np.allclose(Gs * s, G, rtol=1e-5, atol=1e-6 * np.abs(G).max())
    # a turn about a tilted axis and a shift
    a = 0.7
    R = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    R = R @ np.array([[1.0, 0.0, 0.0], [0.0, math.cos(0.4), -math.sin(0.4)], [0.0, math.sin(0.4), math.cos(0.4)]])
    w = (v.astype(np.float64) @ R.T + np.array([3.0, -5.0, 1.5])).astype(np.float32)
    Gw = oracle.curvature(w, f).astype(np.float64)
    assert np.max(np.abs(Gw - G)) <= 1e-3 * np.abs(G).max()


def _obtuse_triangles(v, f):
    p = v.astype(np.float64)[f]
    n = 0
    for k in range(3):
        a = p[:, (k + 1) % 3] - p[:, k]
        b = p[:, (k + 2) % 3] - p[:, k]
        n += int(((a * b).sum(1) < 0).sum())
    return n


def _voronoi_cells(p):
    """Areas of the three Voronoi cells of a non-obtuse planar triangle p [3][2], built from its
    circumcentre: cell of vertex i = polygon (p_i, midpoint to p_j, circumcentre, midpoint to p_k)."""
    (ax, ay), (bx, by), (cx, cy) = p
    d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / d
    uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / d
    out = []
    for i in range(3):
        P0, P1, P2 = p[i], p[(i + 1) % 3], p[(i + 2) % 3]
        poly = [P0, (P0 + P1) / 2, np.array([ux, uy]), (P0 + P2) / 2]
        s = sum(poly[q][0] * poly[(q + 1) % 4][1] - poly[(q + 1) % 4][0] * poly[q][1] for q in range(4))
        out.append(abs(s) / 2)
    return np.array(out)


def test_mixed_area_of_single_triangles():
    """Meyer et al.'s mixed area at each vertex of one triangle, from the geometry alone: a non-obtuse
    triangle gives each vertex its Voronoi cell (circumcentre construction, shoelace areas: 11/16, 11/16
    and 5/8 for (0,0), (2,0), (1,2)); a right angle gives its vertex half the area; an obtuse triangle
    gives half its area to the obtuse vertex and a quarter to each other vertex, wherever the obtuse
    vertex sits in the triangle's order.  A mixed area that takes the Voronoi formula for obtuse
    triangles, or swaps the halves and quarters, fails here."""
    cases = [
        ([[0, 0, 0], [2, 0, 0], [1, 2, 0]], [0.6875, 0.6875, 0.625]),
        ([[0, 0, 0], [1, 0, 0], [0, 1, 0]], [0.25, 0.125, 0.125]),
        ([[0, 0, 0], [4, 0, 0], [2, 1, 0]], [0.5, 0.5, 1.0]),
        ([[2, 1, 0], [0, 0, 0], [4, 0, 0]], [1.0, 0.5, 0.5]),
        ([[0, 0, 0], [2, 1, 0], [4, 0, 0]], [0.5, 1.0, 0.5]),
    ]
    f = np.array([[0, 1, 2]], np.int32)
    for v, want in cases:
        v = np.array(v, np.float32)
        _, A = oracle.curvature(v, f, mixed_area=True)
        assert np.allclose(A, want, rtol=1e-6), (v.tolist(), A, want)
        # the same triangle tilted into 3-D by a turn about (1, 2, 3): the areas do not change
        ax = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = np.eye(3) + math.sin(0.9) * K + (1 - math.cos(0.9)) * K @ K
        _, A3 = oracle.curvature((v.astype(np.float64) @ R.T).astype(np.float32), f, mixed_area=True)
        assert np.allclose(A3, want, rtol=1e-5), (A3, want)
    # random acute triangles against the circumcentre construction
    rng = np.random.default_rng(8)
    n = 0
    while n < 50:
        p = rng.uniform(-1, 1, (3, 2))
        e = [p[(k + 1) % 3] - p[k] for k in range(3)]
        if min(np.dot(e[k], -e[(k + 2) % 3]) for k in range(3)) <= 0.05:
            continue                                    # keep clearly acute triangles only
        n += 1
        v = np.concatenate([p, np.zeros((3, 1))], 1).astype(np.float32)
        _, A = oracle.curvature(v, f, mixed_area=True)
        assert np.allclose(A, _voronoi_cells(v[:, :2].astype(np.float64)), rtol=2e-5)


@pytest.mark.parametrize("mesh", ["bumpy_icosphere", "uv_sphere", "three_sided_cylinder"])
def test_mixed_areas_tile_the_surface(mesh):
    """The mixed areas partition every triangle among its vertices (Voronoi cells of a non-obtuse
    triangle, 1/2 + 1/4 + 1/4 of an obtuse one), so over a closed mesh they add up to its area.  Each
    mesh here has obtuse triangles: a bumpy icosphere (147 of 1,280), a latitude-longitude sphere (about
    half) and a cylinder with three sides (its cap fans are obtuse at the centre).  Swapping the half
    and the quarter gives 5/4 of every obtuse triangle's area."""
    if mesh == "bumpy_icosphere":
        rng = np.random.default_rng(5)
        v, f = synth.icosphere(3)
        v = v * (1.0 + 0.15 * rng.uniform(-1, 1, (len(v), 1)))
    elif mesh == "uv_sphere":
        v, f = synth.uv_sphere(24, 48)
        v = 0.7 * v
    else:
        v, f = synth.cylinder(0.1, 0.4, 3)
    v, f = v.astype(np.float32), f.astype(np.int32)
    assert _obtuse_triangles(v, f) > 0
    _, A = oracle.curvature(v, f, mixed_area=True)
    canon = oracle.weld(v)
    total = A[np.unique(canon)].astype(np.float64).sum()
    p = v.astype(np.float64)[f]
    area = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1).sum()
    assert abs(total - area) <= 1e-5 * area, (total, area)
    assert np.all(A > 0)


@pytest.mark.parametrize("R", [0.4, 3.0])
def test_uv_sphere_curvature(R):
    """Mean curvature 1/R on a latitude-longitude sphere, whose triangles are about half obtuse (so
    the obtuse branches of the mixed area carry most vertices' denominators), within 1 %."""
    v, f = synth.uv_sphere(24, 48)
    v, f = (R * v).astype(np.float32), f.astype(np.int32)
    assert _obtuse_triangles(v, f) > len(f) // 3
    G = oracle.curvature(v, f)
    assert np.allclose(G, 1.0 / R, rtol=0.01), np.abs(G * R - 1).max()
