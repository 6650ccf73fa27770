/*
 * CPU oracle for the acoustic path-tracing hot path (SonoTraceUE, arXiv 2602.19652).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct restatement of
 * what the simulator computes.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the product library never calls it and shares no code with it.
 *
 * Precision.  The paper fixes no precision.  Quantities that decide an integer (which triangle
 * a ray hits, whether a segment is occluded, which triangle a diffraction sample lands on) are
 * computed in float32, in the same precision and operation order as the GPU kernels, so that
 * path sets can be compared bit for bit.  Every product is rounded on its own (the file must be
 * compiled with -ffp-contract=off).  Everything after geometry (path lengths, amplitudes, phases,
 * spectra, gradients) is float64.
 *
 * Sections followed (paper numbering; equations are numbered in order of appearance):
 *   Sec. III-B  geometric pre-processing: Meyer mean-curvature normal, G_v, Eq. 1 (C_i)
 *   Sec. III-C  Algorithm 1 (ray tracing), spreading 1/r^2, atmospheric decay, Eq. 2-4
 *   Sec. III-D  curvature-importance-sampled diffraction candidates, filters, Eq. 7-8
 *   Sec. III-E  direct (passive) path, Eq. 11-12
 * The readings taken where the paper is silent are listed at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_API __attribute__((visibility("default")))

/* ======================================================================================
 * Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), written
 * from its published definition: 10 rounds of two 32x32->64 multiplies with the round
 * constants M0 = 0xD2511F53, M1 = 0xCD9E8D57 and Weyl key increments W0 = 0x9E3779B9,
 * W1 = 0xBB67AE85 applied between rounds.
 * ====================================================================================== */
ORA_API void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint64_t seed, uint32_t out[4]) {
    uint32_t ctr[4] = {a, b, c, d};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    ora_philox4x32_10(ctr, key, out);
}

/* ======================================================================================
 * float32 vector helpers.  Each operation is one IEEE-rounded float op; sums of three
 * terms are taken as (a + b) + c.
 * ====================================================================================== */
static inline float dot3f(const float a[3], const float b[3]) {
    float x = a[0] * b[0];
    float y = a[1] * b[1];
    float z = a[2] * b[2];
    return (x + y) + z;
}
static inline void sub3f(const float a[3], const float b[3], float o[3]) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static inline void cross3f(const float a[3], const float b[3], float o[3]) {
    float x1 = a[1] * b[2], x2 = a[2] * b[1];
    float y1 = a[2] * b[0], y2 = a[0] * b[2];
    float z1 = a[0] * b[1], z2 = a[1] * b[0];
    o[0] = x1 - x2; o[1] = y1 - y2; o[2] = z1 - z2;
}
/* v / |v| with |v| = sqrt((x*x + y*y) + z*z); returns |v|.  A zero vector stays zero. */
static inline float normalize3f(const float v[3], float o[3]) {
    float l = sqrtf(dot3f(v, v));
    if (l > 0.0f) {
        o[0] = v[0] / l; o[1] = v[1] / l; o[2] = v[2] / l;
    } else {
        o[0] = o[1] = o[2] = 0.0f;
    }
    return l;
}
/* Rotate v by unit quaternion q = (w, x, y, z): t = 2 (q_v x v); v' = (v + w t) + q_v x t. */
static inline void rotate_qf(const float q[4], const float v[3], float o[3]) {
    float qv[3] = {q[1], q[2], q[3]};
    float c[3], t[3], c2[3];
    cross3f(qv, v, c);
    t[0] = 2.0f * c[0]; t[1] = 2.0f * c[1]; t[2] = 2.0f * c[2];
    cross3f(qv, t, c2);
    for (int i = 0; i < 3; ++i) {
        float wt = q[0] * t[i];
        float a = v[i] + wt;
        o[i] = a + c2[i];
    }
}

/* Geometric triangle normal n = normalize((v1 - v0) x (v2 - v0)); zero for a degenerate triangle. */
ORA_API void ora_tri_normals(int64_t nt, const float* V, const int32_t* tris, float* N) {
    for (int64_t i = 0; i < nt; ++i) {
        const float* a = V + 3 * (int64_t)tris[3 * i];
        const float* b = V + 3 * (int64_t)tris[3 * i + 1];
        const float* c = V + 3 * (int64_t)tris[3 * i + 2];
        float e1[3], e2[3], cr[3];
        sub3f(b, a, e1);
        sub3f(c, a, e2);
        cross3f(e1, e2, cr);
        normalize3f(cr, N + 3 * i);
    }
}

/* ======================================================================================
 * Sec. III-B: welding, one-ring adjacency, Meyer et al. discrete mean-curvature normal,
 * G_v = |K_v| / 2, and the triangle metric C_i of Eq. 1.
 * ====================================================================================== */
static const float* g_weld_V;
static int cmp_vertex(const void* pa, const void* pb) {
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    for (int k = 0; k < 3; ++k) {
        float fa = g_weld_V[3 * (int64_t)a + k] + 0.0f, fb = g_weld_V[3 * (int64_t)b + k] + 0.0f;
        uint32_t ua, ub;
        memcpy(&ua, &fa, 4);
        memcpy(&ub, &fb, 4);
        if (ua != ub) return ua < ub ? -1 : 1;
    }
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* canon[v] = smallest vertex index with exactly the same position (after mapping -0 to +0). */
ORA_API int ora_weld(int64_t nv, const float* V, int32_t* canon) {
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    if (!idx) return -1;
    for (int64_t i = 0; i < nv; ++i) idx[i] = (int32_t)i;
    g_weld_V = V;
    qsort(idx, (size_t)nv, sizeof(int32_t), cmp_vertex);
    int64_t i = 0;
    while (i < nv) {
        int64_t j = i + 1;
        while (j < nv) {
            int same = 1;
            for (int k = 0; k < 3; ++k) {
                float fa = V[3 * (int64_t)idx[i] + k] + 0.0f, fb = V[3 * (int64_t)idx[j] + k] + 0.0f;
                uint32_t ua, ub;
                memcpy(&ua, &fa, 4);
                memcpy(&ub, &fb, 4);
                if (ua != ub) same = 0;
            }
            if (!same) break;
            ++j;
        }
        for (int64_t k = i; k < j; ++k) canon[idx[k]] = idx[i]; /* sorted by index within group */
        i = j;
    }
    free(idx);
    return 0;
}

/*
 * Meyer, Desbrun, Schroeder, Barr (2003) mean-curvature normal at vertex v:
 *   K_v = 1/(2 A_mixed) * sum over incident triangles (v, a, b) of
 *         cot(angle at b) (x_v - x_a) + cot(angle at a) (x_v - x_b),
 *   A_mixed += Voronoi area (1/8)(|v-b|^2 cot(a) + |v-a|^2 cot(b)) for a non-obtuse triangle,
 *              area/2 if the angle at v is obtuse, area/4 if another angle is obtuse.
 *   cot(angle at a) = dot(v - a, b - a) / |(v - a) x (b - a)|.
 * Incident triangles are visited in ascending triangle index, in float32; triangles whose three
 * welded vertices are not distinct, or whose cross product is zero, are skipped.  Boundary
 * vertices use the same formula over the triangles they have.  G is written per input vertex
 * (every copy of a welded vertex receives the value of its canonical vertex).
 */
ORA_API int ora_curvature_mixed(int64_t nv, const float* V, int64_t nt, const int32_t* tris, float* G,
                                float* A_mixed);
ORA_API int ora_curvature(int64_t nv, const float* V, int64_t nt, const int32_t* tris, float* G) {
    return ora_curvature_mixed(nv, V, nt, tris, G, NULL);
}

/* As ora_curvature; A_mixed (NULL or [nv]) also receives each vertex's mixed area (per input vertex,
 * the canonical vertex's value), the denominator of K_v. */
ORA_API int ora_curvature_mixed(int64_t nv, const float* V, int64_t nt, const int32_t* tris, float* G,
                                float* A_mixed) {
    int32_t* canon = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    int64_t* off = (int64_t*)calloc((size_t)nv + 1, sizeof(int64_t));
    if (!canon || !off) return -1;
    ora_weld(nv, V, canon);
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) off[canon[tris[3 * t + k]] + 1]++;
    for (int64_t v = 0; v < nv; ++v) off[v + 1] += off[v];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    int32_t* adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(3 * nt > 0 ? 3 * nt : 1));
    if (!fill || !adj) return -1;
    for (int64_t v = 0; v < nv; ++v) fill[v] = off[v];
    for (int64_t t = 0; t < nt; ++t) /* ascending t => each list ascending */
        for (int k = 0; k < 3; ++k) {
            int32_t cv = canon[tris[3 * t + k]];
            int dup = 0;
            for (int q = 0; q < k; ++q) if (canon[tris[3 * t + q]] == cv) dup = 1;
            if (!dup) adj[fill[cv]++] = (int32_t)t;
        }
    float* Gc = (float*)calloc((size_t)nv + 1, sizeof(float));
    float* Ac = (float*)calloc((size_t)nv + 1, sizeof(float));
    for (int64_t v = 0; v < nv; ++v) {
        if (canon[v] != v) continue;
        float S[3] = {0.0f, 0.0f, 0.0f};
        float Amix = 0.0f;
        const float* xv = V + 3 * v;
        for (int64_t e = off[v]; e < fill[v]; ++e) {
            int64_t t = adj[e];
            int32_t c0 = canon[tris[3 * t]], c1 = canon[tris[3 * t + 1]], c2 = canon[tris[3 * t + 2]];
            if (c0 == c1 || c1 == c2 || c0 == c2) continue;
            int32_t ia, ib;
            if (c0 == v) { ia = c1; ib = c2; }
            else if (c1 == v) { ia = c2; ib = c0; }
            else { ia = c0; ib = c1; }
            const float* xa = V + 3 * (int64_t)ia;
            const float* xb = V + 3 * (int64_t)ib;
            float va[3], ba[3], vb[3], ab[3], av[3], bv[3], cr[3];
            sub3f(xv, xa, va);  /* v - a */
            sub3f(xb, xa, ba);  /* b - a */
            sub3f(xv, xb, vb);  /* v - b */
            sub3f(xa, xb, ab);  /* a - b */
            sub3f(xa, xv, av);  /* a - v */
            sub3f(xb, xv, bv);  /* b - v */
            cross3f(av, bv, cr);
            float cross_len = sqrtf(dot3f(cr, cr));
            if (!(cross_len > 0.0f)) continue;
            float cot_a = dot3f(va, ba) / cross_len;
            float cot_b = dot3f(vb, ab) / cross_len;
            for (int k = 0; k < 3; ++k) {
                float t1 = cot_b * va[k];
                float t2 = cot_a * vb[k];
                S[k] = S[k] + (t1 + t2);
            }
            float area = 0.5f * cross_len;
            float dv = dot3f(av, bv);
            float da = dot3f(va, ba);
            float db = dot3f(vb, ab);
            float amix;
            if (dv < 0.0f) amix = area / 2.0f;
            else if (da < 0.0f || db < 0.0f) amix = area / 4.0f;
            else {
                float lvb = dot3f(vb, vb), lva = dot3f(va, va);
                float p1 = lvb * cot_a;
                float p2 = lva * cot_b;
                amix = (p1 + p2) / 8.0f;
            }
            Amix = Amix + amix;
        }
        float g = 0.0f;
        if (Amix > 0.0f) {
            float den = 2.0f * Amix;
            float K[3] = {S[0] / den, S[1] / den, S[2] / den};
            g = 0.5f * sqrtf(dot3f(K, K));
        }
        Gc[v] = g;
        Ac[v] = Amix;
    }
    for (int64_t v = 0; v < nv; ++v) G[v] = Gc[canon[v]];
    if (A_mixed)
        for (int64_t v = 0; v < nv; ++v) A_mixed[v] = Ac[canon[v]];
    free(Ac); free(Gc); free(adj); free(fill); free(off); free(canon);
    return 0;
}

/* Eq. 1: C_i = eta * w(A_i) * (max_v G_v - min_v G_v), w(A) = clamp(A / A_ref, 0, 1)
 * (the paper calls w a piecewise-linear area weight without giving it; this is the reading).
 * Triangles with repeated welded vertices or zero area get C_i = 0. */
ORA_API void ora_tri_metric(int64_t nv, const float* V, int64_t nt, const int32_t* tris, const float* G,
                            float eta, float area_ref, float* C) {
    int32_t* canon = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    ora_weld(nv, V, canon);
    for (int64_t t = 0; t < nt; ++t) {
        int32_t i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
        if (canon[i0] == canon[i1] || canon[i1] == canon[i2] || canon[i0] == canon[i2]) { C[t] = 0.0f; continue; }
        float e1[3], e2[3], cr[3];
        sub3f(V + 3 * (int64_t)i1, V + 3 * (int64_t)i0, e1);
        sub3f(V + 3 * (int64_t)i2, V + 3 * (int64_t)i0, e2);
        cross3f(e1, e2, cr);
        float A = 0.5f * sqrtf(dot3f(cr, cr));
        if (!(A > 0.0f)) { C[t] = 0.0f; continue; }
        float w = A / area_ref;
        if (w > 1.0f) w = 1.0f;
        if (w < 0.0f) w = 0.0f;
        float g0 = G[i0], g1 = G[i1], g2 = G[i2];
        float gmax = fmaxf(fmaxf(g0, g1), g2), gmin = fminf(fminf(g0, g1), g2);
        float ew = eta * w;
        C[t] = ew * (gmax - gmin);
    }
    free(canon);
}

/* ======================================================================================
 * Sec. III-D: per-mesh dithered importance CDF, sample counts, samples.
 *
 * Readings (the paper gives the idea, not the constants):
 *  - weights in integer form: Q_i = floor(C_i / Cmax_mesh * 2^24) (float32), dither
 *    d_i = floor((delta * mean_mesh(Q)) * xi_i) with xi_i = (Philox(tri,0,0,1).x0 >> 8) * 2^-24,
 *    q_i = Q_i + d_i; the CDF is the exact uint64 inclusive prefix of q over the mesh's
 *    triangles in ascending triangle index (sorting by C_i only relabels, so it is omitted);
 *  - per mesh, n = samples_per_vertex * (#distinct welded vertices of triangles with
 *    C_i >= hc_frac * Cmax_mesh and C_i > 0), scaled down to a global budget by
 *    n_m <- n_m * budget / total (integer division) when the total exceeds it;
 *  - sample s of mesh m: x = Philox(s, m, pose, 0); target = high 64 bits of
 *    ((x0 << 32 | x1) * W_m); triangle = first CDF entry > target; barycentric
 *    a = (x2 >> 8) 2^-24, b = (x3 >> 8) 2^-24, reflected to a' = 1-a, b' = 1-b when a + b > 1;
 *    point = (v0 + a (v1 - v0)) + b (v2 - v0) in float32.
 * ====================================================================================== */
ORA_API int ora_diffraction_cdf(int64_t nv, const float* V, int64_t nt, const int32_t* tris, const float* C,
                                const int32_t* tri_obj, int32_t n_obj, double dither, uint64_t seed,
                                float hc_frac, int32_t samples_per_vertex, int64_t budget,
                                int32_t* mesh_tris /*[nt]*/, int64_t* mesh_off /*[n_obj+1]*/,
                                uint64_t* cdf /*[nt], in mesh_tris order*/, int64_t* n_samples /*[n_obj]*/) {
    /* group triangles by mesh, ascending triangle index within a mesh */
    memset(mesh_off, 0, sizeof(int64_t) * (size_t)(n_obj + 1));
    for (int64_t t = 0; t < nt; ++t) mesh_off[tri_obj[t] + 1]++;
    for (int32_t m = 0; m < n_obj; ++m) mesh_off[m + 1] += mesh_off[m];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_obj + 1));
    for (int32_t m = 0; m <= n_obj; ++m) fill[m] = mesh_off[m];
    for (int64_t t = 0; t < nt; ++t) mesh_tris[fill[tri_obj[t]]++] = (int32_t)t;
    free(fill);
    float* cmax = (float*)calloc((size_t)n_obj + 1, sizeof(float));
    for (int64_t t = 0; t < nt; ++t) if (C[t] > cmax[tri_obj[t]]) cmax[tri_obj[t]] = C[t];
    for (int32_t m = 0; m < n_obj; ++m) {
        uint64_t sumQ = 0;
        int64_t n = mesh_off[m + 1] - mesh_off[m];
        uint64_t* Q = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) {
            int32_t t = mesh_tris[mesh_off[m] + i];
            uint64_t q = 0;
            if (cmax[m] > 0.0f) {
                float r = C[t] / cmax[m];
                float s = r * 16777216.0f;
                q = (uint64_t)floorf(s);
            }
            Q[i] = q;
            sumQ += q;
        }
        double mean = n > 0 ? (double)sumQ / (double)n : 0.0;
        double scale = dither * mean;
        uint64_t acc = 0;
        for (int64_t i = 0; i < n; ++i) {
            int32_t t = mesh_tris[mesh_off[m] + i];
            uint32_t x[4];
            philox((uint32_t)t, 0u, 0u, 1u, seed, x);
            double xi = (double)(x[0] >> 8) * (1.0 / 16777216.0);
            uint64_t d = (uint64_t)floor(scale * xi);
            acc += Q[i] + d;
            cdf[mesh_off[m] + i] = acc;
        }
        free(Q);
    }
    /* high-curvature vertex counts */
    int32_t* canon = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    ora_weld(nv, V, canon);
    /* mark (canonical vertex, mesh) pairs: per mesh a boolean array would be O(n_obj * nv);
     * instead collect pairs, sort, count distinct. */
    int64_t np = 0;
    uint64_t* pairs = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(3 * nt > 0 ? 3 * nt : 1));
    for (int64_t t = 0; t < nt; ++t) {
        int32_t m = tri_obj[t];
        float thr = hc_frac * cmax[m];
        if (C[t] > 0.0f && C[t] >= thr)
            for (int k = 0; k < 3; ++k)
                pairs[np++] = ((uint64_t)(uint32_t)m << 32) | (uint32_t)canon[tris[3 * t + k]];
    }
    int cmpu64(const void* a, const void* b);
    qsort(pairs, (size_t)np, sizeof(uint64_t), cmpu64);
    for (int32_t m = 0; m < n_obj; ++m) n_samples[m] = 0;
    for (int64_t i = 0; i < np; ++i)
        if (i == 0 || pairs[i] != pairs[i - 1]) n_samples[pairs[i] >> 32] += samples_per_vertex;
    int64_t total = 0;
    for (int32_t m = 0; m < n_obj; ++m) {
        int64_t n = mesh_off[m + 1] - mesh_off[m];
        if (n == 0 || cdf[mesh_off[m + 1] - 1] == 0) n_samples[m] = 0;
        total += n_samples[m];
    }
    if (budget >= 0 && total > budget) {
        for (int32_t m = 0; m < n_obj; ++m)
            n_samples[m] = (int64_t)(((unsigned __int128)(uint64_t)n_samples[m] * (uint64_t)budget) / (uint64_t)total);
    }
    free(pairs); free(canon); free(cmax);
    return 0;
}

int cmpu64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

ORA_API int64_t ora_diffraction_samples(const float* V, const int32_t* tris, int32_t n_obj,
                                        const int32_t* mesh_tris, const int64_t* mesh_off, const uint64_t* cdf,
                                        const int64_t* n_samples, uint64_t seed, uint32_t pose,
                                        int32_t* cand_tri, float* cand_p /*[K][3]*/) {
    int64_t g = 0;
    for (int32_t m = 0; m < n_obj; ++m) {
        int64_t lo = mesh_off[m], hi = mesh_off[m + 1];
        if (hi <= lo) continue;
        uint64_t W = cdf[hi - 1];
        for (int64_t s = 0; s < n_samples[m]; ++s, ++g) {
            uint32_t x[4];
            philox((uint32_t)s, (uint32_t)m, pose, 0u, seed, x);
            uint64_t u = ((uint64_t)x[0] << 32) | x[1];
            uint64_t target = (uint64_t)(((unsigned __int128)u * W) >> 64);
            int64_t a = lo, b = hi - 1; /* first index with cdf > target */
            while (a < b) {
                int64_t mid = a + (b - a) / 2;
                if (cdf[mid] > target) b = mid; else a = mid + 1;
            }
            int32_t t = mesh_tris[a];
            float ba = (float)(x[2] >> 8) * (1.0f / 16777216.0f);
            float bb = (float)(x[3] >> 8) * (1.0f / 16777216.0f);
            float sum = ba + bb;
            if (sum > 1.0f) { ba = 1.0f - ba; bb = 1.0f - bb; }
            const float* v0 = V + 3 * (int64_t)tris[3 * t];
            const float* v1 = V + 3 * (int64_t)tris[3 * t + 1];
            const float* v2 = V + 3 * (int64_t)tris[3 * t + 2];
            for (int k = 0; k < 3; ++k) {
                float e1 = v1[k] - v0[k];
                float e2 = v2[k] - v0[k];
                float p1 = ba * e1;
                float p2 = bb * e2;
                float q = v0[k] + p1;
                cand_p[3 * g + k] = q + p2;
            }
            cand_tri[g] = t;
        }
    }
    return g;
}

/* ======================================================================================
 * Ray-triangle intersection: the watertight test of Woop, Benthin and Wald (JCGT 2013),
 * two-sided, float32 only (no double fallback), t = T / det.  Closest hit = the
 * lexicographically smallest (t, triangle index) with t > t_min, skipping one excluded
 * triangle (the surface the ray leaves).
 * ====================================================================================== */
typedef struct {
    float o[3];
    int kx, ky, kz;
    float Sx, Sy, Sz;
} WTRay;

static void wt_setup(const float o[3], const float d[3], WTRay* r) {
    r->o[0] = o[0]; r->o[1] = o[1]; r->o[2] = o[2];
    float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
    int kz = (ax >= ay) ? ((ax >= az) ? 0 : 2) : ((ay >= az) ? 1 : 2);
    int kx = kz + 1; if (kx == 3) kx = 0;
    int ky = kx + 1; if (ky == 3) ky = 0;
    if (d[kz] < 0.0f) { int tmp = kx; kx = ky; ky = tmp; }
    r->kx = kx; r->ky = ky; r->kz = kz;
    r->Sx = d[kx] / d[kz];
    r->Sy = d[ky] / d[kz];
    r->Sz = 1.0f / d[kz];
}

/* returns 1 and *t on hit */
static int wt_intersect(const WTRay* r, const float v0[3], const float v1[3], const float v2[3], float* t) {
    float A[3], B[3], Cc[3];
    sub3f(v0, r->o, A);
    sub3f(v1, r->o, B);
    sub3f(v2, r->o, Cc);
    const int kx = r->kx, ky = r->ky, kz = r->kz;
    float Ax = A[kx] - r->Sx * A[kz];
    float Ay = A[ky] - r->Sy * A[kz];
    float Bx = B[kx] - r->Sx * B[kz];
    float By = B[ky] - r->Sy * B[kz];
    float Cx = Cc[kx] - r->Sx * Cc[kz];
    float Cy = Cc[ky] - r->Sy * Cc[kz];
    float U = Cx * By - Cy * Bx;
    float Vv = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if ((U < 0.0f || Vv < 0.0f || W < 0.0f) && (U > 0.0f || Vv > 0.0f || W > 0.0f)) return 0;
    float det = (U + Vv) + W;
    if (det == 0.0f) return 0;
    float Az = r->Sz * A[kz];
    float Bz = r->Sz * B[kz];
    float Cz = r->Sz * Cc[kz];
    float T = (U * Az + Vv * Bz) + W * Cz;
    *t = T / det;
    return 1;
}

/* ---------------------------------------------------------------- scene + median-split BVH */
typedef struct {
    double lo[3], hi[3];
    int32_t left, right; /* internal: child indices; leaf: left = -1, right unused */
    int32_t first, count;
} OraNode;

typedef struct {
    int64_t nt;
    const float* V;
    const int32_t* tris;
    OraNode* nodes;
    int32_t* order;   /* triangle indices in leaf order */
    int64_t n_nodes;
    double pad;
} OraScene;

static const float* g_cent;
static int g_axis;
static int cmp_cent(const void* pa, const void* pb) {
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    float ca = g_cent[3 * (int64_t)a + g_axis], cb = g_cent[3 * (int64_t)b + g_axis];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static int32_t bvh_build_rec(OraScene* S, const float* cent, int32_t first, int32_t count) {
    int32_t id = (int32_t)S->n_nodes++;
    OraNode* n = &S->nodes[id];
    for (int k = 0; k < 3; ++k) { n->lo[k] = INFINITY; n->hi[k] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t i = first; i < first + count; ++i) {
        int32_t t = S->order[i];
        for (int j = 0; j < 3; ++j) {
            const float* v = S->V + 3 * (int64_t)S->tris[3 * (int64_t)t + j];
            for (int k = 0; k < 3; ++k) {
                if (v[k] < n->lo[k]) n->lo[k] = v[k];
                if (v[k] > n->hi[k]) n->hi[k] = v[k];
            }
        }
        for (int k = 0; k < 3; ++k) {
            double c = cent[3 * (int64_t)t + k];
            if (c < clo[k]) clo[k] = c;
            if (c > chi[k]) chi[k] = c;
        }
    }
    for (int k = 0; k < 3; ++k) { n->lo[k] -= S->pad; n->hi[k] += S->pad; }
    if (count <= 4) {
        n->left = -1; n->right = -1; n->first = first; n->count = count;
        return id;
    }
    int axis = 0;
    double ext = chi[0] - clo[0];
    for (int k = 1; k < 3; ++k) if (chi[k] - clo[k] > ext) { ext = chi[k] - clo[k]; axis = k; }
    g_cent = cent; g_axis = axis;
    qsort(S->order + first, (size_t)count, sizeof(int32_t), cmp_cent);
    int32_t half = count / 2;
    int32_t l = bvh_build_rec(S, cent, first, half);
    int32_t r = bvh_build_rec(S, cent, first + half, count - half);
    n = &S->nodes[id];
    n->left = l; n->right = r; n->first = first; n->count = count;
    return id;
}

/* use_bvh = 0: every query tests every triangle (brute force). */
ORA_API void* ora_scene_new(int64_t nt, const float* V, int64_t nv, const int32_t* tris, int use_bvh) {
    OraScene* S = (OraScene*)calloc(1, sizeof(OraScene));
    S->nt = nt; S->V = V; S->tris = tris;
    if (use_bvh && nt > 0) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = 0; i < nv; ++i)
            for (int k = 0; k < 3; ++k) {
                if (V[3 * i + k] < lo[k]) lo[k] = V[3 * i + k];
                if (V[3 * i + k] > hi[k]) hi[k] = V[3 * i + k];
            }
        double diag = 0.0;
        for (int k = 0; k < 3; ++k) diag += (hi[k] - lo[k]) * (hi[k] - lo[k]);
        S->pad = 1e-5 * sqrt(diag) + 1e-6;
        float* cent = (float*)malloc(sizeof(float) * 3 * (size_t)nt);
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += V[3 * (int64_t)tris[3 * t + j] + k];
                cent[3 * t + k] = (float)(s / 3.0);
            }
        S->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)nt);
        for (int64_t t = 0; t < nt; ++t) S->order[t] = (int32_t)t;
        S->nodes = (OraNode*)malloc(sizeof(OraNode) * (size_t)(2 * nt));
        S->n_nodes = 0;
        bvh_build_rec(S, cent, 0, (int32_t)nt);
        free(cent);
    }
    return S;
}

ORA_API void ora_scene_free(void* p) {
    OraScene* S = (OraScene*)p;
    if (!S) return;
    free(S->nodes); free(S->order); free(S);
}

/* slab test in double against a padded box; conservative for the float32 triangle test */
static int box_hit(const OraNode* n, const float o[3], const double inv[3], double tlo, double thi) {
    double t0 = tlo, t1 = thi;
    for (int k = 0; k < 3; ++k) {
        double a = (n->lo[k] - (double)o[k]) * inv[k];
        double b = (n->hi[k] - (double)o[k]) * inv[k];
        if (isnan(a) || isnan(b)) { /* direction component zero and origin on the slab plane */
            if ((double)o[k] < n->lo[k] || (double)o[k] > n->hi[k]) return 0;
            continue;
        }
        if (a > b) { double tmp = a; a = b; b = tmp; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    return 1;
}

static const float* tv(const OraScene* S, int32_t t, int j) {
    return S->V + 3 * (int64_t)S->tris[3 * (int64_t)t + j];
}

/* closest hit; returns triangle index or -1 */
static int32_t closest_hit(const OraScene* S, const float o[3], const float d[3], int32_t exclude, float t_min,
                           float* t_out) {
    WTRay r;
    wt_setup(o, d, &r);
    int32_t best = -1;
    float tb = INFINITY;
    if (!S->nodes) {
        for (int64_t t = 0; t < S->nt; ++t) {
            if (t == exclude) continue;
            float th;
            if (!wt_intersect(&r, tv(S, (int32_t)t, 0), tv(S, (int32_t)t, 1), tv(S, (int32_t)t, 2), &th)) continue;
            if (!(th > t_min)) continue;
            if (th < tb || (th == tb && t < best)) { tb = th; best = (int32_t)t; }
        }
    } else {
        double inv[3] = {1.0 / (double)d[0], 1.0 / (double)d[1], 1.0 / (double)d[2]};
        int32_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const OraNode* n = &S->nodes[stack[--sp]];
            double thi = (best >= 0) ? (double)tb * (1.0 + 1e-6) + S->pad : INFINITY;
            if (!box_hit(n, o, inv, -S->pad, thi)) continue;
            if (n->left < 0) {
                for (int32_t i = n->first; i < n->first + n->count; ++i) {
                    int32_t t = S->order[i];
                    if (t == exclude) continue;
                    float th;
                    if (!wt_intersect(&r, tv(S, t, 0), tv(S, t, 1), tv(S, t, 2), &th)) continue;
                    if (!(th > t_min)) continue;
                    if (th < tb || (th == tb && t < best)) { tb = th; best = t; }
                }
            } else {
                stack[sp++] = n->left;
                stack[sp++] = n->right;
            }
        }
    }
    *t_out = tb;
    return best;
}

/* any hit with t_min < t < t_max (strict), skipping one excluded triangle */
static int any_hit(const OraScene* S, const float o[3], const float d[3], int32_t exclude, float t_min, float t_max) {
    WTRay r;
    wt_setup(o, d, &r);
    if (!S->nodes) {
        for (int64_t t = 0; t < S->nt; ++t) {
            if (t == exclude) continue;
            float th;
            if (!wt_intersect(&r, tv(S, (int32_t)t, 0), tv(S, (int32_t)t, 1), tv(S, (int32_t)t, 2), &th)) continue;
            if (th > t_min && th < t_max) return 1;
        }
        return 0;
    }
    double inv[3] = {1.0 / (double)d[0], 1.0 / (double)d[1], 1.0 / (double)d[2]};
    int32_t stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const OraNode* n = &S->nodes[stack[--sp]];
        if (!box_hit(n, o, inv, -S->pad, (double)t_max * (1.0 + 1e-6) + S->pad)) continue;
        if (n->left < 0) {
            for (int32_t i = n->first; i < n->first + n->count; ++i) {
                int32_t t = S->order[i];
                if (t == exclude) continue;
                float th;
                if (!wt_intersect(&r, tv(S, t, 0), tv(S, t, 1), tv(S, t, 2), &th)) continue;
                if (th > t_min && th < t_max) return 1;
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
    return 0;
}

/* Visibility of `target` from `o`: the segment is tested with direction u = (target - o)/|target - o|
 * and t in (t_min, |target - o| - eps).  Returns 1 when visible. */
static int visible(const OraScene* S, const float o[3], const float target[3], int32_t exclude, float t_min, float eps) {
    float v[3], u[3];
    sub3f(target, o, v);
    float L = normalize3f(v, u);
    float tmax = L - eps;
    if (!(tmax > t_min)) return 1;
    return !any_hit(S, o, u, exclude, t_min, tmax);
}

ORA_API int32_t ora_closest_hit(void* scene, const float o[3], const float d[3], int32_t exclude, float t_min, float* t) {
    return closest_hit((const OraScene*)scene, o, d, exclude, t_min, t);
}

ORA_API int ora_visible(void* scene, const float o[3], const float target[3], int32_t exclude, float t_min, float eps) {
    return visible((const OraScene*)scene, o, target, exclude, t_min, eps);
}

/* Receiver reference point for the per-hit visibility ray: the centroid of the microphones,
 * summed in float64 in microphone order, divided by M, rounded to float32. */
ORA_API void ora_mic_centroid(int32_t M, const float* mics, float R[3]) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int32_t m = 0; m < M; ++m)
        for (int k = 0; k < 3; ++k) acc[k] += (double)mics[3 * m + k];
    for (int k = 0; k < 3; ++k) R[k] = (float)(acc[k] / (double)M);
}

/*
 * Algorithm 1 (Sec. III-C), one emitter.  Per ray i: origin = emitter, direction = q applied to
 * the ray's local direction; for bounce j = 0..B-1: closest hit (skipping the triangle just left,
 * t > t_min); no hit ends the ray; P = o + t d (float32); d' = normalize(d - 2 (d.n) n) about the
 * triangle's geometric normal; r_j = r_{j-1} + t in float64 (t is used for every segment, also the
 * first, whose length equals the source-to-hit distance); visibility of the receiver reference point
 * R from P (skipping the hit triangle); the record (triangle, P, d', r_j, visible) is stored at [i][j];
 * the ray continues from P along d' and ends after the record when r_j >= r_max.
 * Records never written keep tri = -1.
 */
ORA_API int ora_trace(void* scene, const float* nrm, const float s[3], const float q[4], int64_t N,
                      const float* dirs, int32_t B, double r_max, float t_min, float los_eps, const float R[3],
                      int32_t* rec_tri, float* rec_p, float* rec_d, double* rec_r, uint8_t* rec_los,
                      int32_t nthreads) {
    const OraScene* S = (const OraScene*)scene;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < N; ++i) {
        for (int32_t j = 0; j < B; ++j) {
            rec_tri[i * B + j] = -1;
            rec_los[i * B + j] = 0;
            rec_r[i * B + j] = 0.0;
            for (int k = 0; k < 3; ++k) rec_p[(i * B + j) * 3 + k] = rec_d[(i * B + j) * 3 + k] = 0.0f;
        }
        float o[3] = {s[0], s[1], s[2]};
        float d[3];
        rotate_qf(q, dirs + 3 * i, d);
        double r = 0.0;
        int32_t prev = -1;
        for (int32_t j = 0; j < B; ++j) {
            float t;
            int32_t tri = closest_hit(S, o, d, prev, t_min, &t);
            if (tri < 0) break;
            float P[3];
            for (int k = 0; k < 3; ++k) {
                float td = t * d[k];
                P[k] = o[k] + td;
            }
            const float* n = nrm + 3 * (int64_t)tri;
            float dn = dot3f(d, n);
            float k2 = 2.0f * dn;
            float rv[3], dr[3];
            for (int k = 0; k < 3; ++k) {
                float kn = k2 * n[k];
                rv[k] = d[k] - kn;
            }
            normalize3f(rv, dr);
            r = r + (double)t;
            int vis = visible(S, P, R, tri, t_min, los_eps);
            int64_t id = i * B + j;
            rec_tri[id] = tri;
            rec_los[id] = (uint8_t)vis;
            rec_r[id] = r;
            for (int k = 0; k < 3; ++k) { rec_p[3 * id + k] = P[k]; rec_d[3 * id + k] = dr[k]; }
            o[0] = P[0]; o[1] = P[1]; o[2] = P[2];
            d[0] = dr[0]; d[1] = dr[1]; d[2] = dr[2];
            prev = tri;
            if (r >= r_max) break;
        }
    }
    return 0;
}

/*
 * Receiver test per microphone.  Algorithm 1 leaves the receiver test unstated; the default test casts one
 * visibility ray per hit towards the receiver reference point (the microphones' centroid), this variant
 * one ray per microphone: bit m of rec_mask[id] is set when microphone m is visible from
 * the record's hit point (the hit triangle excluded, stopping los_eps short), and rec_los[id] becomes 1
 * when any bit is.  Records without a hit (tri < 0) get 0.  M <= 64.
 */
ORA_API int ora_los_per_mic(void* scene, int64_t NB, const int32_t* rec_tri, const float* rec_p, int32_t M,
                            const float* mics, float t_min, float los_eps, uint64_t* rec_mask, uint8_t* rec_los,
                            int32_t nthreads) {
    const OraScene* S = (const OraScene*)scene;
    if (M < 1 || M > 64) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t id = 0; id < NB; ++id) {
        uint64_t mask = 0;
        if (rec_tri[id] >= 0) {
            for (int32_t m = 0; m < M; ++m)
                if (visible(S, rec_p + 3 * id, mics + 3 * m, rec_tri[id], t_min, los_eps)) mask |= (uint64_t)1 << m;
        }
        rec_mask[id] = mask;
        rec_los[id] = mask != 0;
    }
    return 0;
}

/*
 * Sec. III-D filters for each candidate point o on triangle T:
 *   field of view: the angle between the emitter forward axis (q applied to +x) and
 *     normalize(o - s) is at most fov_half: dot >= cos_fov (skipped when cos_fov <= -1);
 *   incidence: |n_T . normalize(s - o)| >= cos_inc;
 *   visibility of the emitter from o (skipping T).
 * The paper applies the field of view per mesh; here it is applied per candidate point.
 */
ORA_API void ora_diffraction_filter(void* scene, const float* nrm, const float s[3], const float q[4], int64_t K,
                                    const int32_t* cand_tri, const float* cand_p, float cos_fov, float cos_inc,
                                    float t_min, float los_eps, uint8_t* keep, int32_t nthreads) {
    const OraScene* S = (const OraScene*)scene;
    float ex[3] = {1.0f, 0.0f, 0.0f}, fwd[3];
    rotate_qf(q, ex, fwd);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t i = 0; i < K; ++i) {
        const float* o = cand_p + 3 * i;
        int32_t t = cand_tri[i];
        int ok = 1;
        if (cos_fov > -1.0f) {
            float w[3], wn[3];
            sub3f(o, s, w);
            normalize3f(w, wn);
            if (!(dot3f(fwd, wn) >= cos_fov)) ok = 0;
        }
        if (ok) {
            float v[3], vn[3];
            sub3f(s, o, v);
            normalize3f(v, vn);
            float ci = fabsf(dot3f(nrm + 3 * (int64_t)t, vn));
            if (!(ci >= cos_inc)) ok = 0;
        }
        if (ok) ok = visible(S, o, s, t, t_min, los_eps);
        keep[i] = (uint8_t)ok;
    }
}

/* Sec. III-E: visibility of every microphone from the emitter. */
ORA_API void ora_direct_visibility(void* scene, const float s[3], int32_t M, const float* mics, float t_min,
                                   float los_eps, uint8_t* vis) {
    for (int32_t m = 0; m < M; ++m) vis[m] = (uint8_t)visible((const OraScene*)scene, s, mics + 3 * m, -1, t_min, los_eps);
}

/* ======================================================================================
 * Spectra, float64.  For every path, microphone m and bin f_k (uniform grid, f_k = f_lo +
 * k (f_hi - f_lo)/(F - 1)):
 *   S[m][k] += A e^{+j 2 pi f_k r / c}                                  (Eq. 4, 8, 12)
 *   A = (1/r^2) 10^{-alpha(f_k) r / 20} D_e D_m X                        (Eq. 3, 7, 11)
 *   alpha(f) = a0 + a1 f[kHz] in dB/m (amplitude decay; the paper's L_atm = 10^{r alpha})
 *   specular X = exp(-gamma^2 g(T_j, f)) prod_{q<=j} k(T_q, f)          (Eq. 2, cumulative reading)
 *            or exp(-gamma^2 g(T_j, f)) k(T_j, f)                        (reflection_mode 1, literal Eq. 2)
 *     gamma = angle between d' and the direction from P to m, g = 1/(2 beta^2)
 *     (Eq. 2 prints exp(+gamma^2/2beta^2); the decaying Gaussian lobe is the reading), r = r_j + |m - P|
 *   diffraction X = I_d(T, f), r = |s - o| + |o - m|                      (Eq. 7)
 *   direct X = I_p, r = |m - s|, only if m is visible from s             (Eq. 11)
 * Material curves k, g, I_d are linear in f between band centres and constant beyond the end
 * bands (g is interpolated as g = 1/(2 beta^2), i.e. on the lobe exponent).
 * D_e: emitter table [n_theta][F] over theta = angle(forward, departure direction) in [0, pi],
 * linear in theta.  D_m: per-microphone table [n_el][n_az][n_bands] in the microphone frame,
 * bilinear in (az, el) of the arrival direction (from m towards the last point), linear in band.
 * ====================================================================================== */
typedef struct {
    int32_t F;
    double f_lo, f_hi, c, a0, a1_per_khz;
    int32_t n_mat, n_bands;
    const float* band_hz;
    const float* k_band;
    const float* beta_band;
    const float* diff_band;
    int32_t M;
    const float* mics;
    const float* mic_quats;   /* [M][4] or NULL */
    const float* mic_tables;  /* [M][n_el][n_az][n_bands] or NULL */
    int32_t n_az, n_el;
    const float* s;
    const float* q;
    const float* emit_table;  /* [n_theta][F] or NULL */
    int32_t n_theta;
    int32_t reflection_mode;
    double direct_gain;
} OraSpecParams;

static double freq_of(const OraSpecParams* P, int k) {
    if (P->F == 1) return P->f_lo;
    return P->f_lo + (double)k * (P->f_hi - P->f_lo) / (double)(P->F - 1);
}

static void band_weights(const OraSpecParams* P, double f, int* b0, double* w) {
    int nb = P->n_bands;
    if (nb == 1) { *b0 = 0; *w = 0.0; return; }
    if (f <= (double)P->band_hz[0]) { *b0 = 0; *w = 0.0; return; }
    if (f >= (double)P->band_hz[nb - 1]) { *b0 = nb - 2; *w = 1.0; return; }
    int b = 0;
    while (b + 1 < nb && (double)P->band_hz[b + 1] <= f) ++b;
    if (b >= nb - 1) b = nb - 2;
    *b0 = b;
    *w = (f - (double)P->band_hz[b]) / ((double)P->band_hz[b + 1] - (double)P->band_hz[b]);
}

static double band_interp(const OraSpecParams* P, const float* row, int b0, double w) {
    if (P->n_bands == 1) return (double)row[0];
    return (1.0 - w) * (double)row[b0] + w * (double)row[b0 + 1];
}

static double g_interp(const OraSpecParams* P, int mat, int b0, double w) {
    const float* row = P->beta_band + (int64_t)mat * P->n_bands;
    double g0 = 1.0 / (2.0 * (double)row[b0] * (double)row[b0]);
    if (P->n_bands == 1) return g0;
    double g1 = 1.0 / (2.0 * (double)row[b0 + 1] * (double)row[b0 + 1]);
    return (1.0 - w) * g0 + w * g1;
}

static void rotate_qd(const float qf[4], const double v[3], double o[3]) {
    double q[4] = {qf[0], qf[1], qf[2], qf[3]};
    double t[3] = {2.0 * (q[2] * v[2] - q[3] * v[1]), 2.0 * (q[3] * v[0] - q[1] * v[2]), 2.0 * (q[1] * v[1] - q[2] * v[0])};
    double c[3] = {q[2] * t[2] - q[3] * t[1], q[3] * t[0] - q[1] * t[2], q[1] * t[1] - q[2] * t[0]};
    for (int k = 0; k < 3; ++k) o[k] = v[k] + q[0] * t[k] + c[k];
}

static double emit_dir(const OraSpecParams* P, const double dir[3], int k) {
    if (!P->emit_table) return 1.0;
    double ex[3] = {1.0, 0.0, 0.0}, fwd[3];
    rotate_qd(P->q, ex, fwd);
    double c = fwd[0] * dir[0] + fwd[1] * dir[1] + fwd[2] * dir[2];
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c);
    double x = th / (M_PI / (double)(P->n_theta - 1));
    int i = (int)floor(x);
    if (i > P->n_theta - 2) i = P->n_theta - 2;
    if (i < 0) i = 0;
    double w = x - (double)i;
    return (1.0 - w) * (double)P->emit_table[(int64_t)i * P->F + k] + w * (double)P->emit_table[(int64_t)(i + 1) * P->F + k];
}

/* band values of the receiver directivity for arrival direction `a` (unit, world frame) */
static void mic_dir_bands(const OraSpecParams* P, int m, const double a[3], double* out) {
    const float* qq = P->mic_quats ? P->mic_quats + 4 * m : NULL;
    double l[3] = {a[0], a[1], a[2]};
    if (qq) { /* world -> local: rotate by the conjugate quaternion */
        float qc[4] = {qq[0], -qq[1], -qq[2], -qq[3]};
        rotate_qd(qc, a, l);
    }
    double az = atan2(l[1], l[0]);
    double zc = l[2]; if (zc > 1.0) zc = 1.0; if (zc < -1.0) zc = -1.0;
    double el = asin(zc);
    double x = (az + M_PI) / (2.0 * M_PI) * (double)P->n_az;
    double fx = floor(x);
    double wa = x - fx;
    int i0 = ((int)fx % P->n_az + P->n_az) % P->n_az;
    int i1 = (i0 + 1) % P->n_az;
    double y = (el + M_PI / 2.0) / M_PI * (double)(P->n_el - 1);
    int j0 = (int)floor(y);
    if (j0 > P->n_el - 2) j0 = P->n_el - 2;
    if (j0 < 0) j0 = 0;
    double wb = y - (double)j0;
    const float* T = P->mic_tables + (int64_t)m * P->n_el * P->n_az * P->n_bands;
    for (int b = 0; b < P->n_bands; ++b) {
        double v00 = T[((int64_t)j0 * P->n_az + i0) * P->n_bands + b];
        double v01 = T[((int64_t)j0 * P->n_az + i1) * P->n_bands + b];
        double v10 = T[((int64_t)(j0 + 1) * P->n_az + i0) * P->n_bands + b];
        double v11 = T[((int64_t)(j0 + 1) * P->n_az + i1) * P->n_bands + b];
        out[b] = (1.0 - wb) * ((1.0 - wa) * v00 + wa * v01) + wb * ((1.0 - wa) * v10 + wa * v11);
    }
}

static double mic_dir(const OraSpecParams* P, const double* bands, int b0, double w) {
    if (!P->mic_tables) return 1.0;
    if (P->n_bands == 1) return bands[0];
    return (1.0 - w) * bands[b0] + w * bands[b0 + 1];
}

/* one path's contribution to one microphone over all (selected) bins, accumulated into out */
typedef struct {
    int kind;            /* 0 specular, 1 diffraction, 2 direct */
    double P[3];         /* start of the last leg */
    double dref[3];      /* specular: reflected direction */
    double r_pre;        /* path length before the last leg */
    int chain_len;
    int chain[16];       /* materials along the path (specular) / of the diffraction triangle */
    double dep[3];       /* departure direction at the emitter (unit) */
} Path;

static void add_path(const OraSpecParams* P, const Path* p, int m, int nk, const int32_t* ks, double* outm /*[F][2]*/) {
    const float* mf = P->mics + 3 * m;
    double v[3] = {(double)mf[0] - p->P[0], (double)mf[1] - p->P[1], (double)mf[2] - p->P[2]};
    double dist = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double r = p->r_pre + dist;
    double u[3] = {v[0] / dist, v[1] / dist, v[2] / dist};
    double gamma2 = 0.0;
    if (p->kind == 0) {
        double cx[3] = {p->dref[1] * u[2] - p->dref[2] * u[1], p->dref[2] * u[0] - p->dref[0] * u[2],
                        p->dref[0] * u[1] - p->dref[1] * u[0]};
        double sg = sqrt(cx[0] * cx[0] + cx[1] * cx[1] + cx[2] * cx[2]);
        double cg = p->dref[0] * u[0] + p->dref[1] * u[1] + p->dref[2] * u[2];
        double gm = atan2(sg, cg);
        gamma2 = gm * gm;
    }
    double mb[64];
    if (P->mic_tables) {
        double a[3] = {-u[0], -u[1], -u[2]};
        mic_dir_bands(P, m, a, mb);
    }
    for (int kk = 0; kk < nk; ++kk) {
        int k = ks ? ks[kk] : kk;
        double f = freq_of(P, k);
        int b0; double w;
        band_weights(P, f, &b0, &w);
        double X;
        if (p->kind == 0) {
            int mj = p->chain[p->chain_len - 1];
            double lobe = exp(-gamma2 * g_interp(P, mj, b0, w));
            double kc = 1.0;
            if (P->reflection_mode == 1) kc = band_interp(P, P->k_band + (int64_t)mj * P->n_bands, b0, w);
            else for (int q = 0; q < p->chain_len; ++q) kc *= band_interp(P, P->k_band + (int64_t)p->chain[q] * P->n_bands, b0, w);
            X = lobe * kc;
        } else if (p->kind == 1) {
            X = band_interp(P, P->diff_band + (int64_t)p->chain[0] * P->n_bands, b0, w);
        } else {
            X = P->direct_gain;
        }
        double alpha = P->a0 + P->a1_per_khz * (f / 1000.0);
        double A = X / (r * r) * pow(10.0, -alpha * r / 20.0) * emit_dir(P, p->dep, k) * mic_dir(P, mb, b0, w);
        double ph = 2.0 * M_PI * f * r / P->c;
        outm[2 * kk] += A * cos(ph);
        outm[2 * kk + 1] += A * sin(ph);
    }
}

static void unit_d(const float a[3], const float b[3], double o[3]) { /* normalize(a - b) in double */
    double v[3] = {(double)a[0] - b[0], (double)a[1] - b[1], (double)a[2] - b[2]};
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int k = 0; k < 3; ++k) o[k] = l > 0 ? v[k] / l : 0.0;
}

/*
 * Full or sampled spectra.  out has layout [3][n_m][n_k][2] for the selected microphones
 * (ms, or all when NULL) and bins (ks, or all when NULL).  Specular paths are the records with
 * rec_tri >= 0 and rec_los = 1 ([N][B] layout); the departure direction of ray i is q applied to
 * dirs[i].  Diffraction paths are the kept candidates; direct paths the visible microphones.
 */
ORA_API int ora_spectra(const OraSpecParams* P, int64_t N, int32_t B, const int32_t* rec_tri, const float* rec_p,
                        const float* rec_d, const double* rec_r, const uint8_t* rec_los, const float* dirs,
                        const int32_t* tri_mat, int64_t K, const int32_t* cand_tri, const float* cand_p,
                        const uint8_t* cand_keep, const uint8_t* direct_vis, int32_t n_m, const int32_t* ms,
                        int32_t n_k, const int32_t* ks, int32_t nthreads, const uint64_t* rec_mask, double* out) {
    int nm = ms ? n_m : P->M;
    int nk = ks ? n_k : P->F;
    memset(out, 0, sizeof(double) * 3 * (size_t)nm * nk * 2);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int mm = 0; mm < nm; ++mm) {
        int m = ms ? ms[mm] : mm;
        double* o_spec = out + ((0 * (int64_t)nm + mm) * nk) * 2;
        double* o_diff = out + ((1 * (int64_t)nm + mm) * nk) * 2;
        double* o_dir = out + ((2 * (int64_t)nm + mm) * nk) * 2;
        for (int64_t i = 0; i < N; ++i) {
            float d0[3];
            rotate_qf(P->q, dirs + 3 * i, d0);
            Path p;
            p.kind = 0;
            double dl = sqrt((double)d0[0] * d0[0] + (double)d0[1] * d0[1] + (double)d0[2] * d0[2]);
            for (int k = 0; k < 3; ++k) p.dep[k] = (double)d0[k] / dl;
            for (int32_t j = 0; j < B; ++j) {
                int64_t id = i * B + j;
                if (rec_tri[id] < 0) break;
                p.chain[j] = tri_mat[rec_tri[id]];
                if (!rec_los[id]) continue;
                if (rec_mask && !((rec_mask[id] >> m) & 1u)) continue;  /* per-microphone receiver test */
                for (int k = 0; k < 3; ++k) { p.P[k] = rec_p[3 * id + k]; p.dref[k] = rec_d[3 * id + k]; }
                p.r_pre = rec_r[id];
                p.chain_len = j + 1;
                add_path(P, &p, m, nk, ks, o_spec);
            }
        }
        for (int64_t c = 0; c < K; ++c) {
            if (cand_keep && !cand_keep[c]) continue;
            Path p;
            p.kind = 1;
            for (int k = 0; k < 3; ++k) p.P[k] = cand_p[3 * c + k];
            double v[3] = {p.P[0] - P->s[0], p.P[1] - P->s[1], p.P[2] - P->s[2]};
            p.r_pre = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            unit_d(cand_p + 3 * c, P->s, p.dep);
            p.chain_len = 1;
            p.chain[0] = tri_mat[cand_tri[c]];
            add_path(P, &p, m, nk, ks, o_diff);
        }
        if (direct_vis && direct_vis[m]) {
            Path p;
            p.kind = 2;
            for (int k = 0; k < 3; ++k) p.P[k] = P->s[k];
            p.r_pre = 0.0;
            unit_d(P->mics + 3 * m, P->s, p.dep);
            p.chain_len = 0;
            add_path(P, &p, m, nk, ks, o_dir);
        }
    }
    return 0;
}

/*
 * Analytic gradient (float64) of L through the spectra with the path set frozen, given
 * G = dL/dRe S + j dL/dIm S ([3][M][F][2]): dL/dtheta = sum Re(conj(G) dS/dtheta).
 *   dk  [n_mat][n_bands]: reflection band values (specular paths).
 *   dmic[M][3]: microphone positions (all three components; omni microphones).
 *   demit[3]:   emitter position through the diffraction and direct paths (omni emitter);
 *               the specular paths' dependence on the emitter (through the whole chain) is not included.
 * rec_mask (NULL or [N][B]): with the per-microphone receiver test a record reaches microphone m only
 * when bit m is set, as in ora_spectra; the terms it does not reach have no gradient.
 * Directivity tables must be absent for the position gradients (returns -1 otherwise).
 */
ORA_API int ora_spectra_grad(const OraSpecParams* P, int64_t N, int32_t B, const int32_t* rec_tri, const float* rec_p,
                             const float* rec_d, const double* rec_r, const uint8_t* rec_los, const float* dirs,
                             const int32_t* tri_mat, int64_t K, const int32_t* cand_tri, const float* cand_p,
                             const uint8_t* cand_keep, const uint8_t* direct_vis, const double* G,
                             double* dk, double* dmic, double* demit, double* dbeta, const float* tri_nrm,
                             double* demit_spec, const uint64_t* rec_mask) {
    if (P->emit_table || P->mic_tables) return -1;
    int F = P->F, M = P->M;
    memset(dk, 0, sizeof(double) * (size_t)P->n_mat * P->n_bands);
    if (dbeta) memset(dbeta, 0, sizeof(double) * (size_t)P->n_mat * P->n_bands);
    if (demit_spec) memset(demit_spec, 0, sizeof(double) * 3);
    memset(dmic, 0, sizeof(double) * 3 * (size_t)M);
    memset(demit, 0, sizeof(double) * 3);
    for (int m = 0; m < M; ++m) {
        const float* mf = P->mics + 3 * m;
        /* ---- specular */
        for (int64_t i = 0; i < N; ++i) {
            int chain[16];
            for (int32_t j = 0; j < B; ++j) {
                int64_t id = i * B + j;
                if (rec_tri[id] < 0) break;
                chain[j] = tri_mat[rec_tri[id]];
                if (!rec_los[id]) continue;
                if (rec_mask && !((rec_mask[id] >> m) & 1u)) continue;  /* per-microphone receiver test */
                double Pp[3] = {rec_p[3 * id], rec_p[3 * id + 1], rec_p[3 * id + 2]};
                double dr[3] = {rec_d[3 * id], rec_d[3 * id + 1], rec_d[3 * id + 2]};
                double v[3] = {mf[0] - Pp[0], mf[1] - Pp[1], mf[2] - Pp[2]};
                double dist = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                double u[3] = {v[0] / dist, v[1] / dist, v[2] / dist};
                double r = rec_r[id] + dist;
                double cx[3] = {dr[1] * u[2] - dr[2] * u[1], dr[2] * u[0] - dr[0] * u[2], dr[0] * u[1] - dr[1] * u[0]};
                double sg = sqrt(cx[0] * cx[0] + cx[1] * cx[1] + cx[2] * cx[2]);
                double cg = dr[0] * u[0] + dr[1] * u[1] + dr[2] * u[2];
                double gm = atan2(sg, cg);
                /* d gamma / d m: gamma = acos(dr . u), du/dm = (I - u u^T)/dist
                 * => dgamma/dm = -(dr - (dr.u) u) / (dist sin gamma)  (0 when sin gamma = 0) */
                double dgdm[3] = {0, 0, 0};
                if (sg > 1e-300)
                    for (int k = 0; k < 3; ++k) dgdm[k] = -(dr[k] - cg * u[k]) / (dist * sg);
                int mj = chain[j];
                double acc_r = 0.0, acc_g = 0.0;
                for (int k = 0; k < F; ++k) {
                    double f = freq_of(P, k);
                    int b0; double w;
                    band_weights(P, f, &b0, &w);
                    double g = g_interp(P, mj, b0, w);
                    double lobe = exp(-gm * gm * g);
                    double kv[16], kc = 1.0;
                    int L = (P->reflection_mode == 1) ? 1 : j + 1;
                    for (int q = 0; q < L; ++q) {
                        int mat = (P->reflection_mode == 1) ? mj : chain[q];
                        kv[q] = band_interp(P, P->k_band + (int64_t)mat * P->n_bands, b0, w);
                        kc *= kv[q];
                    }
                    double alpha = P->a0 + P->a1_per_khz * (f / 1000.0);
                    double atm = pow(10.0, -alpha * r / 20.0);
                    double base = lobe * atm / (r * r);
                    double ph = 2.0 * M_PI * f * r / P->c;
                    double zr = cos(ph), zi = sin(ph);
                    const double* Gk = G + ((0 * (int64_t)M + m) * F + k) * 2;
                    double re_gz = Gk[0] * zr + Gk[1] * zi;       /* Re(conj(G) e^{j ph}) */
                    double im_gz = Gk[0] * zi - Gk[1] * zr;       /* Im(conj(G) e^{j ph}) */
                    /* reflection coefficient gradient */
                    for (int q = 0; q < L; ++q) {
                        int mat = (P->reflection_mode == 1) ? mj : chain[q];
                        double others = 1.0;
                        for (int q2 = 0; q2 < L; ++q2) if (q2 != q) others *= kv[q2];
                        double d = base * others * re_gz;
                        if (P->n_bands == 1) dk[(int64_t)mat * P->n_bands] += d;
                        else {
                            dk[(int64_t)mat * P->n_bands + b0] += (1.0 - w) * d;
                            dk[(int64_t)mat * P->n_bands + b0 + 1] += w * d;
                        }
                    }
                    double A = base * kc;
                    /* lobe widths: lobe = exp(-gamma^2 g), g = (1 - w) / (2 beta_b0^2) + w / (2 beta_b1^2)
                     * => d lobe / d beta_b = lobe gamma^2 weight_b / beta_b^3 (last hit's material) */
                    if (dbeta) {
                        const float* brow = P->beta_band + (int64_t)mj * P->n_bands;
                        double d = A * re_gz * gm * gm;
                        if (P->n_bands == 1) {
                            double bb = (double)brow[0];
                            dbeta[(int64_t)mj * P->n_bands] += d / (bb * bb * bb);
                        } else {
                            double bl = (double)brow[b0], bh = (double)brow[b0 + 1];
                            dbeta[(int64_t)mj * P->n_bands + b0] += d * (1.0 - w) / (bl * bl * bl);
                            dbeta[(int64_t)mj * P->n_bands + b0 + 1] += d * w / (bh * bh * bh);
                        }
                    }
                    /* dA/dr = A (-2/r - alpha ln10 / 20); dphase/dr = 2 pi f / c */
                    double dlnA_dr = -2.0 / r - alpha * M_LN10 / 20.0;
                    acc_r += A * (dlnA_dr * re_gz - (2.0 * M_PI * f / P->c) * im_gz);
                    acc_g += A * (-2.0 * gm * g) * re_gz;
                }
                for (int k = 0; k < 3; ++k) dmic[3 * m + k] += acc_r * u[k] + acc_g * dgdm[k];
                /* emitter through the hit points (ray directions and triangle chain frozen): hit q is
                 * the intersection of the line from P_{q-1} along d_q with triangle q's plane, so
                 * dP_q/dP_{q-1} = I - d_q n_q^T / (n_q . d_q) and dt_q/dP_{q-1} = -n_q^T / (n_q . d_q),
                 * P_{-1} = s.  With J = dP_j/ds and dr_j/ds = sum_q dt_q/ds:
                 * dL/ds += (dr_j/ds) acc_r - J^T (acc_r u + acc_g dgamma/dm)   (d|m - P|/dP = -u,
                 * dgamma/dP = -dgamma/dm). */
                if (demit_spec && tri_nrm) {
                    double J[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, drds[3] = {0, 0, 0};
                    float d0f[3];
                    rotate_qf(P->q, dirs + 3 * i, d0f);
                    double dq[3] = {d0f[0], d0f[1], d0f[2]};
                    for (int32_t q = 0; q <= j; ++q) {
                        const float* nf = tri_nrm + 3 * (int64_t)rec_tri[i * B + q];
                        double n[3] = {nf[0], nf[1], nf[2]};
                        double nd = n[0] * dq[0] + n[1] * dq[1] + n[2] * dq[2];
                        double nJ[3];
                        for (int c2 = 0; c2 < 3; ++c2) nJ[c2] = n[0] * J[c2] + n[1] * J[3 + c2] + n[2] * J[6 + c2];
                        for (int c2 = 0; c2 < 3; ++c2) drds[c2] -= nJ[c2] / nd;
                        for (int r2 = 0; r2 < 3; ++r2)
                            for (int c2 = 0; c2 < 3; ++c2) J[3 * r2 + c2] -= dq[r2] * nJ[c2] / nd;
                        const float* dn = rec_d + 3 * (i * B + q);
                        dq[0] = dn[0];
                        dq[1] = dn[1];
                        dq[2] = dn[2];
                    }
                    double gp[3];
                    for (int k = 0; k < 3; ++k) gp[k] = acc_r * u[k] + acc_g * dgdm[k];
                    for (int c2 = 0; c2 < 3; ++c2)
                        demit_spec[c2] += drds[c2] * acc_r - (J[c2] * gp[0] + J[3 + c2] * gp[1] + J[6 + c2] * gp[2]);
                }
            }
        }
        /* ---- diffraction */
        for (int64_t c = 0; c < K; ++c) {
            if (cand_keep && !cand_keep[c]) continue;
            double o[3] = {cand_p[3 * c], cand_p[3 * c + 1], cand_p[3 * c + 2]};
            double vs[3] = {o[0] - P->s[0], o[1] - P->s[1], o[2] - P->s[2]};
            double d1 = sqrt(vs[0] * vs[0] + vs[1] * vs[1] + vs[2] * vs[2]);
            double vm[3] = {mf[0] - o[0], mf[1] - o[1], mf[2] - o[2]};
            double d2 = sqrt(vm[0] * vm[0] + vm[1] * vm[1] + vm[2] * vm[2]);
            double r = d1 + d2;
            int mat = tri_mat[cand_tri[c]];
            double acc = 0.0;
            for (int k = 0; k < F; ++k) {
                double f = freq_of(P, k);
                int b0; double w;
                band_weights(P, f, &b0, &w);
                double X = band_interp(P, P->diff_band + (int64_t)mat * P->n_bands, b0, w);
                double alpha = P->a0 + P->a1_per_khz * (f / 1000.0);
                double A = X / (r * r) * pow(10.0, -alpha * r / 20.0);
                double ph = 2.0 * M_PI * f * r / P->c;
                const double* Gk = G + ((1 * (int64_t)M + m) * F + k) * 2;
                double re_gz = Gk[0] * cos(ph) + Gk[1] * sin(ph);
                double im_gz = Gk[0] * sin(ph) - Gk[1] * cos(ph);
                acc += A * ((-2.0 / r - alpha * M_LN10 / 20.0) * re_gz - (2.0 * M_PI * f / P->c) * im_gz);
            }
            for (int k = 0; k < 3; ++k) {
                dmic[3 * m + k] += acc * vm[k] / d2;
                demit[k] += acc * (-vs[k] / d1);
            }
        }
        /* ---- direct */
        if (direct_vis && direct_vis[m]) {
            double v[3] = {mf[0] - P->s[0], mf[1] - P->s[1], mf[2] - P->s[2]};
            double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            double acc = 0.0;
            for (int k = 0; k < F; ++k) {
                double f = freq_of(P, k);
                double alpha = P->a0 + P->a1_per_khz * (f / 1000.0);
                double A = P->direct_gain / (r * r) * pow(10.0, -alpha * r / 20.0);
                double ph = 2.0 * M_PI * f * r / P->c;
                const double* Gk = G + ((2 * (int64_t)M + m) * F + k) * 2;
                double re_gz = Gk[0] * cos(ph) + Gk[1] * sin(ph);
                double im_gz = Gk[0] * sin(ph) - Gk[1] * cos(ph);
                acc += A * ((-2.0 / r - alpha * M_LN10 / 20.0) * re_gz - (2.0 * M_PI * f / P->c) * im_gz);
            }
            for (int k = 0; k < 3; ++k) {
                dmic[3 * m + k] += acc * v[k] / r;
                demit[k] -= acc * v[k] / r;
            }
        }
    }
    return 0;
}
