// Scene pre-processing on the device (Sec. III-B, Sec. III-D):
//   validation, geometric normals, vertex welding, one-ring adjacency (ascending triangle ids),
//   Meyer mean curvature G_v, the triangle metric C_i (Eq. 1), per-mesh dithered integer CDFs and
//   diffraction sample counts, and a linear BVH (Morton codes, radix sort, Karras hierarchy,
//   bottom-up boxes, small subtrees collapsed into leaves of <= 4 triangles).
// Compiled with -fmad=false: curvature and CDF weights decide which triangles are sampled.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "st_geom.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

#define CK(x)                                \
    do {                                     \
        cudaError_t e_ = (x);                \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

constexpr int kB = 256;

__device__ __forceinline__ f3 vload(const float* V, int64_t i) { return f3{V[3 * i], V[3 * i + 1], V[3 * i + 2]}; }

__global__ void k_validate(const float* V, int64_t nv, const int32_t* T, int64_t nt, const int32_t* mat,
                           int32_t n_mat, const int32_t* obj, uint32_t* flags) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv + nt; i += stride) {
        if (i < nv) {
            float x = V[3 * i], y = V[3 * i + 1], z = V[3 * i + 2];
            if (!(isfinite(x) && isfinite(y) && isfinite(z))) atomicOr(flags, kFlagBadVertex);
        } else {
            int64_t t = i - nv;
            for (int k = 0; k < 3; ++k) {
                int32_t v = T[3 * t + k];
                if (v < 0 || v >= nv) atomicOr(flags, kFlagBadIndex);
            }
            if (mat[t] < 0 || mat[t] >= n_mat || obj[t] < 0) atomicOr(flags, kFlagBadIndex);
        }
    }
}

__global__ void k_normals(const float* V, const int32_t* T, int64_t nt, float* N) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        f3 a = vload(V, T[3 * t]), b = vload(V, T[3 * t + 1]), c = vload(V, T[3 * t + 2]);
        float l;
        f3 n = normalize(cross(sub(b, a), sub(c, a)), &l);
        N[3 * t] = n.x;
        N[3 * t + 1] = n.y;
        N[3 * t + 2] = n.z;
    }
}

// ---------------------------------------------------------------- welding
__device__ __forceinline__ uint32_t pos_bits(float x) { return __float_as_uint(x + 0.0f); }  // -0 -> +0

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdull;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ull;
    z ^= z >> 33;
    return z;
}

__global__ void k_pos_keys(const float* V, int64_t nv, uint64_t* keys, uint32_t* vals) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        uint64_t h = mix64(pos_bits(V[3 * i]));
        h = mix64(h ^ pos_bits(V[3 * i + 1]));
        h = mix64(h ^ ((uint64_t)pos_bits(V[3 * i + 2]) << 17));
        keys[i] = h;
        vals[i] = (uint32_t)i;
    }
}

__device__ __forceinline__ bool same_pos(const float* V, uint32_t a, uint32_t b) {
    return pos_bits(V[3 * (int64_t)a]) == pos_bits(V[3 * (int64_t)b]) &&
           pos_bits(V[3 * (int64_t)a + 1]) == pos_bits(V[3 * (int64_t)b + 1]) &&
           pos_bits(V[3 * (int64_t)a + 2]) == pos_bits(V[3 * (int64_t)b + 2]);
}

// One thread per run of equal hashes: canon[v] = smallest index with exactly the same position.
__global__ void k_weld_runs(const float* V, int64_t nv, const uint64_t* keys, const uint32_t* vals, int32_t* canon) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        int64_t j = i + 1;
        while (j < nv && keys[j] == keys[i]) ++j;
        for (int64_t a = i; a < j; ++a) {
            uint32_t va = vals[a];
            uint32_t best = va;
            for (int64_t b = i; b < j; ++b) {
                uint32_t vb = vals[b];
                if (vb < best && same_pos(V, va, vb)) best = vb;
            }
            canon[va] = (int32_t)best;
        }
    }
}

// ---------------------------------------------------------------- adjacency
__device__ __forceinline__ bool tri_corner_dup(const int32_t* canon, const int32_t* T, int64_t t, int k) {
    int32_t c = canon[T[3 * t + k]];
    for (int q = 0; q < k; ++q)
        if (canon[T[3 * t + q]] == c) return true;
    return false;
}

__global__ void k_adj_count(const int32_t* canon, const int32_t* T, int64_t nt, uint32_t* cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride)
        for (int k = 0; k < 3; ++k)
            if (!tri_corner_dup(canon, T, t, k)) atomicAdd(&cnt[canon[T[3 * t + k]]], 1u);
}

__global__ void k_adj_fill(const int32_t* canon, const int32_t* T, int64_t nt, const uint32_t* off, uint32_t* cursor,
                           int32_t* adj) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride)
        for (int k = 0; k < 3; ++k)
            if (!tri_corner_dup(canon, T, t, k)) {
                int32_t c = canon[T[3 * t + k]];
                uint32_t p = atomicAdd(&cursor[c], 1u);
                adj[off[c] + p] = (int32_t)t;
            }
}

__global__ void k_adj_sort(int64_t nv, const uint32_t* off, int32_t* adj) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        uint32_t a = off[v], b = off[v + 1];
        for (uint32_t i = a + 1; i < b; ++i) {
            int32_t x = adj[i];
            uint32_t j = i;
            while (j > a && adj[j - 1] > x) {
                adj[j] = adj[j - 1];
                --j;
            }
            adj[j] = x;
        }
    }
}

// ---------------------------------------------------------------- Meyer curvature (Sec. III-B)
// For canonical vertex v and each incident triangle (v, a, b) in ascending triangle index:
//   cot at a = (v-a).(b-a) / |(a-v) x (b-v)|, cot at b = (v-b).(a-b) / |(a-v) x (b-v)|,
//   sum += cot_b (v - a) + cot_a (v - b); A_mixed += Voronoi area, or area/2 (obtuse at v),
//   or area/4 (obtuse elsewhere);  G_v = |sum / (2 A_mixed)| / 2.
__global__ void k_curvature(const float* V, int64_t nv, const int32_t* T, const int32_t* canon, const uint32_t* off,
                            const int32_t* adj, float* Gc) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        if (canon[v] != v) continue;
        f3 xv = vload(V, v);
        float Sx = 0.0f, Sy = 0.0f, Sz = 0.0f, Amix = 0.0f;
        for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
            int64_t t = adj[e];
            int32_t c0 = canon[T[3 * t]], c1 = canon[T[3 * t + 1]], c2 = canon[T[3 * t + 2]];
            if (c0 == c1 || c1 == c2 || c0 == c2) continue;
            int32_t ia, ib;
            if (c0 == v) {
                ia = c1;
                ib = c2;
            } else if (c1 == v) {
                ia = c2;
                ib = c0;
            } else {
                ia = c0;
                ib = c1;
            }
            f3 xa = vload(V, ia), xb = vload(V, ib);
            f3 va = sub(xv, xa), ba = sub(xb, xa), vb = sub(xv, xb), ab = sub(xa, xb), av = sub(xa, xv),
               bv = sub(xb, xv);
            f3 cr = cross(av, bv);
            float cross_len = sqrtf(dot(cr, cr));
            if (!(cross_len > 0.0f)) continue;
            float cot_a = dot(va, ba) / cross_len;
            float cot_b = dot(vb, ab) / cross_len;
            {
                float t1 = cot_b * va.x, t2 = cot_a * vb.x;
                Sx = Sx + (t1 + t2);
                t1 = cot_b * va.y;
                t2 = cot_a * vb.y;
                Sy = Sy + (t1 + t2);
                t1 = cot_b * va.z;
                t2 = cot_a * vb.z;
                Sz = Sz + (t1 + t2);
            }
            float area = 0.5f * cross_len;
            float dv = dot(av, bv), da = dot(va, ba), db = dot(vb, ab);
            float amix;
            if (dv < 0.0f)
                amix = area / 2.0f;
            else if (da < 0.0f || db < 0.0f)
                amix = area / 4.0f;
            else {
                float lvb = dot(vb, vb), lva = dot(va, va);
                float p1 = lvb * cot_a, p2 = lva * cot_b;
                amix = (p1 + p2) / 8.0f;
            }
            Amix = Amix + amix;
        }
        float g = 0.0f;
        if (Amix > 0.0f) {
            float den = 2.0f * Amix;
            f3 K{Sx / den, Sy / den, Sz / den};
            g = 0.5f * sqrtf(dot(K, K));
        }
        Gc[v] = g;
    }
}

__global__ void k_expand_G(const int32_t* canon, int64_t nv, const float* Gc, float* G) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) G[v] = Gc[canon[v]];
}

// Eq. 1: C_i = eta * w(A_i) * (max G - min G), w(A) = clamp(A / A_ref, 0, 1).
__global__ void k_metric(const float* V, const int32_t* T, int64_t nt, const int32_t* canon, const float* G, float eta,
                         float area_ref, float* C, uint32_t* cmax_bits, const int32_t* obj) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        int32_t i0 = T[3 * t], i1 = T[3 * t + 1], i2 = T[3 * t + 2];
        float c = 0.0f;
        if (!(canon[i0] == canon[i1] || canon[i1] == canon[i2] || canon[i0] == canon[i2])) {
            f3 a = vload(V, i0);
            f3 cr = cross(sub(vload(V, i1), a), sub(vload(V, i2), a));
            float A = 0.5f * sqrtf(dot(cr, cr));
            if (A > 0.0f) {
                float w = A / area_ref;
                if (w > 1.0f) w = 1.0f;
                if (w < 0.0f) w = 0.0f;
                float g0 = G[i0], g1 = G[i1], g2 = G[i2];
                float gmax = fmaxf(fmaxf(g0, g1), g2), gmin = fminf(fminf(g0, g1), g2);
                float ew = eta * w;
                c = ew * (gmax - gmin);
            }
        }
        C[t] = c;
        atomicMax(&cmax_bits[obj[t]], __float_as_uint(c));  // c >= 0: bit order = value order
    }
}

// ---------------------------------------------------------------- diffraction CDFs (Sec. III-D)
__device__ __forceinline__ void philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                                         uint32_t out[4]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

__global__ void k_mesh_count(const int32_t* obj, int64_t nt, uint32_t* cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) atomicAdd(&cnt[obj[t]], 1u);
}

__global__ void k_mesh_keys(const int32_t* obj, int64_t nt, uint64_t* keys, uint32_t* vals) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        keys[t] = ((uint64_t)(uint32_t)obj[t] << 32) | (uint64_t)t;
        vals[t] = (uint32_t)t;
    }
}

__global__ void k_quantize(const int32_t* mesh_tris, int64_t nt, const int32_t* obj, const float* C,
                           const uint32_t* cmax_bits, uint64_t* Q, unsigned long long* sumQ) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += stride) {
        int32_t t = mesh_tris[i];
        int32_t m = obj[t];
        float cmax = __uint_as_float(cmax_bits[m]);
        uint64_t q = 0;
        if (cmax > 0.0f) {
            float r = C[t] / cmax;
            float s = r * 16777216.0f;
            q = (uint64_t)floorf(s);
        }
        Q[i] = q;
        atomicAdd(&sumQ[m], (unsigned long long)q);
    }
}

__global__ void k_dither(const int32_t* mesh_tris, int64_t nt, const int32_t* obj, const uint32_t* mesh_off,
                         const unsigned long long* sumQ, double dither, uint64_t seed, uint64_t* Q) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += stride) {
        int32_t t = mesh_tris[i];
        int32_t m = obj[t];
        double n = (double)(mesh_off[m + 1] - mesh_off[m]);
        double mean = (double)sumQ[m] / n;
        double scale = dither * mean;
        uint32_t x[4];
        philox10((uint32_t)t, 0u, 0u, 1u, seed, x);
        double xi = (double)(x[0] >> 8) * (1.0 / 16777216.0);
        double d = floor(scale * xi);
        Q[i] += (uint64_t)d;
    }
}

__global__ void k_cdf_fix(const uint64_t* S, int64_t nt, const int32_t* mesh_tris, const int32_t* obj,
                          const uint32_t* mesh_off, uint64_t* cdf) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += stride) {
        int32_t m = obj[mesh_tris[i]];
        uint32_t start = mesh_off[m];
        cdf[i] = S[i] - (start > 0 ? S[start - 1] : 0ull);
    }
}

// Per canonical vertex: the distinct meshes among its incident high-curvature triangles
// (C > 0 and C >= hc_frac * max C of the mesh) each count the vertex once.
__global__ void k_hc_vertices(int64_t nv, const int32_t* canon, const uint32_t* off, const int32_t* adj,
                              const int32_t* obj, const float* C, const uint32_t* cmax_bits, float hc_frac,
                              int32_t spv, unsigned long long* ns) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        if (canon[v] != v) continue;
        for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
            int32_t t = adj[e];
            int32_t m = obj[t];
            float thr = hc_frac * __uint_as_float(cmax_bits[m]);
            if (!(C[t] > 0.0f && C[t] >= thr)) continue;
            bool seen = false;
            for (uint32_t e2 = off[v]; e2 < e && !seen; ++e2) {
                int32_t t2 = adj[e2];
                if (obj[t2] != m) continue;
                if (C[t2] > 0.0f && C[t2] >= thr) seen = true;
            }
            if (!seen) atomicAdd(&ns[m], (unsigned long long)spv);
        }
    }
}

// (n * budget) / total without overflow (n <= total, budget < 2^63): 128-by-64 long division on 64-bit halves
__device__ __forceinline__ unsigned long long scaled_count(unsigned long long n, unsigned long long budget,
                                                           unsigned long long total) {
    const unsigned long long hi = __umul64hi(n, budget), lo = n * budget;
    unsigned long long q = 0, r = 0;
    for (int bit = 127; bit >= 0; --bit) {
        const unsigned long long b = bit >= 64 ? (hi >> (bit - 64)) & 1ull : (lo >> bit) & 1ull;
        const unsigned long long top = r >> 63;
        r = (r << 1) | b;
        if (top || r >= total) {
            r -= total;
            if (bit < 64) q |= 1ull << bit;
        }
    }
    return q;
}

// One block: empty meshes get no samples, the total is capped by the budget, offsets scanned.  Each thread takes
// the meshes tid, tid + kScThreads, ...; integer sums, so the result does not depend on the order.
constexpr int kScThreads = 1024;
__global__ void __launch_bounds__(kScThreads) k_sample_counts(int32_t n_obj, const uint32_t* mesh_off,
                                                              const uint64_t* cdf, unsigned long long* ns,
                                                              int64_t budget, int64_t* n_samples, int64_t* sample_off) {
    __shared__ unsigned long long wsum[kScThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long part = 0;
    for (int32_t m = tid; m < n_obj; m += kScThreads) {
        const uint32_t a = mesh_off[m], b = mesh_off[m + 1];
        if (b <= a || cdf[b - 1] == 0) ns[m] = 0;
        part += ns[m];
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) wsum[warp] = part;
    __syncthreads();
    unsigned long long total = 0;
    for (int w = 0; w < kScThreads / 32; ++w) total += wsum[w];
    __syncthreads();  // wsum is reused by the scans below
    const bool cap = budget >= 0 && total > (unsigned long long)budget;
    int64_t carry = 0;
    for (int32_t base = 0; base < n_obj; base += kScThreads) {
        const int32_t m = base + tid;
        unsigned long long n = m < n_obj ? ns[m] : 0ull;
        if (m < n_obj && cap) n = scaled_count(n, (unsigned long long)budget, total);
        // exclusive scan over the block: within the warp, then over the warp totals
        unsigned long long x = n;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        unsigned long long before = 0, chunk = 0;
        for (int w = 0; w < kScThreads / 32; ++w) {
            if (w < warp) before += wsum[w];
            chunk += wsum[w];
        }
        if (m < n_obj) {
            n_samples[m] = (int64_t)n;
            sample_off[m] = carry + (int64_t)(before + x - n);
        }
        carry += (int64_t)chunk;
        __syncthreads();  // wsum is rewritten by the next chunk
    }
    if (tid == 0) sample_off[n_obj] = carry;
}

// ---------------------------------------------------------------- LBVH
__device__ __forceinline__ uint32_t ord(float f) {  // monotone float -> uint
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_bounds(const float* V, int64_t nv, uint32_t* bnd /*[6]: lo ord, hi ord*/) {
    __shared__ uint32_t s[6];
    if (threadIdx.x < 3) s[threadIdx.x] = 0xffffffffu;
    else if (threadIdx.x < 6) s[threadIdx.x] = 0u;
    __syncthreads();
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride)
        for (int k = 0; k < 3; ++k) {
            uint32_t o = ord(V[3 * i + k]);
            lo[k] = min(lo[k], o);
            hi[k] = max(hi[k], o);
        }
    for (int k = 0; k < 3; ++k) {
        atomicMin(&s[k], lo[k]);
        atomicMax(&s[3 + k], hi[k]);
    }
    __syncthreads();
    if (threadIdx.x < 3) atomicMin(&bnd[threadIdx.x], s[threadIdx.x]);
    else if (threadIdx.x < 6) atomicMax(&bnd[threadIdx.x], s[threadIdx.x]);
}

__device__ __forceinline__ uint64_t spread21(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__global__ void k_morton(const float* V, const int32_t* T, int64_t nt, const uint32_t* bnd, uint64_t* keys,
                         uint32_t* vals) {
    float lo[3], ext[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = unord(bnd[k]);
        float hi = unord(bnd[3 + k]);
        ext[k] = hi - lo[k];
    }
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        uint64_t q[3];
        for (int k = 0; k < 3; ++k) {
            float c = (V[3 * (int64_t)T[3 * t] + k] + V[3 * (int64_t)T[3 * t + 1] + k]) + V[3 * (int64_t)T[3 * t + 2] + k];
            c = c * (1.0f / 3.0f);
            float u = ext[k] > 0.0f ? (c - lo[k]) / ext[k] : 0.5f;
            u = fminf(fmaxf(u, 0.0f), 1.0f);
            uint32_t qi = (uint32_t)(u * 2097151.0f);
            q[k] = qi;
        }
        keys[t] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
        vals[t] = (uint32_t)t;
    }
}

// Morton keys of n points P [n][3] in the bounds bnd (the top level's instance box centres)
__global__ void k_morton_pts(const float* P, int64_t n, const uint32_t* bnd, uint64_t* keys, uint32_t* vals) {
    float lo[3], ext[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = unord(bnd[k]);
        ext[k] = unord(bnd[3 + k]) - lo[k];
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        uint64_t q[3];
        for (int k = 0; k < 3; ++k) {
            float u = ext[k] > 0.0f ? (P[3 * t + k] - lo[k]) / ext[k] : 0.5f;
            u = fminf(fmaxf(u, 0.0f), 1.0f);
            q[k] = (uint32_t)(u * 2097151.0f);
        }
        keys[t] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
        vals[t] = (uint32_t)t;
    }
}

__device__ __forceinline__ int delta(const uint64_t* k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    uint64_t a = k[i], b = k[j];
    if (a == b) return 64 + __clz((uint32_t)(i ^ j));
    return __clzll(a ^ b);
}

// Karras (HPG 2012): internal node i covers a key range; children are leaves at the range ends.
__global__ void k_karras(const uint64_t* keys, int n, int2* child /*[n-1]: encoded (x<0 = leaf ~idx)*/,
                         int2* range, int32_t* parent_int, int32_t* parent_leaf) {
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += stride) {
        int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
        int dmin = delta(keys, n, i, i - d);
        int lmax = 2;
        while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
        int l = 0;
        for (int t = lmax / 2; t >= 1; t /= 2)
            if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
        int j = i + l * d;
        int dnode = delta(keys, n, i, j);
        int s = 0;
        int t = l;
        do {
            t = (t + 1) >> 1;
            if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
        } while (t > 1);
        int gamma = i + s * d + min(d, 0);
        int lo = min(i, j), hi = max(i, j);
        int left = (lo == gamma) ? ~gamma : gamma;
        int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
        child[i] = make_int2(left, right);
        range[i] = make_int2(lo, hi);
        if (left < 0) parent_leaf[gamma] = i; else parent_int[gamma] = i;
        if (right < 0) parent_leaf[gamma + 1] = i; else parent_int[gamma + 1] = i;
    }
}

struct Box {
    float lo[3], hi[3];
};

// leaf boxes: a triangle's vertex bounds grown by pad; an instance's world box (from its record)
struct TriLeafBox {
    const float* V;
    const int32_t* T;
    const uint32_t* sorted;
    float pad;
    __device__ __forceinline__ Box operator()(int p) const {
        const int64_t t = sorted[p];
        Box b;
        for (int k = 0; k < 3; ++k) {
            float a = V[3 * (int64_t)T[3 * t] + k], bb = V[3 * (int64_t)T[3 * t + 1] + k],
                  c = V[3 * (int64_t)T[3 * t + 2] + k];
            b.lo[k] = fminf(fminf(a, bb), c) - pad;
            b.hi[k] = fmaxf(fmaxf(a, bb), c) + pad;
        }
        return b;
    }
};
struct InstLeafBox {
    const float4* rec;
    const int32_t* sorted;
    __device__ __forceinline__ Box operator()(int p) const {
        const int64_t i = sorted[p];
        const float4 lo = rec[8 * i + 6], hi = rec[8 * i + 7];
        return Box{{lo.x, lo.y, lo.z}, {hi.x, hi.y, hi.z}};
    }
};

// Bottom-up boxes: each leaf writes its box into its parent's slot; the second child to arrive at
// a node unites both slots and climbs.  box_tmp: [n-1][2] boxes.
template <class LeafBox>
__global__ void k_boxes(const LeafBox leaf, int n, const int2* child, const int32_t* parent_int,
                        const int32_t* parent_leaf, Box* box_tmp, uint32_t* visits, uint32_t* err) {
    int stride = gridDim.x * blockDim.x;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const Box b = leaf(p);
        int node = parent_leaf[p];
        int slot = (child[node].x == ~p) ? 0 : 1;
        box_tmp[2 * node + slot] = b;
        for (int climb = 0;; ++climb) {
            if (climb > n) {  // deeper than the node count: not a tree
                atomicOr(err, kFlagBadTree);
                break;
            }
            __threadfence();
            uint32_t old = atomicAdd(&visits[node], 1u);
            if (old == 0) break;
            if (old > 1) {  // a node has two children: a third arrival means a malformed hierarchy
                atomicOr(err, kFlagBadTree);
                break;
            }
            __threadfence();
            const volatile float* b0 = reinterpret_cast<const volatile float*>(&box_tmp[2 * node]);
            const volatile float* b1 = reinterpret_cast<const volatile float*>(&box_tmp[2 * node + 1]);
            Box u;
            for (int k = 0; k < 3; ++k) {
                u.lo[k] = fminf(b0[k], b1[k]);
                u.hi[k] = fmaxf(b0[3 + k], b1[3 + k]);
            }
            if (node == 0) break;
            int par = parent_int[node];
            int s2 = (child[par].x == node) ? 0 : 1;
            volatile float* dst = reinterpret_cast<volatile float*>(&box_tmp[2 * par + s2]);
            for (int k = 0; k < 3; ++k) {
                dst[k] = u.lo[k];
                dst[3 + k] = u.hi[k];
            }
            node = par;
        }
    }
}

__host__ __device__ __forceinline__ int32_t leaf_ref(int first, int count) { return ~((first << 3) | (count - 1)); }

// child reference of binary node i's side c: a leaf code for single triangles and for subtrees of at
// most kLeafMax triangles (a contiguous range of the leaf order), else the internal node index
__device__ __forceinline__ int32_t child_ref(int32_t cc, const int2* range, int32_t leaf_off) {
    if (cc < 0) return leaf_ref(~cc + leaf_off, 1);
    const int2 r = range[cc];
    const int cnt = r.y - r.x + 1;
    return cnt <= kLeafMax ? leaf_ref(r.x + leaf_off, cnt) : cc;
}

// Binary internal nodes that stay internal (range above kLeafMax, or the root) at even depth become
// the nodes of the 4-wide BVH: each takes its children, with internal children replaced by theirs.
__global__ void k_wide_flags(int n, const int2* range, const int32_t* parent_int, uint32_t* flag, uint32_t* err) {
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += stride) {
        const int2 r = range[i];
        const bool internal = i == 0 || r.y - r.x + 1 > kLeafMax;
        uint32_t f = 0;
        if (internal) {
            int d = 0, x = i;
            while (x != 0) {
                x = parent_int[x];
                if (++d > n) {  // deeper than the node count: not a tree
                    atomicOr(err, kFlagBadTree);
                    break;
                }
            }
            f = (d & 1) == 0 ? 1u : 0u;
        }
        flag[i] = f;
    }
}

// nodes: the first node of this hierarchy; stored node references are offset by node_off and leaf codes'
// first triangles by leaf_off (several hierarchies in one array)
__global__ void k_pack_wide(int n, const int2* child, const int2* range, const Box* box_tmp, const uint32_t* flag,
                            const uint32_t* idx, float4* nodes, int32_t node_off, int32_t leaf_off) {
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += stride) {
        if (!flag[i]) continue;
        float lo[3][4], hi[3][4];
        int32_t ref[4];
        int cnt = 0;
        auto add = [&](const Box& b, int32_t r) {
            for (int k = 0; k < 3; ++k) {
                lo[k][cnt] = b.lo[k];
                hi[k][cnt] = b.hi[k];
            }
            ref[cnt++] = r;
        };
        const int2 c = child[i];
        const int32_t cs[2] = {c.x, c.y};
        const int32_t self = (int32_t)idx[i] + node_off;
        for (int sd = 0; sd < 2; ++sd) {
            const int32_t r = child_ref(cs[sd], range, leaf_off);
            if (r < 0) {
                add(box_tmp[2 * i + sd], r);
            } else {
                const int2 g = child[r];
                const int32_t gs[2] = {g.x, g.y};
                for (int t = 0; t < 2; ++t) {
                    const int32_t rg = child_ref(gs[t], range, leaf_off);
                    if (rg >= 0)  // row 7 of a child node: its parent and its slot here (the stackless walk)
                        nodes[8 * (size_t)idx[rg] + 7] = make_float4(__int_as_float(self), __int_as_float(cnt), 0.0f,
                                                                     0.0f);
                    add(box_tmp[2 * r + t], rg < 0 ? rg : (int32_t)idx[rg] + node_off);
                }
            }
        }
        for (; cnt < 4; ++cnt) {
            for (int k = 0; k < 3; ++k) {
                lo[k][cnt] = 0.0f;
                hi[k][cnt] = 0.0f;
            }
            ref[cnt] = kEmptyRef;
        }
        float4* o = nodes + 8 * (size_t)idx[i];
        for (int k = 0; k < 3; ++k) {
            o[2 * k] = make_float4(lo[k][0], lo[k][1], lo[k][2], lo[k][3]);
            o[2 * k + 1] = make_float4(hi[k][0], hi[k][1], hi[k][2], hi[k][3]);
        }
        o[6] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]),
                           __int_as_float(ref[3]));
        if (i == 0) o[7] = make_float4(__int_as_float(-1), 0.0f, 0.0f, 0.0f);  // the root has no parent
    }
}

__global__ void k_reorder(const float* V, const int32_t* T, int64_t nt, const uint32_t* sorted_tri, float4* tri_v) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nt; p += stride) {
        int64_t t = sorted_tri[p];
        const float* a = V + 3 * (int64_t)T[3 * t];
        const float* b = V + 3 * (int64_t)T[3 * t + 1];
        const float* c = V + 3 * (int64_t)T[3 * t + 2];
        tri_v[3 * p + 0] = make_float4(a[0], a[1], a[2], __int_as_float((int32_t)t));
        tri_v[3 * p + 1] = make_float4(b[0], b[1], b[2], 0.0f);
        tri_v[3 * p + 2] = make_float4(c[0], c[1], c[2], 0.0f);
    }
}

}  // namespace

static cudaError_t build_two_level(SceneDev& S, float pad_world, uint32_t* flags, cudaStream_t s);

cudaError_t scene_build(SceneDev& S, const CurvParamsDev& cp, cudaStream_t s, bool* mesh_error, std::string* msg,
                        bool refit, bool keep_curvature) {
    *mesh_error = false;
    refit = refit && (S.two_level ? S.tl_ready : S.bvh_ready);
    keep_curvature = keep_curvature && refit;
    const int64_t nv = S.n_verts, nt = S.n_tris;
    const float* V = ptr<float>(S.verts);
    const int32_t* T = ptr<int32_t>(S.tris);
    const int32_t* obj = ptr<int32_t>(S.tri_obj);
    // ---- scratch (freed at the end of the build)
    DevBuf flags, canon, keys, vals, sort_scr, cnt, off, cursor, adj, Gc, cmax, sumQ, Q, S64, nsu, bnd, boxes, visits,
        moff, wscan_scr, wtotal;
    auto cleanup = [&]() {
        for (DevBuf* b : {&flags, &canon, &keys, &vals, &sort_scr, &cnt, &off, &cursor, &adj, &Gc, &cmax, &sumQ, &Q,
                          &S64, &nsu, &bnd, &boxes, &visits, &moff, &wscan_scr, &wtotal})
            release(*b);
    };
    struct Guard {
        decltype(cleanup)& f;
        ~Guard() { f(); }
    } guard{cleanup};

    const int64_t nmax = std::max<int64_t>(std::max<int64_t>(nv, nt), 1);
    CK(grow(flags, 16));
    CK(cudaMemsetAsync(flags.p, 0, 16, s));
    note_launch();
    k_validate<<<grid_for(nv + nt, kB), kB, 0, s>>>(V, nv, T, nt, ptr<int32_t>(S.tri_mat), S.n_mat, obj,
                                                    ptr<uint32_t>(flags));
    CK(cudaGetLastError());
    uint32_t hflags = 0;
    CK(cudaMemcpyAsync(&hflags, flags.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hflags) {
        *mesh_error = true;
        *msg = (hflags & kFlagBadVertex) ? "non-finite vertex coordinate" : "triangle index, material or object out of range";
        return cudaSuccess;
    }
    // n_obj from the host copy is known by the caller (S.n_obj)
    const int32_t n_obj = S.n_obj;

    CK(grow(S.nrm, (size_t)nt * 3 * sizeof(float)));
    note_launch();
    k_normals<<<grid_for(nt, kB), kB, 0, s>>>(V, T, nt, ptr<float>(S.nrm));
    CK(cudaGetLastError());

    CK(grow(keys, (size_t)nmax * 8));
    CK(grow(vals, (size_t)nmax * 4));
    CK(grow(sort_scr, sort_scratch_bytes(nmax) + scan_scratch_bytes(nmax + n_obj + 1)));
    if (!keep_curvature) {
        // ---- weld
        CK(grow(canon, (size_t)nv * 4));
        CK(grow(keys, (size_t)nmax * 8));
        CK(grow(vals, (size_t)nmax * 4));
        CK(grow(sort_scr, sort_scratch_bytes(nmax) + scan_scratch_bytes(nmax + n_obj + 1)));
        note_launch();
        k_pos_keys<<<grid_for(nv, kB), kB, 0, s>>>(V, nv, ptr<uint64_t>(keys), ptr<uint32_t>(vals));
        CK(cudaGetLastError());
        CK(radix_sort_u64(ptr<uint64_t>(keys), ptr<uint32_t>(vals), nv, 64, sort_scr.p, s));
        note_launch();
        k_weld_runs<<<grid_for(nv, kB), kB, 0, s>>>(V, nv, ptr<uint64_t>(keys), ptr<uint32_t>(vals), ptr<int32_t>(canon));
        CK(cudaGetLastError());

        // ---- adjacency CSR over canonical vertices
        CK(grow(cnt, (size_t)(nv + 1) * 4));
        CK(grow(off, (size_t)(nv + 1) * 4));
        CK(grow(cursor, (size_t)(nv + 1) * 4));
        CK(grow(adj, (size_t)std::max<int64_t>(3 * nt, 1) * 4));
        CK(cudaMemsetAsync(cnt.p, 0, (size_t)(nv + 1) * 4, s));
        CK(cudaMemsetAsync(cursor.p, 0, (size_t)(nv + 1) * 4, s));
        note_launch();
        k_adj_count<<<grid_for(nt, kB), kB, 0, s>>>(ptr<int32_t>(canon), T, nt, ptr<uint32_t>(cnt));
        CK(cudaGetLastError());
        CK(exclusive_scan_u32(ptr<uint32_t>(cnt), ptr<uint32_t>(off), nv + 1, nullptr, sort_scr.p, s));
        note_launch();
        k_adj_fill<<<grid_for(nt, kB), kB, 0, s>>>(ptr<int32_t>(canon), T, nt, ptr<uint32_t>(off), ptr<uint32_t>(cursor),
                                                  ptr<int32_t>(adj));
        CK(cudaGetLastError());
        note_launch();
        k_adj_sort<<<grid_for(nv, kB), kB, 0, s>>>(nv, ptr<uint32_t>(off), ptr<int32_t>(adj));
        CK(cudaGetLastError());

        // ---- curvature and metric
        CK(grow(Gc, (size_t)nv * 4));
        CK(grow(S.G, (size_t)nv * 4));
        CK(grow(S.C, (size_t)nt * 4));
        note_launch();
        k_curvature<<<grid_for(nv, kB), kB, 0, s>>>(V, nv, T, ptr<int32_t>(canon), ptr<uint32_t>(off), ptr<int32_t>(adj),
                                                   ptr<float>(Gc));
        CK(cudaGetLastError());
        note_launch();
        k_expand_G<<<grid_for(nv, kB), kB, 0, s>>>(ptr<int32_t>(canon), nv, ptr<float>(Gc), ptr<float>(S.G));
        CK(cudaGetLastError());
        CK(grow(cmax, (size_t)(n_obj + 1) * 4));
        CK(cudaMemsetAsync(cmax.p, 0, (size_t)(n_obj + 1) * 4, s));
        note_launch();
        k_metric<<<grid_for(nt, kB), kB, 0, s>>>(V, T, nt, ptr<int32_t>(canon), ptr<float>(S.G), cp.eta, cp.area_ref,
                                                ptr<float>(S.C), ptr<uint32_t>(cmax), obj);
        CK(cudaGetLastError());

        // ---- per-mesh triangle lists (ascending), integer weights, CDFs
        CK(grow(moff, (size_t)(n_obj + 2) * 4));
        CK(cudaMemsetAsync(cnt.p, 0, (size_t)(n_obj + 1) * 4, s));
        CK(cudaMemsetAsync(cursor.p, 0, (size_t)(n_obj + 1) * 4, s));
        note_launch();
        k_mesh_count<<<grid_for(nt, kB), kB, 0, s>>>(obj, nt, ptr<uint32_t>(cnt));
        CK(cudaGetLastError());
        CK(exclusive_scan_u32(ptr<uint32_t>(cnt), ptr<uint32_t>(moff), n_obj + 1, nullptr, sort_scr.p, s));
        CK(grow(S.mesh_tris, (size_t)nt * 4));
        {
            // (mesh, triangle) keys sorted: triangles grouped by mesh, ascending inside a mesh
            int mesh_bits = 1;
            while ((1ll << mesh_bits) <= (int64_t)n_obj) ++mesh_bits;
            note_launch();
            k_mesh_keys<<<grid_for(nt, kB), kB, 0, s>>>(obj, nt, ptr<uint64_t>(keys), ptr<uint32_t>(vals));
            CK(cudaGetLastError());
            CK(radix_sort_u64(ptr<uint64_t>(keys), ptr<uint32_t>(vals), nt, 32 + mesh_bits, sort_scr.p, s));
            CK(cudaMemcpyAsync(S.mesh_tris.p, vals.p, (size_t)nt * 4, cudaMemcpyDeviceToDevice, s));
        }
        CK(grow(sumQ, (size_t)(n_obj + 1) * 8));
        CK(cudaMemsetAsync(sumQ.p, 0, (size_t)(n_obj + 1) * 8, s));
        CK(grow(Q, (size_t)nmax * 8));
        CK(grow(S64, (size_t)nmax * 8));
        note_launch();
        k_quantize<<<grid_for(nt, kB), kB, 0, s>>>(ptr<int32_t>(S.mesh_tris), nt, obj, ptr<float>(S.C), ptr<uint32_t>(cmax),
                                                  ptr<uint64_t>(Q), ptr<unsigned long long>(sumQ));
        CK(cudaGetLastError());
        note_launch();
        k_dither<<<grid_for(nt, kB), kB, 0, s>>>(ptr<int32_t>(S.mesh_tris), nt, obj, ptr<uint32_t>(moff),
                                                ptr<unsigned long long>(sumQ), cp.dither, cp.seed, ptr<uint64_t>(Q));
        CK(cudaGetLastError());
        CK(inclusive_scan_u64(ptr<uint64_t>(Q), ptr<uint64_t>(S64), nt, sort_scr.p, s));
        CK(grow(S.cdf, (size_t)nt * 8));
        note_launch();
        k_cdf_fix<<<grid_for(nt, kB), kB, 0, s>>>(ptr<uint64_t>(S64), nt, ptr<int32_t>(S.mesh_tris), obj,
                                                 ptr<uint32_t>(moff), ptr<uint64_t>(S.cdf));
        CK(cudaGetLastError());
        // mesh offsets as int64 for the sampling kernels
        CK(grow(S.mesh_off, (size_t)(n_obj + 1) * 8));
        {
            std::vector<uint32_t> h32(n_obj + 1);
            CK(cudaMemcpyAsync(h32.data(), moff.p, (size_t)(n_obj + 1) * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            std::vector<int64_t> h64(h32.begin(), h32.end());
            CK(cudaMemcpyAsync(S.mesh_off.p, h64.data(), (size_t)(n_obj + 1) * 8, cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));
        }
        // sample counts
        CK(grow(nsu, (size_t)(n_obj + 1) * 8));
        CK(cudaMemsetAsync(nsu.p, 0, (size_t)(n_obj + 1) * 8, s));
        note_launch();
        k_hc_vertices<<<grid_for(nv, kB), kB, 0, s>>>(nv, ptr<int32_t>(canon), ptr<uint32_t>(off), ptr<int32_t>(adj), obj,
                                                     ptr<float>(S.C), ptr<uint32_t>(cmax), cp.hc_frac,
                                                     cp.samples_per_vertex, ptr<unsigned long long>(nsu));
        CK(cudaGetLastError());
        CK(grow(S.n_samples, (size_t)(n_obj + 1) * 8));
        CK(grow(S.sample_off, (size_t)(n_obj + 1) * 8));
        note_launch();
        k_sample_counts<<<1, kScThreads, 0, s>>>(n_obj, ptr<uint32_t>(moff), ptr<uint64_t>(S.cdf), ptr<unsigned long long>(nsu),
                                        cp.budget, ptr<int64_t>(S.n_samples), ptr<int64_t>(S.sample_off));
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&S.total_samples, ptr<int64_t>(S.sample_off) + n_obj, 8, cudaMemcpyDeviceToHost, s));

    }  // !keep_curvature

    // ---- LBVH
    CK(grow(bnd, 64));
    {
        uint32_t init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
        CK(cudaMemcpyAsync(bnd.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
    }
    note_launch();
    k_bounds<<<grid_for(nv, kB, 152 * 4), kB, 0, s>>>(V, nv, ptr<uint32_t>(bnd));
    CK(cudaGetLastError());
    if (!refit && !S.two_level) {
        note_launch();
        k_morton<<<grid_for(nt, kB), kB, 0, s>>>(V, T, nt, ptr<uint32_t>(bnd), ptr<uint64_t>(keys), ptr<uint32_t>(vals));
        CK(cudaGetLastError());
        CK(radix_sort_u64(ptr<uint64_t>(keys), ptr<uint32_t>(vals), nt, 63, sort_scr.p, s));
        CK(grow(S.bvh_perm, (size_t)nt * 4));
        CK(cudaMemcpyAsync(S.bvh_perm.p, vals.p, (size_t)nt * 4, cudaMemcpyDeviceToDevice, s));
    }
    uint32_t hb[6];
    CK(cudaMemcpyAsync(hb, bnd.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    {
        double diag2 = 0;
        for (int k = 0; k < 3; ++k) {
            auto un = [](uint32_t u) {
                uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
                float f;
                memcpy(&f, &b, 4);
                return f;
            };
            S.bounds_lo[k] = un(hb[k]);
            S.bounds_hi[k] = un(hb[3 + k]);
            double e = (double)S.bounds_hi[k] - S.bounds_lo[k];
            diag2 += e * e;
        }
        const float pad = (float)(1e-5 * sqrt(diag2) + 1e-7);
        const int n = (int)nt;
        if (S.two_level) {
            // no hierarchy over the world triangles: the prototypes' BVHs and one over the instances
            for (DevBuf* b : {&S.tri_v, &S.bvh_child, &S.bvh_range, &S.bvh_par_i, &S.bvh_par_l, &S.bvh_perm,
                              &S.bvh_wflag, &S.bvh_widx})
                release(*b);
            S.bvh_ready = false;
            CK(build_two_level(S, pad, ptr<uint32_t>(flags), s));
        } else {
            S.tl_ready = false;
            CK(grow(S.tri_v, (size_t)nt * 3 * sizeof(float4)));
            note_launch();
            k_reorder<<<grid_for(nt, kB), kB, 0, s>>>(V, T, nt, ptr<uint32_t>(S.bvh_perm), ptr<float4>(S.tri_v));
            CK(cudaGetLastError());
            if (n == 1 || n <= kLeafMax) {
                CK(grow(S.nodes, 8 * sizeof(float4)));
                S.root = leaf_ref(0, n);
            } else {
                S.root = 0;
                int2* child_p = ptr<int2>(S.bvh_child);
                int2* range_p = ptr<int2>(S.bvh_range);
                if (!refit) {
                    CK(grow(S.bvh_child, (size_t)(n - 1) * sizeof(int2)));
                    CK(grow(S.bvh_range, (size_t)(n - 1) * sizeof(int2)));
                    CK(grow(S.bvh_par_i, (size_t)n * 4));
                    CK(grow(S.bvh_par_l, (size_t)n * 4));
                    child_p = ptr<int2>(S.bvh_child);
                    range_p = ptr<int2>(S.bvh_range);
                    note_launch();
                    k_karras<<<grid_for(n - 1, kB), kB, 0, s>>>(ptr<uint64_t>(keys), n, child_p, range_p,
                                                                ptr<int32_t>(S.bvh_par_i), ptr<int32_t>(S.bvh_par_l));
                    CK(cudaGetLastError());
                }
                CK(grow(boxes, (size_t)(n - 1) * 2 * sizeof(Box)));
                CK(grow(visits, (size_t)(n - 1) * 4));
                CK(cudaMemsetAsync(visits.p, 0, (size_t)(n - 1) * 4, s));
                note_launch();
                k_boxes<<<grid_for(n, kB), kB, 0, s>>>(TriLeafBox{V, T, ptr<uint32_t>(S.bvh_perm), pad}, n, child_p,
                                                       ptr<int32_t>(S.bvh_par_i), ptr<int32_t>(S.bvh_par_l),
                                                       ptr<Box>(boxes), ptr<uint32_t>(visits), ptr<uint32_t>(flags));
                CK(cudaGetLastError());
                if (!refit) {
                    // 4-wide BVH: flag the binary nodes that become wide nodes, number them
                    CK(grow(S.bvh_wflag, (size_t)(n - 1) * 4));
                    CK(grow(S.bvh_widx, (size_t)(n - 1) * 4));
                    CK(grow(wscan_scr, scan_scratch_bytes(n - 1)));
                    CK(grow(wtotal, 4));
                    note_launch();
                    k_wide_flags<<<grid_for(n - 1, kB), kB, 0, s>>>(n, range_p, ptr<int32_t>(S.bvh_par_i),
                                                                    ptr<uint32_t>(S.bvh_wflag), ptr<uint32_t>(flags));
                    CK(cudaGetLastError());
                    CK(exclusive_scan_u32(ptr<uint32_t>(S.bvh_wflag), ptr<uint32_t>(S.bvh_widx), n - 1,
                                          ptr<uint32_t>(wtotal), wscan_scr.p, s));
                    uint32_t n4 = 0;
                    CK(cudaMemcpyAsync(&n4, wtotal.p, 4, cudaMemcpyDeviceToHost, s));
                    CK(cudaStreamSynchronize(s));
                    CK(grow(S.nodes, (size_t)std::max<uint32_t>(n4, 1) * 8 * sizeof(float4)));
                    S.n_nodes = n4;
                }
                note_launch();
                k_pack_wide<<<grid_for(n - 1, kB), kB, 0, s>>>(n, child_p, range_p, ptr<Box>(boxes),
                                                               ptr<uint32_t>(S.bvh_wflag), ptr<uint32_t>(S.bvh_widx),
                                                               ptr<float4>(S.nodes), 0, 0);
                CK(cudaGetLastError());
            }
        }
    }
    CK(cudaMemcpyAsync(&hflags, flags.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hflags & kFlagBadTree) {
        *mesh_error = true;
        *msg = "LBVH construction produced a malformed hierarchy";
        return cudaSuccess;
    }
    if (hflags & kFlagBadVertex) {
        *mesh_error = true;
        *msg = "an instance map is singular or its inverse is not finite";
        return cudaSuccess;
    }
    S.built = true;
    S.bvh_ready = !S.two_level;
    S.tl_ready = S.two_level;
    return cudaSuccess;
}

// ------------------------------------------------------------------ instanced scenes
// Instance i of prototype iproto[i] owns world vertices vbase[i] .. vbase[i+1] and triangles tbase[i] ..
// tbase[i+1]; the instance of an element is found by binary search over the (ascending) bases.
namespace {

__device__ __forceinline__ int instance_of(const int64_t* base, int32_t n_inst, int64_t e) {
    int lo = 0, hi = n_inst - 1;  // largest i with base[i] <= e (base[0] = 0 <= e)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// x' = A x + b per instance, each component ((A_r0 x + A_r1 y) + A_r2 z) + b_r, every product and sum
// rounded to float32 in that order (this unit is compiled without contraction)
__global__ void k_inst_verts(const float* __restrict__ pv, const int64_t* __restrict__ pvoff,
                             const int32_t* __restrict__ iproto, const int64_t* __restrict__ vbase,
                             const float* __restrict__ xf, int32_t n_inst, int64_t nv, float* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        const int i = instance_of(vbase, n_inst, v);
        const int64_t src = pvoff[iproto[i]] + (v - vbase[i]);
        const float x = pv[3 * src], y = pv[3 * src + 1], z = pv[3 * src + 2];
        const float* a = xf + 12 * (int64_t)i;
#pragma unroll
        for (int r = 0; r < 3; ++r)
            out[3 * v + r] = affine_row(make_float4(a[4 * r], a[4 * r + 1], a[4 * r + 2], a[4 * r + 3]), x, y, z);
    }
}

__global__ void k_inst_tris(const int32_t* __restrict__ pt, const int32_t* __restrict__ pmat,
                            const int64_t* __restrict__ ptoff, const int32_t* __restrict__ iproto,
                            const int64_t* __restrict__ vbase, const int64_t* __restrict__ tbase, int32_t n_inst,
                            int64_t nt, int32_t* __restrict__ tris, int32_t* __restrict__ mat,
                            int32_t* __restrict__ obj) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = instance_of(tbase, n_inst, t);
        const int64_t src = ptoff[iproto[i]] + (t - tbase[i]);
        const int32_t off = (int32_t)vbase[i];
#pragma unroll
        for (int k = 0; k < 3; ++k) tris[3 * t + k] = pt[3 * src + k] + off;
        mat[t] = pmat[src];
        obj[t] = i;
    }
}

// Instance records of the two-level structure (8 float4 per instance): rows (A_r, b_r); rows of A^-1 computed
// in float64 and rounded, with |A^-1|_inf rounded up (w of row 0), the prototype's root reference (w of row 1)
// and the first world triangle (w of row 2); the world box of the prototype's vertex bounds pbox under the
// map, from float64 interval arithmetic rounded outwards, grown by the float32 rounding bound of a mapped
// vertex and by pad (w of the box's hi: 1 for a prototype without triangles, which the walk skips).  Also the
// box centre for the top level's Morton keys.  A singular map (or a non-finite inverse) sets kFlagBadVertex.
__global__ void k_inst_records(const float* __restrict__ xf, const int32_t* __restrict__ iproto,
                               const int64_t* __restrict__ tbase, const int64_t* __restrict__ ptoff, int32_t n_inst,
                               const float* __restrict__ pbox, const int32_t* __restrict__ proot, float pad,
                               float4* __restrict__ rec, float* __restrict__ cen, uint32_t* flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst; i += gridDim.x * blockDim.x) {
        const float* a = xf + 12 * (int64_t)i;
        double A[3][3], b[3];
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) A[r][k] = a[4 * r + k];
            b[r] = a[4 * r + 3];
        }
        const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1], c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2],
                     c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
        const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
        double inv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        bool ok = isfinite(det) && fabs(det) > 1e-300;
        if (ok) {
            const double id = 1.0 / det;
            inv[0][0] = c00 * id;
            inv[1][0] = c01 * id;
            inv[2][0] = c02 * id;
            inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
            inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
            inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
            inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
            inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
            inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
        }
        float fi[3][3];
        double ninv = 0.0;
        for (int r = 0; r < 3; ++r) {
            double row = 0.0;
            for (int k = 0; k < 3; ++k) {
                fi[r][k] = (float)inv[r][k];
                ok = ok && isfinite(fi[r][k]);
                row += fabs((double)fi[r][k]);
            }
            ninv = fmax(ninv, row);
        }
        if (!ok) atomicOr(flags, kFlagBadVertex);
        const int q = iproto[i];
        const bool empty = ptoff[q + 1] == ptoff[q];
        const float* pb = pbox + 6 * q;
        float lo[3], hi[3];
        for (int r = 0; r < 3; ++r) {
            double c = b[r], e = 0.0, mag = fabs(b[r]);
            for (int k = 0; k < 3; ++k) {
                const double l = pb[k], h = pb[3 + k];
                c += A[r][k] * (0.5 * (l + h));
                e += fabs(A[r][k]) * (0.5 * (h - l));
                mag += fabs(A[r][k]) * fmax(fabs(l), fabs(h));
            }
            const double slack = mag * 4.76837158203125e-07;  // 2^-21: six float32 roundings of the mapped vertex
            lo[r] = __fsub_rd(__double2float_rd(c - e - slack), pad);
            hi[r] = __fadd_ru(__double2float_ru(c + e + slack), pad);
        }
        float4* o = rec + 8 * (int64_t)i;
        for (int r = 0; r < 3; ++r) o[r] = make_float4(a[4 * r], a[4 * r + 1], a[4 * r + 2], a[4 * r + 3]);
        o[3] = make_float4(fi[0][0], fi[0][1], fi[0][2], __double2float_ru(ninv * (1.0 + 1e-6)));
        o[4] = make_float4(fi[1][0], fi[1][1], fi[1][2], __int_as_float(proot[q]));
        o[5] = make_float4(fi[2][0], fi[2][1], fi[2][2], __int_as_float((int32_t)tbase[i]));
        o[6] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        o[7] = make_float4(hi[0], hi[1], hi[2], empty ? 1.0f : 0.0f);
        for (int r = 0; r < 3; ++r) cen[3 * (int64_t)i + r] = 0.5f * lo[r] + 0.5f * hi[r];
    }
}

// Tighter world boxes: the bounds of each instance's expanded world vertices (the very vertices its
// triangles are tested with) grown by pad, intersected with the box from the map; one warp per instance.
__global__ void k_inst_world_boxes(const float* __restrict__ V, const int64_t* __restrict__ vbase, int32_t n_inst,
                                   float pad, float4* __restrict__ rec, float* __restrict__ cen) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_inst; i += warps) {
        float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
        for (int64_t v = vbase[i] + lane; v < vbase[i + 1]; v += 32)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], V[3 * v + k]);
                hi[k] = fmaxf(hi[k], V[3 * v + k]);
            }
        for (int o = 16; o > 0; o >>= 1)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        if (lane == 0 && vbase[i + 1] > vbase[i]) {
            float4* o = rec + 8 * i;
            const float4 l0 = o[6], h0 = o[7];
            const float4 l = make_float4(fmaxf(l0.x, __fsub_rd(lo[0], pad)), fmaxf(l0.y, __fsub_rd(lo[1], pad)),
                                         fmaxf(l0.z, __fsub_rd(lo[2], pad)), 0.0f);
            const float4 h = make_float4(fminf(h0.x, __fadd_ru(hi[0], pad)), fminf(h0.y, __fadd_ru(hi[1], pad)),
                                         fminf(h0.z, __fadd_ru(hi[2], pad)), h0.w);
            o[6] = l;
            o[7] = h;
            cen[3 * i] = 0.5f * l.x + 0.5f * h.x;
            cen[3 * i + 1] = 0.5f * l.y + 0.5f * h.y;
            cen[3 * i + 2] = 0.5f * l.z + 0.5f * h.z;
        }
    }
}

// top level of at most kLeafMax instances: one root node holding each instance as a leaf of its own
__global__ void k_tlas_small(const float4* __restrict__ rec, const int32_t* __restrict__ tinst, int32_t n,
                             float4* __restrict__ nodes) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float lo[3][4], hi[3][4];
    int32_t ref[4];
    for (int j = 0; j < 4; ++j) {
        const bool use = j < n;
        const float4 l = use ? rec[8 * (int64_t)tinst[j] + 6] : make_float4(0, 0, 0, 0);
        const float4 h = use ? rec[8 * (int64_t)tinst[j] + 7] : make_float4(0, 0, 0, 0);
        lo[0][j] = l.x, lo[1][j] = l.y, lo[2][j] = l.z;
        hi[0][j] = h.x, hi[1][j] = h.y, hi[2][j] = h.z;
        ref[j] = use ? leaf_ref(j, 1) : kEmptyRef;
    }
    for (int k = 0; k < 3; ++k) {
        nodes[2 * k] = make_float4(lo[k][0], lo[k][1], lo[k][2], lo[k][3]);
        nodes[2 * k + 1] = make_float4(hi[k][0], hi[k][1], hi[k][2], hi[k][3]);
    }
    nodes[6] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]),
                           __int_as_float(ref[3]));
    nodes[7] = make_float4(__int_as_float(-1), 0.0f, 0.0f, 0.0f);
}

}  // namespace

// Scratch of one 4-wide build over n primitives (binary topology, boxes, wide-node numbering).
struct WideScratch {
    DevBuf child, range, par_i, par_l, boxes, visits, wflag, widx, wscan, wtotal;
    ~WideScratch() {
        for (DevBuf* b : {&child, &range, &par_i, &par_l, &boxes, &visits, &wflag, &widx, &wscan, &wtotal}) release(*b);
    }
};

// 4-wide BVH over n > kLeafMax primitives whose Morton keys are sorted in keys (leaf p's box from leaf(p)):
// Karras topology, boxes bottom-up, the wide nodes written from nodes[node_off] on (at most node_cap nodes
// in all) with references offset by node_off and leaf codes by leaf_off; the node count in *n4.
template <class LeafBox>
static cudaError_t wide_from_sorted(int n, const uint64_t* keys, LeafBox leaf, float4* nodes, int64_t node_cap,
                                    int32_t node_off, int32_t leaf_off, uint32_t* flags, WideScratch& w,
                                    cudaStream_t s, int64_t* n4_out) {
    CK(grow(w.child, (size_t)(n - 1) * sizeof(int2)));
    CK(grow(w.range, (size_t)(n - 1) * sizeof(int2)));
    CK(grow(w.par_i, (size_t)n * 4));
    CK(grow(w.par_l, (size_t)n * 4));
    CK(grow(w.boxes, (size_t)(n - 1) * 2 * sizeof(Box)));
    CK(grow(w.visits, (size_t)(n - 1) * 4));
    CK(grow(w.wflag, (size_t)(n - 1) * 4));
    CK(grow(w.widx, (size_t)(n - 1) * 4));
    CK(grow(w.wscan, scan_scratch_bytes(n - 1)));
    CK(grow(w.wtotal, 4));
    note_launch();
    k_karras<<<grid_for(n - 1, kB), kB, 0, s>>>(keys, n, ptr<int2>(w.child), ptr<int2>(w.range), ptr<int32_t>(w.par_i),
                                                ptr<int32_t>(w.par_l));
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(w.visits.p, 0, (size_t)(n - 1) * 4, s));
    note_launch();
    k_boxes<<<grid_for(n, kB), kB, 0, s>>>(leaf, n, ptr<int2>(w.child), ptr<int32_t>(w.par_i), ptr<int32_t>(w.par_l),
                                           ptr<Box>(w.boxes), ptr<uint32_t>(w.visits), flags);
    CK(cudaGetLastError());
    note_launch();
    k_wide_flags<<<grid_for(n - 1, kB), kB, 0, s>>>(n, ptr<int2>(w.range), ptr<int32_t>(w.par_i),
                                                    ptr<uint32_t>(w.wflag), flags);
    CK(cudaGetLastError());
    CK(exclusive_scan_u32(ptr<uint32_t>(w.wflag), ptr<uint32_t>(w.widx), n - 1, ptr<uint32_t>(w.wtotal), w.wscan.p, s));
    uint32_t n4 = 0;
    CK(cudaMemcpyAsync(&n4, w.wtotal.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((int64_t)node_off + n4 > node_cap) return cudaErrorInvalidValue;  // cannot happen: n4 <= n - 1
    note_launch();
    k_pack_wide<<<grid_for(n - 1, kB), kB, 0, s>>>(n, ptr<int2>(w.child), ptr<int2>(w.range), ptr<Box>(w.boxes),
                                                   ptr<uint32_t>(w.wflag), ptr<uint32_t>(w.widx),
                                                   nodes + 8 * (int64_t)node_off, node_off, leaf_off);
    CK(cudaGetLastError());
    *n4_out = n4;
    return cudaSuccess;
}

// The two-level structure of an instanced scene: the prototypes' BVHs (object space, once), then the
// instance records and the top-level BVH over the instances' world boxes (every build and move).
static cudaError_t build_two_level(SceneDev& S, float pad_world, uint32_t* flags, cudaStream_t s) {
    const InstanceDev& I = *S.inst;
    const int32_t P = I.n_proto;
    int64_t nmax = std::max<int64_t>(I.n_inst, 1);
    for (int32_t q = 0; q < P; ++q) nmax = std::max(nmax, I.ptoff_h[q + 1] - I.ptoff_h[q]);
    DevBuf keys, vals, sort_scr, bnd, cen;
    struct Rel {
        DevBuf* b[5];
        ~Rel() {
            for (DevBuf* x : b) release(*x);
        }
    } rel{{&keys, &vals, &sort_scr, &bnd, &cen}};
    CK(grow(keys, (size_t)nmax * 8));
    CK(grow(vals, (size_t)nmax * 4));
    CK(grow(sort_scr, sort_scratch_bytes(nmax)));
    CK(grow(bnd, 64));
    WideScratch w;
    auto bounds = [&](const float* pts, int64_t n, float lo[3], float hi[3]) -> cudaError_t {
        const uint32_t init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
        CK(cudaMemcpyAsync(bnd.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
        note_launch();
        k_bounds<<<grid_for(n, kB, 152 * 4), kB, 0, s>>>(pts, n, ptr<uint32_t>(bnd));
        CK(cudaGetLastError());
        uint32_t hb[6];
        CK(cudaMemcpyAsync(hb, bnd.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int k = 0; k < 6; ++k) {
            const uint32_t u = hb[k], bits = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
            float f;
            memcpy(&f, &bits, 4);
            (k < 3 ? lo[k] : hi[k - 3]) = f;
        }
        return cudaSuccess;
    };
    if (!S.blas_ready) {
        int64_t cap = 1;
        for (int32_t q = 0; q < P; ++q) cap += std::max<int64_t>(I.ptoff_h[q + 1] - I.ptoff_h[q] - 1, 0);
        const int64_t pt = I.ptoff_h[P];
        CK(grow(S.blas_nodes, (size_t)cap * 8 * sizeof(float4)));
        CK(grow(S.blas_tri, (size_t)std::max<int64_t>(pt, 1) * 3 * sizeof(float4)));
        std::vector<int32_t> root(P, kEmptyRef);
        std::vector<float> box(6 * (size_t)P, 0.0f);
        int64_t node_off = 0;
        for (int32_t q = 0; q < P; ++q) {
            const int64_t nvq = I.pvoff_h[q + 1] - I.pvoff_h[q], ntq = I.ptoff_h[q + 1] - I.ptoff_h[q];
            if (ntq == 0 || nvq == 0) continue;
            const float* Vq = ptr<float>(I.pverts) + 3 * I.pvoff_h[q];
            const int32_t* Tq = ptr<int32_t>(I.ptris) + 3 * I.ptoff_h[q];
            float lo[3], hi[3];
            CK(bounds(Vq, nvq, lo, hi));
            double diag2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                box[6 * q + k] = lo[k];
                box[6 * q + 3 + k] = hi[k];
                diag2 += ((double)hi[k] - lo[k]) * ((double)hi[k] - lo[k]);
            }
            const float pad_q = (float)(1e-5 * sqrt(diag2) + 1e-7);
            note_launch();
            k_morton<<<grid_for(ntq, kB), kB, 0, s>>>(Vq, Tq, ntq, ptr<uint32_t>(bnd), ptr<uint64_t>(keys),
                                                      ptr<uint32_t>(vals));
            CK(cudaGetLastError());
            CK(radix_sort_u64(ptr<uint64_t>(keys), ptr<uint32_t>(vals), ntq, 63, sort_scr.p, s));
            note_launch();
            k_reorder<<<grid_for(ntq, kB), kB, 0, s>>>(Vq, Tq, ntq, ptr<uint32_t>(vals),
                                                       ptr<float4>(S.blas_tri) + 3 * I.ptoff_h[q]);
            CK(cudaGetLastError());
            if (ntq <= kLeafMax) {
                root[q] = leaf_ref((int)I.ptoff_h[q], (int)ntq);
            } else {
                int64_t n4 = 0;
                CK(wide_from_sorted((int)ntq, ptr<uint64_t>(keys), TriLeafBox{Vq, Tq, ptr<uint32_t>(vals), pad_q},
                                    ptr<float4>(S.blas_nodes), cap, (int32_t)node_off, (int32_t)I.ptoff_h[q], flags, w,
                                    s, &n4));
                root[q] = (int32_t)node_off;
                node_off += n4;
            }
        }
        S.blas_n_nodes = node_off;
        CK(grow(S.blas_root, (size_t)P * 4));
        CK(grow(S.proto_box, (size_t)P * 24));
        CK(cudaMemcpyAsync(S.blas_root.p, root.data(), (size_t)P * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(S.proto_box.p, box.data(), (size_t)P * 24, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));  // the host tables above go out of scope
        S.blas_ready = true;
    }
    // instance records and the top level
    const int32_t n = I.n_inst;
    CK(grow(S.inst_rec, (size_t)n * 8 * sizeof(float4)));
    CK(grow(S.tlas_inst, (size_t)n * 4));
    CK(grow(cen, (size_t)n * 12));
    note_launch();
    k_inst_records<<<grid_for(n, kB), kB, 0, s>>>(ptr<float>(I.xform), ptr<int32_t>(I.iproto), ptr<int64_t>(I.tbase),
                                                  ptr<int64_t>(I.ptoff), n, ptr<float>(S.proto_box),
                                                  ptr<int32_t>(S.blas_root), pad_world, ptr<float4>(S.inst_rec),
                                                  ptr<float>(cen), flags);
    CK(cudaGetLastError());
    note_launch();
    k_inst_world_boxes<<<grid_for((int64_t)n * 32, kB), kB, 0, s>>>(ptr<float>(S.verts), ptr<int64_t>(I.vbase), n,
                                                                     pad_world, ptr<float4>(S.inst_rec), ptr<float>(cen));
    CK(cudaGetLastError());
    float lo[3], hi[3];
    CK(bounds(ptr<float>(cen), n, lo, hi));
    note_launch();
    k_morton_pts<<<grid_for(n, kB), kB, 0, s>>>(ptr<float>(cen), n, ptr<uint32_t>(bnd), ptr<uint64_t>(keys),
                                                ptr<uint32_t>(vals));
    CK(cudaGetLastError());
    CK(radix_sort_u64(ptr<uint64_t>(keys), ptr<uint32_t>(vals), n, 63, sort_scr.p, s));
    CK(cudaMemcpyAsync(S.tlas_inst.p, vals.p, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    if (n <= kLeafMax) {
        if (S.nodes.cap > ((size_t)1 << 20)) release(S.nodes);
        CK(grow(S.nodes, 8 * sizeof(float4)));
        note_launch();
        k_tlas_small<<<1, 32, 0, s>>>(ptr<float4>(S.inst_rec), ptr<int32_t>(S.tlas_inst), n, ptr<float4>(S.nodes));
        CK(cudaGetLastError());
        S.n_nodes = 1;
    } else {
        const size_t need = (size_t)(n - 1) * 8 * sizeof(float4);
        if (S.nodes.cap > 4 * need + ((size_t)1 << 20)) release(S.nodes);  // a flat scene's hierarchy before
        CK(grow(S.nodes, need));
        int64_t n4 = 0;
        CK(wide_from_sorted(n, ptr<uint64_t>(keys), InstLeafBox{ptr<float4>(S.inst_rec), ptr<int32_t>(S.tlas_inst)},
                            ptr<float4>(S.nodes), n - 1, 0, 0, flags, w, s, &n4));
        S.n_nodes = n4;
    }
    S.root = 0;
    return cudaSuccess;
}

cudaError_t expand_instance_verts(const InstanceDev& I, const float* xf, float* out, cudaStream_t s) {
    if (I.nv == 0) return cudaSuccess;
    note_launch();
    k_inst_verts<<<grid_for(I.nv, kB), kB, 0, s>>>(ptr<float>(I.pverts), ptr<int64_t>(I.pvoff), ptr<int32_t>(I.iproto),
                                                   ptr<int64_t>(I.vbase), xf, I.n_inst, I.nv, out);
    return cudaGetLastError();
}

cudaError_t expand_instance_tris(const InstanceDev& I, int32_t* tris, int32_t* mat, int32_t* obj, cudaStream_t s) {
    if (I.nt == 0) return cudaSuccess;
    note_launch();
    k_inst_tris<<<grid_for(I.nt, kB), kB, 0, s>>>(ptr<int32_t>(I.ptris), ptr<int32_t>(I.pmat), ptr<int64_t>(I.ptoff),
                                                  ptr<int32_t>(I.iproto), ptr<int64_t>(I.vbase), ptr<int64_t>(I.tbase),
                                                  I.n_inst, I.nt, tris, mat, obj);
    return cudaGetLastError();
}

}  // namespace st
