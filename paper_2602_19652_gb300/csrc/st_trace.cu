// Ray tracing kernels (Algorithm 1, Sec. III-D filters, Sec. III-E visibility).
//
// Traversal (st_trace_dev.cuh): stack-based walk of the 4-wide BVH (128-byte nodes: the four children's
// boxes as six float4 rows and their references, seven 128-bit loads through the read-only path), the
// nearest hit child next and the others pushed farthest first with their entry distances, skipped on
// pop when a closer hit is known.  Boxes are padded at build time and the slab test widens the far
// distance, so a box is never rejected when the float32 triangle test would hit inside it; the closest
// hit is the smallest (t, triangle index), which makes the result independent of the tree's shape.
//
// Bounces run as a wavefront over a compacted queue of live rays, three launches per bounce: closest
// hits, shading (reflection, float64 path length, the record [ray][bounce], the next queue and the
// visibility queue), and the visibility rays (to the receiver reference point, or one per microphone
// with the per-microphone receiver test).  The traversal kernels are persistent with lane refill: a
// query advances one wide node or one leaf triangle per step, and a lane whose query has finished takes
// the next one from a warp-aggregated atomic counter while the other lanes of its warp continue.  In
// large scenes the visibility queue is sorted by the Morton code of the hit points first.  Results do not
// depend on the order: closest hits are the smallest (t, triangle index), visibility is the absence of
// any hit in the segment.
// Compiled with -fmad=false (see st_geom.cuh).
#include <algorithm>

#include "st_geom.cuh"
#include "st_internal.cuh"
#include "st_trace_dev.cuh"

namespace st {

namespace {

using namespace trv;

// the traversal view of a scene's arguments (flat, or two-level when `inst` is set)
template <class A>
__host__ __device__ __forceinline__ Trav trav_of(const A& a) {
    Trav T{a.nodes, a.tri_v, a.root, a.max_iter, a.visits, a.stack_limit, a.restarts, a.refill};
    T.bnodes = a.bnodes;
    T.btri = a.btri;
    T.inst = a.inst;
    T.tinst = a.tinst;
    for (int k = 0; k < 6; ++k) T.chk[k] = a.chk[k];
    return T;
}

// traversal kernels: eight 128-thread CTAs per SM (64 registers) on flat scenes, six on two-level ones
// (the object-space ray and the instance state take more registers)
#define ST_TRAV_BOUNDS __launch_bounds__(kTravBlock, TL ? 6 : 8)

// Closest hits of one bounce: item idx of the live-ray queue (the first bounce in direction order).
template <bool TL>
__global__ void ST_TRAV_BOUNDS k_closest(const TraceArgs a, int j, int64_t n_first) {
    const Trav T = trav_of(a);
    const int64_t n = (j == 0) ? n_first : (int64_t)*a.n_in;
    const unsigned full = 0xffffffffu;
    int2 stack[kStack];
    typename TravStateOf<TL>::type S;
    int64_t ray = -1;
    bool live = false, exhausted = false;
    while (true) {
        const bool need = !live && !exhausted;
        const int64_t idx = claim(a.ctr + 0, need);
        if (need) {
            if (idx < n) {
                ray = (j == 0) ? (a.perm ? (int64_t)a.perm[idx] : idx) : (int64_t)a.q_in[idx];
                f3 o, d;
                int32_t prev;
                if (j == 0) {
                    o = f3{a.s[0], a.s[1], a.s[2]};
                    d = rotate(a.q, f3{a.dirs[3 * ray], a.dirs[3 * ray + 1], a.dirs[3 * ray + 2]});
                    prev = -1;
                } else {
                    o = f3{a.ox[ray], a.oy[ray], a.oz[ray]};
                    d = f3{a.dx[ray], a.dy[ray], a.dz[ray]};
                    prev = a.prev[ray];
                }
                trav_init(S, T, o, d, prev, a.t_min, __int_as_float(0x7f800000));
                live = true;
            } else {
                exhausted = true;
            }
        }
        if (__ballot_sync(full, live) == 0u) break;
        while (true) {
            if (live && trav_step<false>(T, S, stack, a.flags)) {
                trav_count<false>(T, S);
                a.hit_tri[ray] = S.best;
                a.hit_t[ray] = S.tb;
                live = false;
            }
            const unsigned lv = __ballot_sync(full, live);
            const unsigned nd = __ballot_sync(full, !live && !exhausted);
            if (lv == 0u || __popc(nd) >= (T.refill > 0 ? T.refill : kRefillClosest)) break;
        }
    }
}

// Shading of one bounce: record, next queue, visibility queue (Algorithm 1's steps after the hit).
__global__ void k_shade(const TraceArgs a, int j, int64_t n_first) {
    const int64_t n_live = (j == 0) ? n_first : (int64_t)*a.n_in;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_live; idx += stride) {
        const int64_t ray = (j == 0) ? (a.perm ? (int64_t)a.perm[idx] : idx) : (int64_t)a.q_in[idx];
        warp_count(a.queries + 0);
        const int32_t tri = a.hit_tri[ray];
        if (tri < 0) continue;
        ST_CHECK_OR(tri < a.chk[5], a.flags, continue);
        const float t = a.hit_t[ray];
        f3 o, d;
        double r;
        if (j == 0) {
            o = f3{a.s[0], a.s[1], a.s[2]};
            d = rotate(a.q, f3{a.dirs[3 * ray], a.dirs[3 * ray + 1], a.dirs[3 * ray + 2]});
            r = 0.0;
        } else {
            o = f3{a.ox[ray], a.oy[ray], a.oz[ray]};
            d = f3{a.dx[ray], a.dy[ray], a.dz[ray]};
            r = a.racc[ray];
        }
        const float tdx = t * d.x, tdy = t * d.y, tdz = t * d.z;
        const f3 P{o.x + tdx, o.y + tdy, o.z + tdz};
        const f3 nv{a.nrm[3 * tri], a.nrm[3 * tri + 1], a.nrm[3 * tri + 2]};
        const float dn = dot(d, nv);
        const float k2 = 2.0f * dn;
        const float knx = k2 * nv.x, kny = k2 * nv.y, knz = k2 * nv.z;
        float len;
        const f3 dr = normalize(f3{d.x - knx, d.y - kny, d.z - knz}, &len);
        r = r + (double)t;
        const int64_t id = ray * a.B + j;
        a.rec_tri[id] = tri;
        a.rec_los[id] = 0;
        a.rec_r[id] = r;
        a.rec_p[3 * id] = P.x;
        a.rec_p[3 * id + 1] = P.y;
        a.rec_p[3 * id + 2] = P.z;
        a.rec_d[3 * id] = dr.x;
        a.rec_d[3 * id + 1] = dr.y;
        a.rec_d[3 * id + 2] = dr.z;
        const int lane = threadIdx.x & 31;
        if (a.rec_mask) {  // one visibility query per microphone (warp-aggregated append of M entries a lane)
            a.rec_mask[id] = 0ull;
            const unsigned active = __activemask();
            const int leader = __ffs(active) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(a.vis_n, (uint32_t)__popc(active) * (uint32_t)a.M);
            base = __shfl_sync(active, base, leader);
            const uint32_t q0 = base + (uint32_t)__popc(active & ((1u << lane) - 1u)) * (uint32_t)a.M;
            for (int m = 0; m < a.M; ++m) a.vis_q[q0 + m] = (uint32_t)id * (uint32_t)a.M + (uint32_t)m;
        } else {  // visibility query of this record (warp-aggregated append)
            const unsigned active = __activemask();
            const int leader = __ffs(active) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(a.vis_n, (uint32_t)__popc(active));
            base = __shfl_sync(active, base, leader);
            a.vis_q[base + __popc(active & ((1u << lane) - 1u))] = (uint32_t)id;
        }
        if (r < a.r_max && j + 1 < a.B) {
            a.ox[ray] = P.x;
            a.oy[ray] = P.y;
            a.oz[ray] = P.z;
            a.dx[ray] = dr.x;
            a.dy[ray] = dr.y;
            a.dz[ray] = dr.z;
            a.racc[ray] = r;
            a.prev[ray] = tri;
            const unsigned active = __activemask();
            const int leader = __ffs(active) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(a.n_out, (uint32_t)__popc(active));
            base = __shfl_sync(active, base, leader);
            a.q_out[base + __popc(active & ((1u << lane) - 1u))] = (uint32_t)ray;
        }
    }
}

// Visibility of `target` from the points of a queue (record or candidate ids): out[id] = 1 when no
// triangle other than excl[id] lies on the segment (t_min, |target - p| - eps).
// The target is tgt_dev[0..2] when given (the receiver reference point, written on the device), else (tx, ty, tz).
template <bool TL>
__global__ void ST_TRAV_BOUNDS k_visible(const Trav T, const uint32_t* queue, const uint32_t* count,
                                                           const float* pts, const int32_t* excl,
                                                           const float* tgt_dev, float tx, float ty, float tz,
                                                           float t_min, float eps, uint8_t* out,
                                                           unsigned long long* ctr, uint32_t* flags,
                                                           unsigned long long* queries) {
    const int64_t n = *count;
    const unsigned full = 0xffffffffu;
    const f3 target = tgt_dev ? f3{tgt_dev[0], tgt_dev[1], tgt_dev[2]} : f3{tx, ty, tz};
    int2 stack[kStack];
    typename TravStateOf<TL>::type S;
    int64_t id = -1;
    bool live = false, exhausted = false;
    while (true) {
        const bool need = !live && !exhausted;
        const int64_t idx = claim(ctr, need);
        if (need) {
            if (idx < n) {
                id = queue[idx];
                warp_count(queries + 1);
                const f3 o{pts[3 * id], pts[3 * id + 1], pts[3 * id + 2]};
                float L;
                const f3 u = normalize(sub(target, o), &L);
                const float tmax = L - eps;
                if (!(tmax > t_min)) {
                    out[id] = 1;
                } else {
                    trav_init(S, T, o, u, excl[id], t_min, tmax);
                    live = true;
                }
            } else {
                exhausted = true;
            }
        }
        const unsigned lv0 = __ballot_sync(full, live);
        const unsigned nd0 = __ballot_sync(full, !live && !exhausted);
        if (lv0 == 0u && nd0 == 0u) break;
        while (true) {
            if (live && trav_step<true>(T, S, stack, flags)) {
                trav_count<true>(T, S);
                out[id] = S.best < 0 ? 1 : 0;
                live = false;
            }
            const unsigned lv = __ballot_sync(full, live);
            const unsigned nd = __ballot_sync(full, !live && !exhausted);
            if (lv == 0u || __popc(nd) >= (T.refill > 0 ? T.refill : kRefillAny)) break;
        }
    }
}

// Per-microphone receiver test: query q of the queue is record q / M and microphone q % M; a visible
// microphone sets its bit of the record's mask (and the record's flag: some microphone sees it).
template <bool TL>
__global__ void ST_TRAV_BOUNDS k_visible_mics(const TraceArgs a, unsigned long long* ctr) {
    const Trav T = trav_of(a);
    const int64_t n = *a.vis_n;
    const unsigned full = 0xffffffffu;
    int2 stack[kStack];
    typename TravStateOf<TL>::type S;
    int64_t id = -1;
    int m = 0;
    bool live = false, exhausted = false;
    while (true) {
        const bool need = !live && !exhausted;
        const int64_t idx = claim(ctr, need);
        if (need) {
            if (idx < n) {
                const uint32_t q = a.vis_q[idx];
                id = (int64_t)(q / (uint32_t)a.M);
                m = (int)(q - (uint32_t)id * (uint32_t)a.M);
                warp_count(a.queries + 1);
                const f3 o{a.rec_p[3 * id], a.rec_p[3 * id + 1], a.rec_p[3 * id + 2]};
                const f3 target{a.mics[3 * m], a.mics[3 * m + 1], a.mics[3 * m + 2]};
                float L;
                const f3 u = normalize(sub(target, o), &L);
                const float tmax = L - a.los_eps;
                if (!(tmax > a.t_min)) {
                    atomicOr(reinterpret_cast<unsigned long long*>(&a.rec_mask[id]), 1ull << m);
                    a.rec_los[id] = 1;
                } else {
                    trav_init(S, T, o, u, a.rec_tri[id], a.t_min, tmax);
                    live = true;
                }
            } else {
                exhausted = true;
            }
        }
        const unsigned lv0 = __ballot_sync(full, live);
        const unsigned nd0 = __ballot_sync(full, !live && !exhausted);
        if (lv0 == 0u && nd0 == 0u) break;
        while (true) {
            if (live && trav_step<true>(T, S, stack, a.flags)) {
                trav_count<true>(T, S);
                if (S.best < 0) {
                    atomicOr(reinterpret_cast<unsigned long long*>(&a.rec_mask[id]), 1ull << m);
                    a.rec_los[id] = 1;
                }
                live = false;
            }
            const unsigned lv = __ballot_sync(full, live);
            const unsigned nd = __ballot_sync(full, !live && !exhausted);
            if (lv == 0u || __popc(nd) >= (T.refill > 0 ? T.refill : kRefillAny)) break;
        }
    }
}

// Sec. III-D: sample g of the global list -> mesh m, local index s; Philox(s, m, pose, 0) selects a
// triangle through the mesh's integer CDF and a barycentric point; then the field-of-view and
// incidence filters; the candidates that pass are queued for the line-of-sight test (k_visible).
__global__ void __launch_bounds__(128, 8) k_diffraction(const DiffArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const f3 s{a.s[0], a.s[1], a.s[2]};
    const f3 fwd{a.fwd[0], a.fwd[1], a.fwd[2]};
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.K; g += stride) {
        // mesh: last m with sample_off[m] <= g
        int lo = 0, hi = a.n_obj;  // sample_off has n_obj + 1 entries
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.sample_off[mid] <= g) lo = mid; else hi = mid;
        }
        const int m = lo;
        const int64_t sl = g - a.sample_off[m];
        uint32_t x[4];
        philox10((uint32_t)sl, (uint32_t)m, a.pose, 0u, a.seed, x);
        const int64_t b0 = a.mesh_off[m], b1 = a.mesh_off[m + 1];
        const uint64_t W = a.cdf[b1 - 1];
        const uint64_t u = ((uint64_t)x[0] << 32) | x[1];
        const uint64_t target = __umul64hi(u, W);
        int64_t l = b0, h = b1 - 1;
        while (l < h) {
            const int64_t mid = l + ((h - l) >> 1);
            if (a.cdf[mid] > target) h = mid; else l = mid + 1;
        }
        int32_t t = a.mesh_tris[l];
        ST_CHECK_OR(t >= 0 && t < a.chk[5], a.flags, t = 0);
        float ba = (float)(x[2] >> 8) * (1.0f / 16777216.0f);
        float bb = (float)(x[3] >> 8) * (1.0f / 16777216.0f);
        const float sum = ba + bb;
        if (sum > 1.0f) {
            ba = 1.0f - ba;
            bb = 1.0f - bb;
        }
        const float* v0 = a.verts + 3 * (int64_t)a.tris[3 * t];
        const float* v1 = a.verts + 3 * (int64_t)a.tris[3 * t + 1];
        const float* v2 = a.verts + 3 * (int64_t)a.tris[3 * t + 2];
        float p[3];
        for (int k = 0; k < 3; ++k) {
            const float e1 = v1[k] - v0[k];
            const float e2 = v2[k] - v0[k];
            const float p1 = ba * e1;
            const float p2 = bb * e2;
            const float qv = v0[k] + p1;
            p[k] = qv + p2;
        }
        const f3 o{p[0], p[1], p[2]};
        bool ok = true;
        if (a.cos_fov > -1.0f) {
            float L;
            const f3 wn = normalize(sub(o, s), &L);
            if (!(dot(fwd, wn) >= a.cos_fov)) ok = false;
        }
        if (ok) {
            float L;
            const f3 vn = normalize(sub(s, o), &L);
            const f3 n{a.nrm[3 * t], a.nrm[3 * t + 1], a.nrm[3 * t + 2]};
            if (!(fabsf(dot(n, vn)) >= a.cos_inc)) ok = false;
        }
        a.cand_tri[g] = t;
        a.cand_p[3 * g] = p[0];
        a.cand_p[3 * g + 1] = p[1];
        a.cand_p[3 * g + 2] = p[2];
        a.keep[g] = 0;  // set by the line-of-sight kernel for the candidates that passed the filters
        if (ok) {
            const unsigned active = __activemask();
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(active) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(a.los_n, (uint32_t)__popc(active));
            base = __shfl_sync(active, base, leader);
            a.los_q[base + __popc(active & ((1u << lane) - 1u))] = (uint32_t)g;
        }
    }
}

template <bool TL>
__global__ void k_direct(const DirectArgs a) {
    const Trav T = trav_of(a);
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.M) return;
    const f3 s{a.s[0], a.s[1], a.s[2]};
    const f3 mic{a.mics[3 * m], a.mics[3 * m + 1], a.mics[3 * m + 2]};
    warp_count(a.queries + 1);
    a.vis[m] = visible<TL>(T, s, mic, -1, a.t_min, a.los_eps, a.flags) ? 1 : 0;
}

// Receiver reference point: float64 sum of the microphones in order, divided by M, rounded.
__global__ void k_centroid(const float* mics, int32_t M, float* R) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < M; ++m)
        for (int k = 0; k < 3; ++k) acc[k] += (double)mics[3 * m + k];
    for (int k = 0; k < 3; ++k) R[k] = (float)(acc[k] / (double)M);
}

// 10 bits of x spread to every third bit
__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// Morton code (kVisBits per axis) of the hit point of every queued visibility query, 2^(3 kVisBits) past the
// count (10 bits measured faster than 5 or 7 on the vegetation workload, the sort included)
constexpr int kVisBits = 10;
__global__ void k_vis_keys(const TraceArgs a, uint64_t* keys) {
    const int64_t n = *a.vis_n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += stride) {
        uint64_t key = 1ull << (3 * kVisBits);
        if (c < n) {
            const int64_t id = a.vis_q[c];
            const float cells = (float)(1 << kVisBits);
            uint32_t m = 0;
            for (int k = 0; k < 3; ++k) {
                const float u = (a.rec_p[3 * id + k] - a.blo[k]) * a.bscale[k] * (cells * (1.0f / 1024.0f));
                m |= spread10((uint32_t)fminf(fmaxf(u, 0.0f), cells - 1.0f)) << (2 - k);
            }
            key = m;
        }
        keys[c] = key;
    }
}

// Morton code (kLosBits per axis) of the candidate point of every queued line-of-sight query
constexpr int kLosBits = 10;  // swept 0, 5, 10 bits: 10 fastest on the clutter workload (5 on vegetation)
__global__ void k_los_keys(const DiffArgs a, uint64_t* keys) {
    const int64_t n = *a.los_n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.K; c += stride) {
        uint64_t key = 1ull << (3 * kLosBits);
        if (c < n) {
            const int64_t g = a.los_q[c];
            const float cells = (float)(1 << kLosBits);
            uint32_t m = 0;
            for (int k = 0; k < 3; ++k) {
                const float u = (a.cand_p[3 * g + k] - a.blo[k]) * a.bscale[k] * (cells * (1.0f / 1024.0f));
                m |= spread10((uint32_t)fminf(fmaxf(u, 0.0f), cells - 1.0f)) << (2 - k);
            }
            key = m;
        }
        keys[c] = key;
    }
}

// Octahedral map of a direction to [0,1]^2, 16 bits per axis, Morton-interleaved: nearby directions
// get nearby keys, so sorting by the key groups rays that traverse the same part of the scene.
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__global__ void k_dir_keys(const float* dirs, int64_t n, uint64_t* keys, uint32_t* vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float x = dirs[3 * i], y = dirs[3 * i + 1], z = dirs[3 * i + 2];
        const float l1 = fabsf(x) + fabsf(y) + fabsf(z);
        float px = l1 > 0.0f ? x / l1 : 0.0f, py = l1 > 0.0f ? y / l1 : 0.0f;
        if (z < 0.0f) {
            const float qx = (1.0f - fabsf(py)) * (px >= 0.0f ? 1.0f : -1.0f);
            const float qy = (1.0f - fabsf(px)) * (py >= 0.0f ? 1.0f : -1.0f);
            px = qx;
            py = qy;
        }
        const uint32_t u = (uint32_t)fminf(fmaxf((px + 1.0f) * 32767.5f, 0.0f), 65535.0f);
        const uint32_t v = (uint32_t)fminf(fmaxf((py + 1.0f) * 32767.5f, 0.0f), 65535.0f);
        keys[i] = (uint64_t)((spread16(u) << 1) | spread16(v));
        vals[i] = (uint32_t)i;
    }
}

}  // namespace

cudaError_t direction_order(const float* dirs, int64_t n, uint64_t* keys, uint32_t* perm, void* scratch,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    note_launch();
    k_dir_keys<<<grid_for(n, 256), 256, 0, s>>>(dirs, n, keys, perm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return radix_sort_u64(keys, perm, n, 32, scratch, s);
}

// persistent traversal grid: one CTA per resident slot (eight per SM on flat scenes, six on two-level ones)
static unsigned trav_grid(int64_t n, bool tl) {
    const int64_t full = 152 * (tl ? 6 : 8);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(full, (n + kTravBlock - 1) / kTravBlock));
}

cudaError_t trace_rays(TraceArgs& a, cudaStream_t s, int block) {
    const unsigned grid = grid_for(a.N, block, 152 * 16);
    const Trav T = trav_of(a);
    const bool tl = a.inst != nullptr;
    for (int j = 0; j < a.B; ++j) {
        if (j > 0) {
            uint32_t* t = a.q_in;
            a.q_in = a.q_out;
            a.q_out = t;
            uint32_t* c = a.n_in;
            a.n_in = a.n_out;
            a.n_out = c;
        }
        cudaError_t e = cudaMemsetAsync(a.n_out, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.vis_n, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.ctr, 0, 2 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
        note_launch();
        if (tl)
            k_closest<true><<<trav_grid(a.N, true), kTravBlock, 0, s>>>(a, j, a.N);
        else
            k_closest<false><<<trav_grid(a.N, false), kTravBlock, 0, s>>>(a, j, a.N);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        note_launch();
        k_shade<<<grid, block, 0, s>>>(a, j, a.N);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (a.sort_keys) {  // stable sort: equal codes keep the queue order
            note_launch();
            k_vis_keys<<<grid_for(a.N, 256), 256, 0, s>>>(a, a.sort_keys);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = radix_sort_u64(a.sort_keys, a.vis_q, a.N, 3 * kVisBits + 1, a.sort_scr, s)) != cudaSuccess)
                return e;
        }
        note_launch();
        if (a.rec_mask && tl)
            k_visible_mics<true><<<trav_grid(a.N * a.M, true), kTravBlock, 0, s>>>(a, a.ctr + 1);
        else if (a.rec_mask)
            k_visible_mics<false><<<trav_grid(a.N * a.M, false), kTravBlock, 0, s>>>(a, a.ctr + 1);
        else
            (tl ? k_visible<true> : k_visible<false>)<<<trav_grid(a.N, tl), kTravBlock, 0, s>>>(
                T, a.vis_q, a.vis_n, a.rec_p, a.rec_tri, a.R, 0.0f, 0.0f, 0.0f, a.t_min, a.los_eps, a.rec_los,
                a.ctr + 1, a.flags, a.queries);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t diffraction_sample(DiffArgs& a, cudaStream_t s) {
    if (a.K <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.los_n, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.ctr, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_diffraction<<<grid_for(a.K, 128, 152 * 16), 128, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.sort_keys && kLosBits > 0) {  // stable: equal codes keep the queue order
        note_launch();
        k_los_keys<<<grid_for(a.K, 256), 256, 0, s>>>(a, a.sort_keys);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = radix_sort_u64(a.sort_keys, a.los_q, a.K, 3 * kLosBits + 1, a.sort_scr, s)) != cudaSuccess) return e;
    }
    const Trav T = trav_of(a);
    const bool tl = a.inst != nullptr;
    note_launch();
    (tl ? k_visible<true> : k_visible<false>)<<<trav_grid(a.K, tl), kTravBlock, 0, s>>>(
        T, a.los_q, a.los_n, a.cand_p, a.cand_tri, nullptr, a.s[0], a.s[1], a.s[2], a.t_min, a.los_eps, a.keep, a.ctr,
        a.flags, a.queries);
    return cudaGetLastError();
}

cudaError_t direct_visibility(DirectArgs& a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    note_launch();
    (a.inst ? k_direct<true> : k_direct<false>)<<<(a.M + 63) / 64, 64, 0, s>>>(a);
    return cudaGetLastError();
}

void mic_centroid_host_order(const float* mics_dev, int32_t M, float* R_dev, cudaStream_t s) {
    note_launch();
    k_centroid<<<1, 1, 0, s>>>(mics_dev, M, R_dev);
}

}  // namespace st
