// Ray tracing kernels (Algorithm 1, Sec. III-D filters, Sec. III-E visibility).
//
// Traversal: stack-based walk of the 64-byte two-child LBVH nodes (both child boxes and child
// references in four float4 loads through the read-only path), nearer child first, far child
// pushed with its entry distance so it is skipped on pop when a closer hit is known.  Boxes are
// padded at build time and the slab test widens the far distance, so a box is never rejected
// when the float32 triangle test would hit inside it; the closest hit is the smallest
// (t, triangle index), which makes the result independent of the tree's shape.
//
// Bounces run as a wavefront: one launch per bounce over a compacted queue of live rays; each
// thread finds the closest hit, reflects, accumulates the float64 path length, traces the
// visibility ray to the receiver reference point and writes the record [ray][bounce].
// Compiled with -fmad=false (see st_geom.cuh).
#include "st_geom.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

struct Trav {
    const float4* __restrict__ nodes;
    const float4* __restrict__ tri_v;
    int32_t root;
    int32_t max_iter;               // 2 * node count + 8: bound on loop iterations of one traversal
    unsigned long long* visits;     // optional [4]: nodes and triangles visited (closest, any-hit)
};

__device__ __forceinline__ float safe_inv(float d) {
    // a zero direction component becomes a huge finite slope so the slab test never forms 0 * inf
    const float big = 1e30f;
    if (fabsf(d) < 1e-30f) return d >= 0.0f ? big : -big;
    return 1.0f / d;
}

// slab test of one box over [tmin, tmax]: true when hit, entry distance in *tn.  tfar is widened
// by (1 + 2 gamma_3) (Ize, "Robust BVH ray traversal", JCGT 2013); boxes are padded as well.
__device__ __forceinline__ bool slab(float lx, float ly, float lz, float hx, float hy, float hz, f3 o, f3 inv,
                                     float tmin, float tmax, float* tn_out) {
    float t0x = (lx - o.x) * inv.x, t1x = (hx - o.x) * inv.x;
    float t0y = (ly - o.y) * inv.y, t1y = (hy - o.y) * inv.y;
    float t0z = (lz - o.z) * inv.z, t1z = (hz - o.z) * inv.z;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), tmin));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
    tf = tf * 1.0000004f;
    *tn_out = tn;
    return tn <= tf;
}

template <bool AnyHit>
__device__ __forceinline__ int32_t traverse(const Trav& T, f3 o, f3 d, int32_t exclude, float t_min, float t_max,
                                            float* t_out, uint32_t* flags) {
    const WRay wr = wray(o, d);
    const f3 inv{safe_inv(d.x), safe_inv(d.y), safe_inv(d.z)};
    int32_t best = -1;
    float tb = t_max;  // closest: +inf; any-hit: the segment end (exclusive)
    int2 stack[kStack];
    int sp = 0;
    int32_t ref = T.root;
    // every node of a proper tree is visited at most once: more iterations than nodes means a
    // malformed hierarchy, reported through the flags instead of looping
    int guard = T.max_iter;
    int n_nodes = 0, n_tris = 0;
    // the search interval for boxes: [-inf, tb]; t_min is enforced on triangles only
    while (true) {
        if (--guard < 0) {
            atomicOr(flags, kFlagBadTree);
            break;
        }
        if (ref >= 0) {
            const float4 a = __ldg(&T.nodes[4 * ref + 0]);
            const float4 b = __ldg(&T.nodes[4 * ref + 1]);
            const float4 c = __ldg(&T.nodes[4 * ref + 2]);
            const float4 e = __ldg(&T.nodes[4 * ref + 3]);
            ++n_nodes;
            // boxes are padded, so a box holding a hit at t > t_min >= 0 exits at t > 0 after rounding
            float tl, tr;
            const bool hl = slab(a.x, a.y, a.z, a.w, b.x, b.y, o, inv, 0.0f, tb, &tl);
            const bool hr = slab(b.z, b.w, c.x, c.y, c.z, c.w, o, inv, 0.0f, tb, &tr);
            const int32_t rl = __float_as_int(e.x), rr = __float_as_int(e.y);
            if (hl && hr) {
                const bool lfirst = tl <= tr;
                ref = lfirst ? rl : rr;
                if (sp < kStack) {
                    stack[sp++] = make_int2(lfirst ? rr : rl, __float_as_int(lfirst ? tr : tl));
                } else {
                    atomicOr(flags, kFlagStackOverflow);
                }
                continue;
            } else if (hl) {
                ref = rl;
                continue;
            } else if (hr) {
                ref = rr;
                continue;
            }
        } else {
            const int32_t code = ~ref;
            const int first = code >> 3, cnt = (code & 7) + 1;
            for (int i = first; i < first + cnt; ++i) {
                const float4 v0 = __ldg(&T.tri_v[3 * i + 0]);
                const int32_t id = __float_as_int(v0.w);
                if (id == exclude) continue;
                const float4 v1 = __ldg(&T.tri_v[3 * i + 1]);
                const float4 v2 = __ldg(&T.tri_v[3 * i + 2]);
                ++n_tris;
                float th;
                if (!wt_hit(wr, f3{v0.x, v0.y, v0.z}, f3{v1.x, v1.y, v1.z}, f3{v2.x, v2.y, v2.z}, &th)) continue;
                if (!(th > t_min)) continue;
                if (AnyHit) {
                    if (th < t_max) {
                        *t_out = th;
                        if (T.visits) {
                            atomicAdd(&T.visits[2], (unsigned long long)n_nodes);
                            atomicAdd(&T.visits[3], (unsigned long long)n_tris);
                        }
                        return id;
                    }
                } else if (th < tb || (th == tb && id < best)) {
                    tb = th;
                    best = id;
                }
            }
        }
        // pop, skipping entries whose box starts beyond the best hit
        bool found = false;
        while (sp > 0) {
            const int2 top = stack[--sp];
            if (__int_as_float(top.y) <= tb) {
                ref = top.x;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
    if (T.visits) {
        atomicAdd(&T.visits[AnyHit ? 2 : 0], (unsigned long long)n_nodes);
        atomicAdd(&T.visits[AnyHit ? 3 : 1], (unsigned long long)n_tris);
    }
    *t_out = tb;
    return best;
}

// Visibility of `target` from o: direction normalize(target - o), t in (t_min, |target - o| - eps).
__device__ __forceinline__ bool visible(const Trav& T, f3 o, f3 target, int32_t exclude, float t_min, float eps,
                                        uint32_t* flags) {
    float L;
    const f3 u = normalize(sub(target, o), &L);
    const float tmax = L - eps;
    if (!(tmax > t_min)) return true;
    float th;
    return traverse<true>(T, o, u, exclude, t_min, tmax, &th, flags) < 0;
}

// adds the number of active lanes to a 64-bit counter with one atomic per warp
__device__ __forceinline__ void warp_count(unsigned long long* ctr) {
    const unsigned m = __activemask();
    if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(ctr, (unsigned long long)__popc(m));
}

// One bounce of Algorithm 1 over the live-ray queue.
__global__ void __launch_bounds__(128) k_bounce(const TraceArgs a, int j, int64_t n_first) {
    const Trav T{a.nodes, a.tri_v, a.root, a.max_iter, a.visits};
    const int64_t n_live = (j == 0) ? n_first : (int64_t)*a.n_in;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const f3 R{a.R[0], a.R[1], a.R[2]};  // device copy written by k_centroid
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_live; idx += stride) {
        const int64_t ray = (j == 0) ? (a.perm ? (int64_t)a.perm[idx] : idx) : (int64_t)a.q_in[idx];
        f3 o, d;
        double r;
        int32_t prev;
        if (j == 0) {
            o = f3{a.s[0], a.s[1], a.s[2]};
            d = rotate(a.q, f3{a.dirs[3 * ray], a.dirs[3 * ray + 1], a.dirs[3 * ray + 2]});
            r = 0.0;
            prev = -1;
        } else {
            o = f3{a.ox[ray], a.oy[ray], a.oz[ray]};
            d = f3{a.dx[ray], a.dy[ray], a.dz[ray]};
            r = a.racc[ray];
            prev = a.prev[ray];
        }
        float t;
        const int32_t tri = traverse<false>(T, o, d, prev, a.t_min, __int_as_float(0x7f800000), &t, a.flags);
        warp_count(a.queries + 0);
        if (tri < 0) continue;
        warp_count(a.queries + 1);
        const float tdx = t * d.x, tdy = t * d.y, tdz = t * d.z;
        const f3 P{o.x + tdx, o.y + tdy, o.z + tdz};
        const f3 n{a.nrm[3 * tri], a.nrm[3 * tri + 1], a.nrm[3 * tri + 2]};
        const float dn = dot(d, n);
        const float k2 = 2.0f * dn;
        const float knx = k2 * n.x, kny = k2 * n.y, knz = k2 * n.z;
        float len;
        const f3 dr = normalize(f3{d.x - knx, d.y - kny, d.z - knz}, &len);
        r = r + (double)t;
        const bool vis = visible(T, P, R, tri, a.t_min, a.los_eps, a.flags);
        const int64_t id = ray * a.B + j;
        a.rec_tri[id] = tri;
        a.rec_los[id] = vis ? 1 : 0;
        a.rec_r[id] = r;
        a.rec_p[3 * id] = P.x;
        a.rec_p[3 * id + 1] = P.y;
        a.rec_p[3 * id + 2] = P.z;
        a.rec_d[3 * id] = dr.x;
        a.rec_d[3 * id + 1] = dr.y;
        a.rec_d[3 * id + 2] = dr.z;
        if (r < a.r_max && j + 1 < a.B) {
            a.ox[ray] = P.x;
            a.oy[ray] = P.y;
            a.oz[ray] = P.z;
            a.dx[ray] = dr.x;
            a.dy[ray] = dr.y;
            a.dz[ray] = dr.z;
            a.racc[ray] = r;
            a.prev[ray] = tri;
            // warp-aggregated append to the next queue
            const unsigned active = __activemask();
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(active) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(a.n_out, (uint32_t)__popc(active));
            base = __shfl_sync(active, base, leader);
            a.q_out[base + __popc(active & ((1u << lane) - 1u))] = (uint32_t)ray;
        }
    }
}

__device__ __forceinline__ void philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                                         uint32_t out[4]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
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

// Sec. III-D: sample g of the global list -> mesh m, local index s; Philox(s, m, pose, 0) selects a
// triangle through the mesh's integer CDF and a barycentric point; then the filters.
__global__ void __launch_bounds__(128) k_diffraction(const DiffArgs a) {
    const Trav T{a.nodes, a.tri_v, a.root, a.max_iter, a.visits};
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
        const int32_t t = a.mesh_tris[l];
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
        if (ok) {
            warp_count(a.queries + 1);
            ok = visible(T, o, s, t, a.t_min, a.los_eps, a.flags);
        }
        a.cand_tri[g] = t;
        a.cand_p[3 * g] = p[0];
        a.cand_p[3 * g + 1] = p[1];
        a.cand_p[3 * g + 2] = p[2];
        a.keep[g] = ok ? 1 : 0;
    }
}

__global__ void k_direct(const DirectArgs a) {
    const Trav T{a.nodes, a.tri_v, a.root, a.max_iter, a.visits};
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.M) return;
    const f3 s{a.s[0], a.s[1], a.s[2]};
    const f3 mic{a.mics[3 * m], a.mics[3 * m + 1], a.mics[3 * m + 2]};
    warp_count(a.queries + 1);
    a.vis[m] = visible(T, s, mic, -1, a.t_min, a.los_eps, a.flags) ? 1 : 0;
}

// Receiver reference point: float64 sum of the microphones in order, divided by M, rounded.
__global__ void k_centroid(const float* mics, int32_t M, float* R) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < M; ++m)
        for (int k = 0; k < 3; ++k) acc[k] += (double)mics[3 * m + k];
    for (int k = 0; k < 3; ++k) R[k] = (float)(acc[k] / (double)M);
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

cudaError_t trace_rays(TraceArgs& a, cudaStream_t s, int block) {
    const unsigned grid = grid_for(a.N, block, 152 * 16);
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
        if (e != cudaSuccess) return e;
        note_launch();
        k_bounce<<<grid, block, 0, s>>>(a, j, a.N);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t diffraction_sample(DiffArgs& a, cudaStream_t s) {
    if (a.K <= 0) return cudaSuccess;
    note_launch();
    k_diffraction<<<grid_for(a.K, 128, 152 * 16), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t direct_visibility(DirectArgs& a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    note_launch();
    k_direct<<<(a.M + 63) / 64, 64, 0, s>>>(a);
    return cudaGetLastError();
}

void mic_centroid_host_order(const float* mics_dev, int32_t M, float* R_dev, cudaStream_t s) {
    note_launch();
    k_centroid<<<1, 1, 0, s>>>(mics_dev, M, R_dev);
}

}  // namespace st
