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
#include "st_trace_dev.cuh"

namespace st {

namespace {

using namespace trv;

// One bounce of Algorithm 1 over the live-ray queue.
__global__ void __launch_bounds__(256, 4) k_bounce(const TraceArgs a, int j, int64_t n_first) {
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

// Sec. III-D: sample g of the global list -> mesh m, local index s; Philox(s, m, pose, 0) selects a
// triangle through the mesh's integer CDF and a barycentric point; then the filters.
__global__ void __launch_bounds__(128, 8) k_diffraction(const DiffArgs a) {
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
