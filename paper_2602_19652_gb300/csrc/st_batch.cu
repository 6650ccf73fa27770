// Batched form: many sensor poses over one or more scenes in one launch per stage.
//
// A job table in device memory describes every pose (scene arrays, sensor inputs read from the
// caller's device memory, offsets into the batch's global arrays).  Every stage runs over the union of
// all jobs' work items, each item finding its job by binary search over the jobs' offsets: ray
// generation with the first bounce, per bounce level a closest-hit, a shading and a visibility launch
// over one live-ray queue across jobs (the traversal launches persistent with lane refill, each lane
// traversing its own job's scene), diffraction sampling and filters with a queued line-of-sight launch,
// direct visibility, path gathering and direct spectra.  Poses are read from device memory at run time,
// so a captured CUDA graph of the batch can be replayed after the caller updates them in place.
// Compiled with -fmad=false like the single-pose tracing kernels (same float32 steps, so the batched
// path sets equal the single-pose ones).
#include <algorithm>

#include "st_geom.cuh"
#include "st_internal.cuh"
#include "st_trace_dev.cuh"

namespace st {

namespace {

using namespace trv;

// a job's scene as the traversal sees it
__device__ __forceinline__ Trav job_trav(const JobDev& b, const BatchArgs& a) {
    Trav T{b.nodes, b.tri_v, b.root, b.max_iter, nullptr, a.stack_limit};
    T.chk[0] = b.chk_nodes;
    T.chk[1] = b.chk_tris;
    T.chk[5] = b.chk_tris;
    return T;
}

// per job: receiver reference point (float64 sum of the microphones in order / M) and forward axis
__global__ void k_batch_prep(const JobDev* J, int n_jobs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_jobs) return;
    const JobDev& b = J[j];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < b.M; ++m)
        for (int k = 0; k < 3; ++k) acc[k] += (double)b.mics[3 * m + k];
    for (int k = 0; k < 3; ++k) b.R[k] = (float)(acc[k] / (double)b.M);
    const float q[4] = {b.q[0], b.q[1], b.q[2], b.q[3]};
    const f3 f = rotate(q, f3{1.0f, 0.0f, 0.0f});
    b.fwd[0] = f.x;
    b.fwd[1] = f.y;
    b.fwd[2] = f.z;
}

// Global ray id of item idx of bounce j's live queue: the first bounce walks each job's rays in its
// direction order.
__device__ __forceinline__ int64_t batch_ray(const BatchArgs& a, int j, int64_t idx, int* job_out) {
    int64_t g = (j == 0) ? idx : (int64_t)a.q_in[idx];
    const int job = find_job(a.ray_offs, a.n_jobs, g);
    if (j == 0) {
        const JobDev& b = a.jobs[job];
        if (b.perm) g = b.ray_off + (int64_t)b.perm[g - b.ray_off];
    }
    *job_out = job;
    return g;
}

// Closest hits of bounce j over the live rays of every job (Algorithm 1), persistent with lane refill:
// each lane traverses its own job's scene.
__global__ void __launch_bounds__(kTravBlock, 8) k_closest_batch(const BatchArgs a, int j, int64_t n_first) {
    const int64_t n = (j == 0) ? n_first : (int64_t)*a.n_in;
    const unsigned full = 0xffffffffu;
    int2 stack[kStack];
    TravState S;
    Trav T{nullptr, nullptr, 0, 0, nullptr};
    int64_t g = -1;
    bool live = false, exhausted = false;
    while (true) {
        const bool need = !live && !exhausted;
        const int64_t idx = claim(a.ctr + 0, need);
        if (need) {
            if (idx < n) {
                int job;
                g = batch_ray(a, j, idx, &job);
                const JobDev& b = a.jobs[job];
                if (j < b.B) {
                    T = job_trav(b, a);
                    f3 o, d;
                    int32_t prev;
                    if (j == 0) {
                        const int64_t local = g - b.ray_off;
                        const float q[4] = {b.q[0], b.q[1], b.q[2], b.q[3]};
                        o = f3{b.s[0], b.s[1], b.s[2]};
                        d = rotate(q, f3{b.dirs[3 * local], b.dirs[3 * local + 1], b.dirs[3 * local + 2]});
                        prev = -1;
                    } else {
                        o = f3{a.ox[g], a.oy[g], a.oz[g]};
                        d = f3{a.dx[g], a.dy[g], a.dz[g]};
                        prev = a.prev[g];
                    }
                    trav_init(S, T, o, d, prev, a.t_min, __int_as_float(0x7f800000));
                    live = true;
                } else {
                    a.hit_tri[g] = -1;
                }
            } else {
                exhausted = true;
            }
        }
        const unsigned lv0 = __ballot_sync(full, live);
        const unsigned nd0 = __ballot_sync(full, !live && !exhausted);
        if (lv0 == 0u && nd0 == 0u) break;
        while (true) {
            if (live && trav_step<false>(T, S, stack, a.flags)) {
                a.hit_tri[g] = S.best;
                a.hit_t[g] = S.tb;
                live = false;
            }
            const unsigned lv = __ballot_sync(full, live);
            const unsigned nd = __ballot_sync(full, !live && !exhausted);
            if (lv == 0u || __popc(nd) >= (a.refill > 0 ? a.refill : kRefillClosest)) break;
        }
    }
}

// Shading of bounce j over every job: the record [job][ray][bounce], the next live queue and the queue
// of records whose visibility to their job's receiver reference point is to be tested.
__global__ void k_shade_batch(const BatchArgs a, int j, int64_t n_first) {
    const int64_t n_live = (j == 0) ? n_first : (int64_t)*a.n_in;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_live; idx += stride) {
        int job;
        const int64_t g = batch_ray(a, j, idx, &job);
        const JobDev& b = a.jobs[job];
        if (j >= b.B) continue;
        warp_count(a.queries + 0);
        const int32_t tri = a.hit_tri[g];
        if (tri < 0) continue;
        ST_CHECK_OR(tri < b.chk_tris, a.flags, continue);
        warp_count(a.queries + 1);
        const float t = a.hit_t[g];
        const int64_t local = g - b.ray_off;
        f3 o, d;
        double r;
        if (j == 0) {
            const float q[4] = {b.q[0], b.q[1], b.q[2], b.q[3]};
            o = f3{b.s[0], b.s[1], b.s[2]};
            d = rotate(q, f3{b.dirs[3 * local], b.dirs[3 * local + 1], b.dirs[3 * local + 2]});
            r = 0.0;
        } else {
            o = f3{a.ox[g], a.oy[g], a.oz[g]};
            d = f3{a.dx[g], a.dy[g], a.dz[g]};
            r = a.racc[g];
        }
        const float tdx = t * d.x, tdy = t * d.y, tdz = t * d.z;
        const f3 P{o.x + tdx, o.y + tdy, o.z + tdz};
        const f3 nv{b.nrm[3 * tri], b.nrm[3 * tri + 1], b.nrm[3 * tri + 2]};
        const float dn = dot(d, nv);
        const float k2 = 2.0f * dn;
        const float knx = k2 * nv.x, kny = k2 * nv.y, knz = k2 * nv.z;
        float len;
        const f3 dr = normalize(f3{d.x - knx, d.y - kny, d.z - knz}, &len);
        r = r + (double)t;
        const int64_t id = b.rec_off + local * b.B + j;
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
        if (a.rec_mask) {  // one visibility query per microphone of the job (M <= 64)
            a.rec_mask[id] = 0ull;
            const uint32_t base = atomicAdd(a.vis_n, (uint32_t)b.M);
            for (int m = 0; m < b.M; ++m) a.vis_qm[base + m] = ((uint64_t)id << 6) | (uint64_t)m;
        } else {
            const unsigned active = __activemask();
            const int leader = __ffs(active) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(a.vis_n, (uint32_t)__popc(active));
            base = __shfl_sync(active, base, leader);
            a.vis_q[base + __popc(active & ((1u << lane) - 1u))] = (uint32_t)id;
        }
        if (r < a.r_max && j + 1 < b.B) {
            a.ox[g] = P.x;
            a.oy[g] = P.y;
            a.oz[g] = P.z;
            a.dx[g] = dr.x;
            a.dy[g] = dr.y;
            a.dz[g] = dr.z;
            a.racc[g] = r;
            a.prev[g] = tri;
            const unsigned active = __activemask();
            const int leader = __ffs(active) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(a.n_out, (uint32_t)__popc(active));
            base = __shfl_sync(active, base, leader);
            a.q_out[base + __popc(active & ((1u << lane) - 1u))] = (uint32_t)g;
        }
    }
}

// Visibility over a queue of global ids (records or diffraction candidates) of every job: out[id] = 1
// when no triangle other than excl[id] lies on the segment from pts[id] towards the job's receiver
// reference point (to_emitter = 0) or its emitter (to_emitter = 1), ending los_eps short of it.
__global__ void __launch_bounds__(kTravBlock, 8) k_visible_batch(const BatchArgs a, const uint32_t* queue,
                                                                 const uint32_t* count, const int64_t* offs,
                                                                 const float* pts, const int32_t* excl, int to_emitter,
                                                                 uint8_t* out, unsigned long long* ctr) {
    const int64_t n = *count;
    const unsigned full = 0xffffffffu;
    int2 stack[kStack];
    TravState S;
    Trav T{nullptr, nullptr, 0, 0, nullptr};
    int64_t id = -1;
    bool live = false, exhausted = false;
    while (true) {
        const bool need = !live && !exhausted;
        const int64_t idx = claim(ctr, need);
        if (need) {
            if (idx < n) {
                id = queue[idx];
                const JobDev& b = a.jobs[find_job(offs, a.n_jobs, id)];
                const float* tp = to_emitter ? b.s : b.R;
                const f3 target{tp[0], tp[1], tp[2]};
                const f3 o{pts[3 * id], pts[3 * id + 1], pts[3 * id + 2]};
                float L;
                const f3 u = normalize(sub(target, o), &L);
                const float tmax = L - a.los_eps;
                if (!(tmax > a.t_min)) {
                    out[id] = 1;
                } else {
                    T = job_trav(b, a);
                    trav_init(S, T, o, u, excl[id], a.t_min, tmax);
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
                out[id] = S.best < 0 ? 1 : 0;
                live = false;
            }
            const unsigned lv = __ballot_sync(full, live);
            const unsigned nd = __ballot_sync(full, !live && !exhausted);
            if (lv == 0u || __popc(nd) >= (a.refill > 0 ? a.refill : kRefillAny)) break;
        }
    }
}

// Per-microphone receiver test of every job: entry (record << 6 | m) of the queue tests the segment from the
// record's hit point towards microphone m of its job (the single-pose kernel's float32 steps) and sets bit
// m of the record's mask, and its visibility flag, when nothing but the record's own triangle lies on it.
__global__ void __launch_bounds__(kTravBlock, 8) k_visible_mics_batch(const BatchArgs a, unsigned long long* ctr) {
    const int64_t n = *a.vis_n;
    const unsigned full = 0xffffffffu;
    int2 stack[kStack];
    TravState S;
    Trav T{nullptr, nullptr, 0, 0, nullptr};
    int64_t id = -1;
    int m = 0;
    bool live = false, exhausted = false;
    while (true) {
        const bool need = !live && !exhausted;
        const int64_t idx = claim(ctr, need);
        if (need) {
            if (idx < n) {
                const uint64_t e = a.vis_qm[idx];
                id = (int64_t)(e >> 6);
                m = (int)(e & 63u);
                const JobDev& b = a.jobs[find_job(a.rec_offs, a.n_jobs, id)];
                const f3 o{a.rec_p[3 * id], a.rec_p[3 * id + 1], a.rec_p[3 * id + 2]};
                const f3 target{b.mics[3 * m], b.mics[3 * m + 1], b.mics[3 * m + 2]};
                float L;
                const f3 u = normalize(sub(target, o), &L);
                const float tmax = L - a.los_eps;
                if (!(tmax > a.t_min)) {
                    atomicOr(reinterpret_cast<unsigned long long*>(&a.rec_mask[id]), 1ull << m);
                    a.rec_los[id] = 1;
                } else {
                    T = job_trav(b, a);
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
                if (S.best < 0) {
                    atomicOr(reinterpret_cast<unsigned long long*>(&a.rec_mask[id]), 1ull << m);
                    a.rec_los[id] = 1;
                }
                live = false;
            }
            const unsigned lv = __ballot_sync(full, live);
            const unsigned nd = __ballot_sync(full, !live && !exhausted);
            if (lv == 0u || __popc(nd) >= (a.refill > 0 ? a.refill : kRefillAny)) break;
        }
    }
}

// diffraction samples of every job (global sample index), same steps as the single-pose kernel; the
// candidates that pass the filters are queued for the line-of-sight test (k_visible_batch)
__global__ void __launch_bounds__(128, 8) k_diffraction_batch(const BatchArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.K_total; g += stride) {
        const int job = find_job(a.samp_offs, a.n_jobs, g);
        const JobDev& b = a.jobs[job];
        const int64_t gl = g - b.samp_off;
        int lo = 0, hi = b.n_obj;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (b.sample_off[mid] <= gl) lo = mid; else hi = mid;
        }
        const int m = lo;
        const int64_t sl = gl - b.sample_off[m];
        uint32_t x[4];
        philox10((uint32_t)sl, (uint32_t)m, b.pose, 0u, a.seed, x);
        const int64_t b0 = b.mesh_off[m], b1 = b.mesh_off[m + 1];
        const uint64_t W = b.cdf[b1 - 1];
        const uint64_t u = ((uint64_t)x[0] << 32) | x[1];
        const uint64_t target = __umul64hi(u, W);
        int64_t l = b0, h = b1 - 1;
        while (l < h) {
            const int64_t mid = l + ((h - l) >> 1);
            if (b.cdf[mid] > target) h = mid; else l = mid + 1;
        }
        int32_t t = b.mesh_tris[l];
        ST_CHECK_OR(t >= 0 && t < b.chk_tris, a.flags, t = 0);
        float ba = (float)(x[2] >> 8) * (1.0f / 16777216.0f);
        float bb = (float)(x[3] >> 8) * (1.0f / 16777216.0f);
        const float sum = ba + bb;
        if (sum > 1.0f) {
            ba = 1.0f - ba;
            bb = 1.0f - bb;
        }
        const float* v0 = b.verts + 3 * (int64_t)b.tris[3 * t];
        const float* v1 = b.verts + 3 * (int64_t)b.tris[3 * t + 1];
        const float* v2 = b.verts + 3 * (int64_t)b.tris[3 * t + 2];
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
        const f3 s{b.s[0], b.s[1], b.s[2]};
        bool ok = true;
        if (b.cos_fov > -1.0f) {
            float L;
            const f3 wn = normalize(sub(o, s), &L);
            if (!(dot(f3{b.fwd[0], b.fwd[1], b.fwd[2]}, wn) >= b.cos_fov)) ok = false;
        }
        if (ok) {
            float L;
            const f3 vn = normalize(sub(s, o), &L);
            const f3 n{b.nrm[3 * t], b.nrm[3 * t + 1], b.nrm[3 * t + 2]};
            if (!(fabsf(dot(n, vn)) >= a.cos_inc)) ok = false;
        }
        a.cand_tri[g] = t;
        a.cand_p[3 * g] = p[0];
        a.cand_p[3 * g + 1] = p[1];
        a.cand_p[3 * g + 2] = p[2];
        a.keep[g] = 0;  // set by the line-of-sight kernel for the candidates that passed the filters
        if (ok) {
            warp_count(a.queries + 1);
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

__global__ void k_direct_batch(const BatchArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.M_total; g += stride) {
        const int job = find_job(a.mic_offs, a.n_jobs, g);
        const JobDev& b = a.jobs[job];
        const int m = (int)(g - b.mic_off);
        const Trav T = job_trav(b, a);
        warp_count(a.queries + 1);
        a.dvis[g] = visible(T, f3{b.s[0], b.s[1], b.s[2]}, f3{b.mics[3 * m], b.mics[3 * m + 1], b.mics[3 * m + 2]},
                            -1, a.t_min, a.los_eps, a.flags)
                        ? 1
                        : 0;
    }
}

// per job: first compacted entry and count of its visible records and kept candidates
__global__ void k_batch_ranges(const BatchArgs a, const uint32_t* scan_rec, const uint32_t* total_rec,
                               const uint32_t* scan_cand, const uint32_t* total_cand) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n_jobs) return;
    const int64_t r0 = a.rec_offs[j], r1 = a.rec_offs[j + 1];
    const uint32_t sb = r0 < a.R_total ? scan_rec[r0] : *total_rec;
    const uint32_t se = r1 < a.R_total ? scan_rec[r1] : *total_rec;
    a.ranges[4 * j + 0] = sb;
    a.ranges[4 * j + 1] = se - sb;
    if (a.K_total > 0) {
        const int64_t c0 = a.samp_offs[j], c1 = a.samp_offs[j + 1];
        const uint32_t cb = c0 < a.K_total ? scan_cand[c0] : *total_cand;
        const uint32_t ce = c1 < a.K_total ? scan_cand[c1] : *total_cand;
        a.ranges[4 * j + 2] = cb;
        a.ranges[4 * j + 3] = ce - cb;
    } else {
        a.ranges[4 * j + 2] = 0;
        a.ranges[4 * j + 3] = 0;
    }
}

}  // namespace

cudaError_t batch_prep(const JobDev* jobs, int n_jobs, cudaStream_t s) {
    note_launch();
    k_batch_prep<<<(n_jobs + 63) / 64, 64, 0, s>>>(jobs, n_jobs);
    return cudaGetLastError();
}

// persistent traversal grid: eight 128-thread CTAs per SM (64 registers)
static unsigned trav_grid(int64_t n) {
    const int64_t full = 152 * 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(full, (n + kTravBlock - 1) / kTravBlock));
}

cudaError_t batch_trace(BatchArgs& a, int max_b, int64_t n_total, int block, cudaStream_t s) {
    const unsigned grid = grid_for(n_total, block, 152 * 16);
    for (int j = 0; j < max_b; ++j) {
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
        k_closest_batch<<<trav_grid(n_total), kTravBlock, 0, s>>>(a, j, n_total);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        note_launch();
        k_shade_batch<<<grid, block, 0, s>>>(a, j, n_total);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        note_launch();
        if (a.rec_mask)
            k_visible_mics_batch<<<trav_grid(a.Q_total), kTravBlock, 0, s>>>(a, a.ctr + 1);
        else
            k_visible_batch<<<trav_grid(n_total), kTravBlock, 0, s>>>(a, a.vis_q, a.vis_n, a.rec_offs, a.rec_p,
                                                                      a.rec_tri, 0, a.rec_los, a.ctr + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t batch_diffraction(const BatchArgs& a, cudaStream_t s) {
    if (a.K_total <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.los_n, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.ctr + 2, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_diffraction_batch<<<grid_for(a.K_total, 128, 152 * 16), 128, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    k_visible_batch<<<trav_grid(a.K_total), kTravBlock, 0, s>>>(a, a.los_q, a.los_n, a.samp_offs, a.cand_p,
                                                                a.cand_tri, 1, a.keep, a.ctr + 2);
    return cudaGetLastError();
}

cudaError_t batch_direct(const BatchArgs& a, cudaStream_t s) {
    if (a.M_total <= 0) return cudaSuccess;
    note_launch();
    k_direct_batch<<<grid_for(a.M_total, 64), 64, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t batch_ranges(const BatchArgs& a, const uint32_t* scan_rec, const uint32_t* total_rec,
                         const uint32_t* scan_cand, const uint32_t* total_cand, cudaStream_t s) {
    note_launch();
    k_batch_ranges<<<(a.n_jobs + 63) / 64, 64, 0, s>>>(a, scan_rec, total_rec, scan_cand, total_cand);
    return cudaGetLastError();
}

}  // namespace st
