// Spectrum accumulation (Eq. 2-4 specular, Eq. 7-8 diffraction, Eq. 11-12 direct).
//
//   S[m][k] = sum over paths p of  A_pmk * exp(+j 2 pi f_k r_pm / c)
//   A_pmk   = r^-2 * 10^(-alpha(f_k) r / 20) * D_e(p, k) * X_p(k) * exp(-gamma_pm^2 g(T_p, f_k))
//
// The work is (paths x microphones x bins).  A CTA owns a tile of microphones x bins and streams
// a chunk of paths in tiles of P_T; partial spectra of the chunks are summed afterwards in a fixed
// order (deterministic, no float atomics).  Per path tile:
//   1a. per (path, bin):  log2(X_p(k) D_e) and the lobe exponent g(T_p, f_k)   -> shared memory
//   1b. per (path, mic):  r = r_pre + |m - P| in float-float (~44 bits), gamma^2, the phasor at the
//       first bin of every thread's bin run (range-reduced phase, sincospi), and the per-bin step
//       W = 2^(r log2-decay per bin) e^(j 2 pi frac(r df / c))                   -> shared memory
//   2.  per thread (R mics x KT consecutive bins): S += 2^(-gamma^2 g + log2 X) z ;  z *= W
// so the inner loop is one ex2, one FFMA for the exponent and six FP32 ops for the complex update.
// Diffraction paths without an emitter table skip 1a: their factor depends on the material and the bin
// only, and the term loop reads it from the CTA's material table at the row the producer names.
// With the per-microphone receiver test a microphone that does not see the path gets a zero anchor.
// The phase never loses precision: only frac(f r / c) enters FP32, and the recurrence runs at most
// KT steps from an exactly reduced anchor.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>

#include "st_accum_dev.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

using namespace acc;

// ---------------------------------------------------------------- per-bin material tables
__global__ void k_tables(int32_t F, int32_t n_mat, int32_t n_bands, const float* band_hz, const float* kb,
                         const float* beta, const float* diff, double f_lo, double df, double c, float* lk, float* g2,
                         float* lid, float* qhi, float* qlo, float2* bw) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F * n_mat) return;
    const int mat = idx / F, k = idx % F;
    const double f = (F == 1) ? f_lo : f_lo + (double)k * df;
    int b0 = 0;
    double w = 0.0;
    if (n_bands > 1) {
        if (f <= (double)band_hz[0]) {
            b0 = 0;
            w = 0.0;
        } else if (f >= (double)band_hz[n_bands - 1]) {
            b0 = n_bands - 2;
            w = 1.0;
        } else {
            int b = 0;
            while (b + 1 < n_bands && (double)band_hz[b + 1] <= f) ++b;
            if (b >= n_bands - 1) b = n_bands - 2;
            b0 = b;
            w = (f - (double)band_hz[b]) / ((double)band_hz[b + 1] - (double)band_hz[b]);
        }
    }
    auto interp = [&](const float* row) {
        if (n_bands == 1) return (double)row[0];
        return (1.0 - w) * (double)row[b0] + w * (double)row[b0 + 1];
    };
    const float* krow = kb + (int64_t)mat * n_bands;
    const float* brow = beta + (int64_t)mat * n_bands;
    const float* drow = diff + (int64_t)mat * n_bands;
    double kv = interp(krow);
    double g0 = 1.0 / (2.0 * (double)brow[b0] * (double)brow[b0]);
    double gv = g0;
    if (n_bands > 1) {
        double g1 = 1.0 / (2.0 * (double)brow[b0 + 1] * (double)brow[b0 + 1]);
        gv = (1.0 - w) * g0 + w * g1;
    }
    double dv = interp(drow);
    lk[idx] = kv > 0.0 ? (float)log2(kv) : kNegInf;
    g2[idx] = (float)(gv * 1.4426950408889634);
    lid[idx] = dv > 0.0 ? (float)log2(dv) : kNegInf;
    if (mat == 0) {
        double q = f / c;
        float h = (float)q;
        qhi[k] = h;
        qlo[k] = (float)(q - (double)h);
        bw[k] = make_float2((float)b0, (float)w);
    }
}

// two CTAs per SM (128 registers) stated explicitly: left to the heuristic, small edits elsewhere in the unit
// have turned it into one CTA of 236 registers; the directional variants keep one CTA (250 registers)
// One CTA of the accumulation: microphone block bx % n_mb, bin block bx / n_mb, chunk by of the path list.
// Threads past TP * NS (a block larger than the tile, as in the persistent batched launch) take part in
// the loads, the producer and the barriers only.
template <int KT, int KIND, int DIR, int SPLIT = 0>
__device__ __forceinline__ void accum_cta(const AccumArgs& a, const Geom& g, int bx, int by, float4* smem4) {
    static_assert((KT & (KT - 1)) == 0 && KT >= 2, "KT must be a power of two");
    const int PT = g.PT, NS = g.NS, TP = g.TP, KB = g.KB, MP = g.MP;
    const Buf B0 = buf_at<KT>(smem4, g, 0), B1 = buf_at<KT>(smem4, g, 1);
    float* pdb = reinterpret_cast<float*>(reinterpret_cast<char*>(smem4) + 2 * g.buf_bytes);  // [2][PT][12]
    int* pvb = reinterpret_cast<int*>(pdb + 2 * PT * 12);                                       // [2][PT]
    // material tables: 16-byte aligned for the 128-bit loads of phase 1a
    float* mt = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(pvb + 2 * PT) + 15) & ~uintptr_t(15));

    const int mb = bx % g.n_mb, bb = bx / g.n_mb;
    const int mic0 = mb * MP, kb = bb * KB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool cons = tid < TP * NS;  // a thread of the tile (term loop and outputs)
    const int tp = tid % TP, s = cons ? tid / TP : 0;

    const int64_t pb0 = a.d_base ? (int64_t)*a.d_base : 0;  // global index of this launch's first path
    const int64_t count = (int64_t)*a.d_count;
    const int64_t n_tiles = (count + PT - 1) / PT;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)by * per, t1 = min(n_tiles, t0 + per);

    u64 Sr[KT], Si[KT];
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) Sr[kk] = Si[kk] = 0ull;

    const float invNS = 1.0f / (float)NS, invKB = 1.0f / (float)KB;
    // per-bin band interpolation of the CTA's bins in table order (directional receivers)
    float2* bwt = reinterpret_cast<float2*>(mt + (g.mat_cached ? 2 * a.n_mat_tab * KB : 0));
    if (DIR && t0 < t1) {
        for (int i = tid; i < KB; i += nthr) {
            const int kk = __float2int_rz(((float)i + 0.5f) * invNS), s_ = i - kk * NS;
            bwt[i] = a.bw[min(kb + s_ * KT + kk, a.F - 1)];
        }
    }
    if (t0 < t1) {
        if (g.mat_cached) {
            const int nm = a.n_mat_tab;
            for (int e = tid; e < nm * KB; e += nthr) {
                const int mat = e / KB, i = e - mat * KB;
                const int kk = __float2int_rz(((float)i + 0.5f) * invNS), s_ = i - kk * NS;
                const int k = min(kb + s_ * KT + kk, a.F - 1);
                if (KIND == 0) {
                    mt[e] = a.lk[(int64_t)mat * a.F + k];
                    mt[nm * KB + e] = a.g2[(int64_t)mat * a.F + k];
                } else if (g.mat_direct) {  // the factor itself, as a pair for the two microphones of a thread
                    const float x = (kb + s_ * KT + kk < a.F) ? ex2(a.lid[(int64_t)mat * a.F + k]) : 0.0f;
                    reinterpret_cast<u64*>(mt)[e] = pk2(x, x);
                } else {
                    mt[e] = a.lid[(int64_t)mat * a.F + k];
                }
            }
        }
        load_paths<KIND>(a, PT, t0 * PT, count, pdb, pvb);
        if (t0 + 1 < t1) load_paths<KIND>(a, PT, (t0 + 1) * PT, count, pdb + PT * 12, pvb + PT);
        __syncthreads();
        produce<KT, KIND, 0, SPLIT>(a, g, B0, pdb, pvb, mt, mic0, kb, invNS, invKB, nullptr, pb0 + t0 * PT);
        __syncthreads();
    }
    // software pipeline: consume tile t from buffer b while producing tile t+1 into buffer b^1
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int b = (int)((tile - t0) & 1);
        const Buf& C = b ? B1 : B0;
        const Buf& Pn = b ? B0 : B1;
        // path data of tile+2 into pd buffer b, in flight during this tile (buffer b held this tile's path data,
        // read by its producer one step ago; the term loop reads only the tile buffers)
        if (tile + 2 < t1) load_paths_cp<KIND>(a, PT, (tile + 2) * PT, count, pdb + b * PT * 12, pvb + b * PT);
        if (tile + 1 < t1) {
            const int nb = b ^ 1;  // path data of tile+1 sits in pd buffer nb
            produce<KT, KIND, 0, SPLIT>(a, g, Pn, pdb + nb * PT * 12, pvb + nb * PT, mt, mic0, kb, invNS, invKB, nullptr,
                              pb0 + (tile + 1) * PT);
        }
        for (int p = 0; p < (cons ? PT : 0); ++p) {
            const ulonglong2 z0 = C.za[((size_t)p * NS + s) * TP + tp];
            const u64* w = C.wst + (size_t)p * 4 * TP + tp;  // component-major: conflict-free 64-bit loads
            const u64 w1r = w[0], w1i = w[TP], w2r = w[2 * TP], w2i = w[3 * TP];
            const u64 nw2i = fmul2(w2i, pk2(-1.0f, -1.0f));
            const u64 ng = C.ngp[(size_t)p * TP + tp];
            u64 er = z0.x, ei = z0.y;  // even chain: bins 0, 2, 4, ...
            u64 orr = er, oi = ei;     // odd chain: bins 1, 3, 5, ...
            cmul2(orr, oi, w1r, w1i, fmul2(w1i, pk2(-1.0f, -1.0f)));
            const float2* trow = reinterpret_cast<const float2*>(C.tab) + (size_t)p * KB + s;
            const float2 ngv = up2(ng);  // -gamma^2 of the two microphones
            // diffraction with the material table read directly: the producer left the offset of the path's
            // material row in the (otherwise unused) lobe slot
            const u64* mrow = reinterpret_cast<const u64*>(mt) + s;
            if (KIND == 1 && g.mat_direct) mrow += (int)(uint32_t)ng;
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) {
                u64 E;
                if (KIND == 1 && g.mat_direct) {
                    E = mrow[kk * NS];
                } else if (KIND == 0) {
                    const float2 t = trow[kk * NS];  // (log2 X, g)
                    E = pk2(ex2(fmaf(ngv.x, t.y, t.x)), ex2(fmaf(ngv.y, t.y, t.x)));
                } else {
                    E = reinterpret_cast<const u64*>(trow)[kk * NS];  // (X, X)
                }
                if (DIR) {  // receiver directivity, linear between bands
                    const float2 bwv = bwt[kk * NS + s];
                    const int b0 = (int)bwv.x;
                    const float* d1 = C.dband + ((size_t)p * MP + 2 * tp) * g.NB;
                    const float* d2 = d1 + g.NB;
                    float D1 = d1[b0], D2 = d2[b0];
                    if (g.NB > 1) {
                        D1 = fmaf(bwv.y, d1[b0 + 1] - D1, D1);
                        D2 = fmaf(bwv.y, d2[b0 + 1] - D2, D2);
                    }
                    E = fmul2(E, pk2(D1, D2));
                }
                if ((kk & 1) == 0) {
                    Sr[kk] = ffma2(E, er, Sr[kk]);
                    Si[kk] = ffma2(E, ei, Si[kk]);
                    cmul2(er, ei, w2r, w2i, nw2i);
                } else {
                    Sr[kk] = ffma2(E, orr, Sr[kk]);
                    Si[kk] = ffma2(E, oi, Si[kk]);
                    cmul2(orr, oi, w2r, w2i, nw2i);
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
    // ---- partial spectra of this chunk
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int m = mic0 + 2 * tp + h;
        if (!cons || m >= a.M) continue;
        float2* out = a.partial + ((size_t)by * a.M + m) * a.F;
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            const int k = kb + s * KT + kk;
            const float2 re = up2(Sr[kk]), im = up2(Si[kk]);
            if (k < a.F) out[k] = h == 0 ? make_float2(re.x, im.x) : make_float2(re.y, im.y);
        }
    }
}

template <int KT, int KIND, int DIR>
__global__ void __launch_bounds__(256, DIR ? 1 : 2) k_accum(const AccumArgs a, const Geom g) {
    extern __shared__ float4 smem4[];
    accum_cta<KT, KIND, DIR>(a, g, blockIdx.x, blockIdx.y, smem4);
}

// Persistent accumulation of a batch: each CTA takes work items -- one CTA's worth of one (job, path kind)
// accumulation: its microphone block, bin block and chunk -- from a device counter until none is left, and
// runs them with the single-pose CTA body.  Items are claimed in task order; no item waits for another.  One
// launch per path kind (the tasks of that kind).
template <int KIND>
__global__ void __launch_bounds__(256, 2) k_accum_queue(const AccumTask* tasks, int32_t n_tasks, int64_t n_items,
                                                        unsigned long long* counter) {
    extern __shared__ float4 smem4[];
    __shared__ long long item_s;
    __shared__ int task_s;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(counter, 1ull);
            int lo = 0, hi = n_tasks - 1;  // last task whose first item is <= it
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tasks[mid].item0 <= it) lo = mid; else hi = mid - 1;
            }
            item_s = it;
            task_s = lo;
        }
        __syncthreads();
        const long long it = item_s;
        const AccumTask& T = tasks[task_s];
        __syncthreads();  // every thread has read the claim before the next one overwrites it
        if (it >= n_items) break;
        const int nxy = T.g.n_mb * T.g.n_bb;
        const int local = (int)(it - T.item0);
        accum_cta<16, KIND, 0, 1>(T.a, T.g, local % nxy, local / nxy, smem4);
        __syncthreads();  // shared memory is reused by the next item
    }
}

// Fixed-order sums of every task's chunk partials into its output: one thread per (task, microphone, bin).
__global__ void k_reduce_tasks(const AccumTask* tasks, int32_t n_tasks, int64_t n_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_out; i += stride) {
        int lo = 0, hi = n_tasks - 1;  // last task whose first output is <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tasks[mid].out0 <= i) lo = mid; else hi = mid - 1;
        }
        const AccumTask& T = tasks[lo];
        const int64_t MF = (int64_t)T.a.M * T.a.F, l = i - T.out0;
        float sx = 0.0f, sy = 0.0f;
        for (int c = 0; c < T.a.n_chunks; ++c) {
            const float2 v = T.a.partial[(int64_t)c * MF + l];
            sx += v.x;
            sy += v.y;
        }
        T.out[l] = make_float2(sx, sy);
    }
}

__global__ void k_reduce(const float2* __restrict__ partial, int32_t n_chunks, int64_t MF, float2* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MF; i += stride) {
        float sx = 0.0f, sy = 0.0f;
        for (int c = 0; c < n_chunks; ++c) {
            const float2 v = partial[(int64_t)c * MF + i];
            sx += v.x;
            sy += v.y;
        }
        out[i] = make_float2(sx, sy);
    }
}

// ---------------------------------------------------------------- direct path (Eq. 11-12)
__device__ float2 direct_term(const DirectAccumArgs& a, const float* qhi, const float* qlo, int m, int k);

__global__ void k_direct_accum(const DirectAccumArgs a, const float* qhi, const float* qlo) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.M * a.F) return;
    const int m = (int)(idx / a.F), k = (int)(idx % a.F);
    a.out[idx] = a.vis[m] ? direct_term(a, qhi, qlo, m, k) : make_float2(0.0f, 0.0f);
}

// the direct path's term at microphone m and bin k (visible)
__device__ float2 direct_term(const DirectAccumArgs& a, const float* qhi, const float* qlo, int m, int k) {
    float2 v;
    {
        const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
        const ff r = dist_ff(mx, my, mz, a.s[0], a.s[1], a.s[2]);
        const double f = a.F == 1 ? a.f_lo : a.f_lo + (double)k * a.df;
        const float alpha = (float)(a.a0 + a.a1 * (f / 1000.0));
        // log2 amplitude: log2(gain) - 2 log2 r - alpha r log2(10) / 20
        float L = log2f(a.gain) - 2.0f * log2_ff(r) - alpha * r.hi * (3.3219280948873623f / 20.0f);
        if (a.etab) {
            const float inv = 1.0f / r.hi;
            const float c = (a.fwd[0] * (mx - a.s[0]) + a.fwd[1] * (my - a.s[1]) + a.fwd[2] * (mz - a.s[2])) * inv;
            const float th = acosf(fminf(1.0f, fmaxf(-1.0f, c)));
            const float x = th * ((float)(a.n_theta - 1) / 3.14159265358979f);
            const int i = min((int)x, a.n_theta - 2);
            const float w = x - (float)i;
            const float de = (1.0f - w) * a.etab[(int64_t)i * a.F + k] + w * a.etab[(int64_t)(i + 1) * a.F + k];
            L += de > 0.0f ? log2f(de) : kNegInf;
        }
        const ff x = ff_mul(r, ff{qhi[k], qlo[k]});
        float sn, cs;
        sincospif(2.0f * ff_frac(x), &sn, &cs);
        float A = exp2f(L);
        if (a.mic_tab) {  // arrival from the emitter
            AccumArgs aa{};
            aa.mic_tab = a.mic_tab;
            aa.mic_q = a.mic_q;
            aa.n_el = a.n_el;
            aa.n_az = a.n_az;
            float band[64];
            mic_bands(aa, m, a.s[0] - mx, a.s[1] - my, a.s[2] - mz, band, a.n_bands);
            const float2 bwv = a.bw[k];
            const int b0 = (int)bwv.x;
            float D = band[b0];
            if (a.n_bands > 1) D = fmaf(bwv.y, band[b0 + 1] - D, D);
            A *= D;
        }
        v = make_float2(A * cs, A * sn);
    }
    return v;
}

// direct path of every job of a batch: one thread per (job, mic, bin), the single-pose term
__global__ void k_direct_accum_batch(const BatchArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.MF_total; g += stride) {
        const JobDev& b = a.jobs[find_job(a.mf_offs, a.n_jobs, g)];
        const int64_t local = g - b.mf_off;
        const int m = (int)(local / b.F), k = (int)(local % b.F);
        float2 v = make_float2(0.0f, 0.0f);
        if (a.dvis[b.mic_off + m]) {
            DirectAccumArgs d{};
            d.s[0] = b.s[0];
            d.s[1] = b.s[1];
            d.s[2] = b.s[2];
            d.mics = b.mics;
            d.M = b.M;
            d.F = b.F;
            d.f_lo = b.f_lo;
            d.df = b.df;
            d.a0 = a.a0;
            d.a1 = a.a1;
            d.gain = a.direct_gain;
            d.etab = b.etab;
            d.n_theta = b.n_theta;
            d.fwd[0] = b.fwd[0];
            d.fwd[1] = b.fwd[1];
            d.fwd[2] = b.fwd[2];
            d.mic_tab = b.mic_tab;
            d.mic_q = b.mic_q;
            d.n_el = b.n_el;
            d.n_az = b.n_az;
            d.n_bands = b.n_bands;
            d.bw = b.bw;
            v = direct_term(d, b.qhi, b.qlo, m, k);
        }
        b.out[(size_t)2 * b.M * b.F + local] = v;
    }
}

// ---------------------------------------------------------------- path gathering
__global__ void k_flags_records(const int32_t* rec_tri, const uint8_t* rec_los, int64_t n, uint32_t* flags) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        flags[i] = (rec_tri[i] >= 0 && rec_los[i]) ? 1u : 0u;
}
__global__ void k_flags_u8(const uint8_t* keep, int64_t n, uint32_t* flags) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) flags[i] = keep[i] ? 1u : 0u;
}
__global__ void k_compact(const uint32_t* flags, const uint32_t* scan, int64_t n, uint32_t* idx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (flags[i]) idx[scan[i]] = (uint32_t)i;
}

__device__ __forceinline__ float3 rot(const float q[4], float vx, float vy, float vz) {
    // q applied to v (float32, same steps as the tracing kernels; used only for directivity angles)
    const float tx = 2.0f * (q[2] * vz - q[3] * vy), ty = 2.0f * (q[3] * vx - q[1] * vz), tz = 2.0f * (q[1] * vy - q[2] * vx);
    return make_float3(vx + q[0] * tx + (q[2] * tz - q[3] * ty), vy + q[0] * ty + (q[3] * tx - q[1] * tz),
                       vz + q[0] * tz + (q[1] * ty - q[2] * tx));
}

__global__ void k_gather_spec(const GatherArgs g, float* px, float* py, float* pz, float* dx, float* dy, float* dz,
                              float* rhi, float* rlo, uint32_t* chl, uint32_t* chh, uint32_t* meta, float* dep,
                              uint64_t* mask) {
    const int64_t n = *g.count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const int64_t id = g.idx[c];
        const int64_t ray = id / g.B;
        const int j = (int)(id % g.B);
        px[c] = g.rec_p[3 * id];
        py[c] = g.rec_p[3 * id + 1];
        pz[c] = g.rec_p[3 * id + 2];
        dx[c] = g.rec_d[3 * id];
        dy[c] = g.rec_d[3 * id + 1];
        dz[c] = g.rec_d[3 * id + 2];
        const double r = g.rec_r[id];
        const float h = (float)r;
        rhi[c] = h;
        rlo[c] = (float)(r - (double)h);
        uint32_t lo = 0, hi = 0;
        int matj = 0;
        for (int q = 0; q <= j; ++q) {
            uint32_t mq = (uint32_t)g.tri_mat[g.rec_tri[ray * g.B + q]] & 255u;
            ST_CHECK_OR((int)mq < g.n_mat, g.chk, mq = 0);
            if (q < 4) lo |= mq << (8 * q); else hi |= mq << (8 * (q - 4));
            matj = (int)mq;
        }
        chl[c] = lo;
        chh[c] = hi;
        meta[c] = (uint32_t)(j + 1) | ((uint32_t)matj << 8);
        if (g.rec_mask) mask[c] = g.rec_mask[id];
        if (g.has_etab) {
            const float3 d = rot(g.q, g.dirs[3 * ray], g.dirs[3 * ray + 1], g.dirs[3 * ray + 2]);
            const float l = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
            const float cth = (g.fwd[0] * d.x + g.fwd[1] * d.y + g.fwd[2] * d.z) / l;
            dep[c] = acosf(fminf(1.0f, fmaxf(-1.0f, cth))) * g.inv_dtheta;
        } else {
            dep[c] = -1.0f;
        }
    }
}

__global__ void k_gather_diff(const GatherArgs g, float* px, float* py, float* pz, float* rhi, float* rlo,
                              uint32_t* meta, float* dep) {
    const int64_t n = *g.count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const int64_t i = g.idx[c];
        const float ox = g.cand_p[3 * i], oy = g.cand_p[3 * i + 1], oz = g.cand_p[3 * i + 2];
        px[c] = ox;
        py[c] = oy;
        pz[c] = oz;
        const ff r = dist_ff(ox, oy, oz, g.s[0], g.s[1], g.s[2]);
        rhi[c] = r.hi;
        rlo[c] = r.lo;
        uint32_t mi = (uint32_t)g.tri_mat[g.cand_tri[i]] & 255u;
        ST_CHECK_OR((int)mi < g.n_mat, g.chk, mi = 0);
        meta[c] = mi << 8;
        if (g.has_etab) {
            const float vx = ox - g.s[0], vy = oy - g.s[1], vz = oz - g.s[2];
            const float cth = (g.fwd[0] * vx + g.fwd[1] * vy + g.fwd[2] * vz) / r.hi;
            dep[c] = acosf(fminf(1.0f, fmaxf(-1.0f, cth))) * g.inv_dtheta;
        } else {
            dep[c] = -1.0f;
        }
    }
}

// accumulator tile shape: mic pairs per CTA and shared-memory budget (set by the tuner or ST_ACCUM_TILE="tp,kb")
int g_tile_tp = 16;
size_t g_tile_budget = 104 * 1024;  // two CTAs per SM (swept 88-110 KB: 104 fastest on the clutter workload)
int g_tile_kt = 16;
bool g_tile_env_read = false;
bool g_tile_env_set = false;  // ST_ACCUM_TILE gave the tile shape

void read_tile_env() {
    if (g_tile_env_read) return;
    g_tile_env_read = true;
    const char* e = getenv("ST_ACCUM_TILE");
    if (!e) return;
    int tp = 0, kbudget = 0, kt = 16;
    if (sscanf(e, "%d,%d,%d", &tp, &kbudget, &kt) >= 2 && tp >= 1 && tp <= 128 && kbudget >= 16 && kbudget <= 200 &&
        (kt == 8 || kt == 16)) {
        g_tile_tp = tp;
        g_tile_budget = (size_t)kbudget * 1024;
        g_tile_kt = kt;
        g_tile_env_set = true;
    }
}

// tile shape of one accumulation (kind 0 specular, 1 diffraction): the tuner's or the defaults
Geom accum_geom(const AccumArgs& a, int kind, int kt, int dir) {
    read_tile_env();
    // diffraction paths whose factor is read from the material table: half the microphone pairs per CTA, so
    // that a CTA covers twice the bins and each (path, microphone) anchor is formed half as often (the tile
    // has no per-(path, bin) table whose cost would grow in return)
    const bool direct_mat = kind == 1 && !a.etab;
    const int tp = a.tile_tp > 0 ? a.tile_tp : (direct_mat && !g_tile_env_set ? std::max(1, g_tile_tp / 2) : g_tile_tp);
    const size_t budget = a.tile_kb > 0 ? (size_t)a.tile_kb * 1024 : g_tile_budget;
    return make_geom(a.M, a.F, kt, a.n_mat_tab, tp, budget, dir ? a.n_bands_tab : 0, direct_mat, 1);
}

template <int KT, int KIND, int DIR>
cudaError_t launch_accum(const AccumArgs& a, cudaStream_t s) {
    const Geom g = accum_geom(a, KIND, KT, DIR);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_accum<KT, KIND, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)(g.n_mb * g.n_bb), (unsigned)a.n_chunks);
    note_launch();
    k_accum<KT, KIND, DIR><<<grid, g.TP * g.NS, g.smem, s>>>(a, g);
    return cudaGetLastError();
}

// path list entries of every job (same layout as the single-pose gather; omni emitter)
__global__ void k_gather_spec_batch(const BatchArgs a, const uint32_t* idx, const uint32_t* count, float* px, float* py,
                                    float* pz, float* dx, float* dy, float* dz, float* rhi, float* rlo, uint32_t* chl,
                                    uint32_t* chh, uint32_t* meta, float* dep, uint64_t* mask) {
    const int64_t n = *count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const int64_t id = idx[c];
        const int job = find_job(a.rec_offs, a.n_jobs, id);
        const JobDev& b = a.jobs[job];
        const int64_t local = id - b.rec_off;
        const int64_t ray = local / b.B;
        const int j = (int)(local % b.B);
        px[c] = a.rec_p[3 * id];
        py[c] = a.rec_p[3 * id + 1];
        pz[c] = a.rec_p[3 * id + 2];
        dx[c] = a.rec_d[3 * id];
        dy[c] = a.rec_d[3 * id + 1];
        dz[c] = a.rec_d[3 * id + 2];
        const double r = a.rec_r[id];
        const float h = (float)r;
        rhi[c] = h;
        rlo[c] = (float)(r - (double)h);
        uint32_t lo = 0, hi = 0;
        int matj = 0;
        for (int q = 0; q <= j; ++q) {
            uint32_t mq = (uint32_t)b.tri_mat[a.rec_tri[b.rec_off + ray * b.B + q]] & 255u;
            ST_CHECK_OR((int)mq < b.n_mat, a.flags, mq = 0);
            if (q < 4) lo |= mq << (8 * q); else hi |= mq << (8 * (q - 4));
            matj = (int)mq;
        }
        chl[c] = lo;
        chh[c] = hi;
        meta[c] = (uint32_t)(j + 1) | ((uint32_t)matj << 8);
        if (b.etab) {  // emission angle of the path's primary ray, as the single-pose gather
            const int64_t rg = ray;
            const float3 d = rot(b.q, b.dirs[3 * rg], b.dirs[3 * rg + 1], b.dirs[3 * rg + 2]);
            const float l = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
            const float cth = (b.fwd[0] * d.x + b.fwd[1] * d.y + b.fwd[2] * d.z) / l;
            dep[c] = acosf(fminf(1.0f, fmaxf(-1.0f, cth))) * b.inv_dtheta;
        } else {
            dep[c] = -1.0f;
        }
        if (mask) mask[c] = a.rec_mask[id];  // per-microphone receiver test
    }
}

__global__ void k_gather_diff_batch(const BatchArgs a, const uint32_t* idx, const uint32_t* count, float* px, float* py,
                                    float* pz, float* rhi, float* rlo, uint32_t* meta, float* dep) {
    const int64_t n = *count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const int64_t i = idx[c];
        const int job = find_job(a.samp_offs, a.n_jobs, i);
        const JobDev& b = a.jobs[job];
        const float ox = a.cand_p[3 * i], oy = a.cand_p[3 * i + 1], oz = a.cand_p[3 * i + 2];
        px[c] = ox;
        py[c] = oy;
        pz[c] = oz;
        const ff r = dist_ff(ox, oy, oz, b.s[0], b.s[1], b.s[2]);
        rhi[c] = r.hi;
        rlo[c] = r.lo;
        uint32_t mi = (uint32_t)b.tri_mat[a.cand_tri[i]] & 255u;
        ST_CHECK_OR((int)mi < b.n_mat, a.flags, mi = 0);
        meta[c] = mi << 8;
        if (b.etab) {
            const float vx = ox - b.s[0], vy = oy - b.s[1], vz = oz - b.s[2];
            const float cth = (b.fwd[0] * vx + b.fwd[1] * vy + b.fwd[2] * vz) / r.hi;
            dep[c] = acosf(fminf(1.0f, fmaxf(-1.0f, cth))) * b.inv_dtheta;
        } else {
            dep[c] = -1.0f;
        }
    }
}

}  // namespace

int32_t accum_chunks(int64_t n_paths_hint, int32_t M, int32_t F, int32_t n_mat, int32_t dir_nb, int32_t tile_tp,
                     int32_t tile_kb, int32_t tile_kt) {
    if (narrow_accum(M)) return narrow_chunks(n_paths_hint, M, F, n_mat, dir_nb);
    read_tile_env();
    const int tp = tile_tp > 0 ? tile_tp : g_tile_tp;
    const size_t budget = tile_kb > 0 ? (size_t)tile_kb * 1024 : g_tile_budget;
    const Geom g = make_geom(M, F, dir_nb ? 16 : (tile_kt > 0 ? tile_kt : g_tile_kt), n_mat, tp, budget, dir_nb, 0, 1);
    const int ctas_per_chunk = g.n_mb * g.n_bb;
    const int threads = g.TP * g.NS;
    int resident = std::max(1, std::min(2048 / std::max(threads, 32), (int)((220 * 1024) / std::max<size_t>(g.smem, 1))));
    int64_t want = (int64_t)152 * resident / std::max(ctas_per_chunk, 1);
    int64_t tiles = (n_paths_hint + g.PT - 1) / g.PT;
    want = std::min<int64_t>(want, std::max<int64_t>(tiles, 1));
    return (int32_t)std::max<int64_t>(1, want);
}

cudaError_t build_accum_tables(AccumTables& T, const SceneDev& S, int32_t F, double f_lo, double f_hi, double c,
                               double a0, double a1, cudaStream_t s) {
    const int n_mat = S.n_mat, nb = S.n_bands;
    cudaError_t e;
    if ((e = grow(T.lk, (size_t)n_mat * F * 4)) != cudaSuccess) return e;
    if ((e = grow(T.g2, (size_t)n_mat * F * 4)) != cudaSuccess) return e;
    if ((e = grow(T.lid, (size_t)n_mat * F * 4)) != cudaSuccess) return e;
    if ((e = grow(T.qhi, (size_t)F * 4)) != cudaSuccess) return e;
    if ((e = grow(T.qlo, (size_t)F * 4)) != cudaSuccess) return e;
    if ((e = grow(T.bw, (size_t)F * 8)) != cudaSuccess) return e;
    DevBuf mt;
    const size_t mb = (size_t)(nb + 3 * n_mat * nb) * 4;
    if ((e = grow(mt, mb)) != cudaSuccess) return e;
    std::vector<float> h;
    h.insert(h.end(), S.band_hz.begin(), S.band_hz.end());
    h.insert(h.end(), S.k_band.begin(), S.k_band.end());
    h.insert(h.end(), S.beta_band.begin(), S.beta_band.end());
    h.insert(h.end(), S.diff_band.begin(), S.diff_band.end());
    e = cudaMemcpyAsync(mt.p, h.data(), mb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        release(mt);
        return e;
    }
    const float* d = ptr<float>(mt);
    const double df = F > 1 ? (f_hi - f_lo) / (double)(F - 1) : 0.0;
    note_launch();
    k_tables<<<(F * n_mat + 127) / 128, 128, 0, s>>>(F, n_mat, nb, d, d + nb, d + nb + n_mat * nb,
                                                    d + nb + 2 * n_mat * nb, f_lo, df, c, ptr<float>(T.lk),
                                                    ptr<float>(T.g2), ptr<float>(T.lid), ptr<float>(T.qhi),
                                                    ptr<float>(T.qlo), ptr<float2>(T.bw));
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(s);  // the staging buffer is freed below
    release(mt);
    if (e != cudaSuccess) return e;
    if (e2 != cudaSuccess) return e2;
    if ((e = grow(T.band, (size_t)nb * 4)) != cudaSuccess) return e;
    if ((e = grow(T.kband, (size_t)n_mat * nb * 4)) != cudaSuccess) return e;
    if ((e = grow(T.bband, (size_t)n_mat * nb * 4)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(T.bband.p, S.beta_band.data(), (size_t)n_mat * nb * 4, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(T.band.p, S.band_hz.data(), (size_t)nb * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(T.kband.p, S.k_band.data(), (size_t)n_mat * nb * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    T.F = F;
    T.n_mat = n_mat;
    T.n_bands = nb;
    T.f_lo = f_lo;
    T.df = df;
    T.c = c;
    T.a0 = a0;
    T.a1 = a1;
    return cudaSuccess;
}

cudaError_t accumulate(const AccumArgs& a, cudaStream_t s) {
    if (narrow_accum(a.M)) return accumulate_narrow(a, s);
    read_tile_env();
    if (a.mic_tab) return a.kind == 0 ? launch_accum<16, 0, 1>(a, s) : launch_accum<16, 1, 1>(a, s);
    if ((a.tile_kt > 0 ? a.tile_kt : g_tile_kt) == 8)
        return a.kind == 0 ? launch_accum<8, 0, 0>(a, s) : launch_accum<8, 1, 0>(a, s);
    return a.kind == 0 ? launch_accum<16, 0, 0>(a, s) : launch_accum<16, 1, 0>(a, s);
}

cudaError_t accum_task(const AccumArgs& a, float2* out, AccumTask* t) {
    t->a = a;
    t->g = accum_geom(a, a.kind, 16, 0);
    t->out = out;
    return cudaSuccess;
}

cudaError_t accumulate_queue(int kind, const AccumTask* tasks, int32_t n_tasks, int64_t n_items, size_t smem,
                             unsigned long long* counter, cudaStream_t s) {
    static bool attr_set[2] = {false, false};
    if (!attr_set[kind]) {
        cudaError_t e = cudaFuncSetAttribute(kind == 0 ? k_accum_queue<0> : k_accum_queue<1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[kind] = true;
    }
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n_tasks <= 0 || n_items <= 0) return e;
    int dev = 0, n_sm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = smem > 110 * 1024 ? 1 : 2;
    const unsigned grid = (unsigned)std::min<int64_t>((int64_t)n_sm * per_sm, n_items);
    note_launch();
    if (kind == 0) k_accum_queue<0><<<grid, 256, smem, s>>>(tasks, n_tasks, n_items, counter);
    else k_accum_queue<1><<<grid, 256, smem, s>>>(tasks, n_tasks, n_items, counter);
    return cudaGetLastError();
}

cudaError_t reduce_tasks(const AccumTask* tasks, int32_t n_tasks, int64_t n_out, cudaStream_t s) {
    if (n_tasks <= 0 || n_out <= 0) return cudaSuccess;
    note_launch();
    k_reduce_tasks<<<grid_for(n_out, 256), 256, 0, s>>>(tasks, n_tasks, n_out);
    return cudaGetLastError();
}

cudaError_t reduce_partials(const float2* partial, int32_t n_chunks, int64_t MF, float2* out, cudaStream_t s) {
    note_launch();
    k_reduce<<<grid_for(MF, 256), 256, 0, s>>>(partial, n_chunks, MF, out);
    return cudaGetLastError();
}

cudaError_t accumulate_direct(const DirectAccumArgs& a, const float* qhi, const float* qlo, cudaStream_t s) {
    const int64_t n = (int64_t)a.M * a.F;
    if (n <= 0) return cudaSuccess;
    note_launch();
    k_direct_accum<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, qhi, qlo);
    return cudaGetLastError();
}

cudaError_t batch_direct_accum(const BatchArgs& a, cudaStream_t s) {
    if (a.MF_total <= 0) return cudaSuccess;
    note_launch();
    k_direct_accum_batch<<<grid_for(a.MF_total, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t flags_visible_records(const int32_t* rec_tri, const uint8_t* rec_los, int64_t n, uint32_t* flags,
                                  cudaStream_t s) {
    note_launch();
    k_flags_records<<<grid_for(n, 256), 256, 0, s>>>(rec_tri, rec_los, n, flags);
    return cudaGetLastError();
}
cudaError_t flags_from_u8(const uint8_t* keep, int64_t n, uint32_t* flags, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    note_launch();
    k_flags_u8<<<grid_for(n, 256), 256, 0, s>>>(keep, n, flags);
    return cudaGetLastError();
}
cudaError_t compact_indices(const uint32_t* flags, const uint32_t* scan, int64_t n, uint32_t* idx, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    note_launch();
    k_compact<<<grid_for(n, 256), 256, 0, s>>>(flags, scan, n, idx);
    return cudaGetLastError();
}

// Emitter-table row of every compacted specular path (the floor of its angle coordinate), 0xffff past the
// count: sorting the compacted list by it lets the paths of an accumulator tile share table rows.
__global__ void k_theta_keys(const GatherArgs g, int64_t cap, uint64_t* keys) {
    const int64_t n = *g.count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cap; c += stride) {
        uint64_t key = 0xffffu;
        if (c < n) {
            const int64_t ray = (int64_t)g.idx[c] / g.B;
            const float3 d = rot(g.q, g.dirs[3 * ray], g.dirs[3 * ray + 1], g.dirs[3 * ray + 2]);
            const float l = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
            const float cth = (g.fwd[0] * d.x + g.fwd[1] * d.y + g.fwd[2] * d.z) / l;
            const float x = acosf(fminf(1.0f, fmaxf(-1.0f, cth))) * g.inv_dtheta;
            key = (uint64_t)min((int)x, 0xfffe);
        }
        keys[c] = key;
    }
}

cudaError_t theta_order(const GatherArgs& g, int64_t cap, uint32_t* idx, uint64_t* keys, void* scratch,
                        cudaStream_t s) {
    if (cap <= 1) return cudaSuccess;
    note_launch();
    k_theta_keys<<<grid_for(cap, 256), 256, 0, s>>>(g, cap, keys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return radix_sort_u64(keys, idx, cap, 16, scratch, s);  // stable: equal rows keep the compaction order
}

// Key of a compacted specular path for chain order: the counts of materials 0..3 in its reflection chain in
// base 9 (cumulative reflection), or its last hit's material (last-hit reflection); entries past *g.count last.
__global__ void k_chain_keys(const GatherArgs g, int64_t cap, int last_only, uint64_t* keys) {
    const int64_t n = *g.count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cap; c += stride) {
        uint64_t key = 0x3fffu;
        if (c < n) {
            const int64_t id = g.idx[c];
            const int64_t ray = id / g.B;
            const int j = (int)(id % g.B);
            if (last_only) {
                key = (uint64_t)((uint32_t)g.tri_mat[g.rec_tri[id]] & 255u);
            } else {
                int cnt[4] = {0, 0, 0, 0};
                for (int q = 0; q <= j; ++q) {
                    const int mq = g.tri_mat[g.rec_tri[ray * g.B + q]];
                    if (mq >= 0 && mq < 4) cnt[mq]++;
                }
                key = (uint64_t)(((cnt[3] * 9 + cnt[2]) * 9 + cnt[1]) * 9 + cnt[0]);
            }
        }
        keys[c] = key;
    }
}

cudaError_t chain_order(const GatherArgs& g, int64_t cap, int last_only, uint32_t* idx, uint64_t* keys, void* scratch,
                        cudaStream_t s) {
    if (cap <= 1) return cudaSuccess;
    note_launch();
    k_chain_keys<<<grid_for(cap, 256), 256, 0, s>>>(g, cap, last_only, keys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return radix_sort_u64(keys, idx, cap, 14, scratch, s);  // stable: equal chains keep the compaction order
}

cudaError_t gather_specular(const GatherArgs& g, cudaStream_t s) {
    PathList& P = *g.out;
    note_launch();
    k_gather_spec<<<grid_for(g.N * g.B, 256), 256, 0, s>>>(
        g, ptr<float>(P.px), ptr<float>(P.py), ptr<float>(P.pz), ptr<float>(P.dx), ptr<float>(P.dy), ptr<float>(P.dz),
        ptr<float>(P.rhi), ptr<float>(P.rlo), ptr<uint32_t>(P.chain_lo), ptr<uint32_t>(P.chain_hi),
        ptr<uint32_t>(P.meta), ptr<float>(P.dep), g.rec_mask ? ptr<uint64_t>(P.mask) : nullptr);
    return cudaGetLastError();
}

cudaError_t gather_diffraction(const GatherArgs& g, cudaStream_t s) {
    PathList& P = *g.out;
    if (g.K <= 0) return cudaSuccess;
    note_launch();
    k_gather_diff<<<grid_for(g.K, 256), 256, 0, s>>>(g, ptr<float>(P.px), ptr<float>(P.py), ptr<float>(P.pz),
                                                     ptr<float>(P.rhi), ptr<float>(P.rlo), ptr<uint32_t>(P.meta),
                                                     ptr<float>(P.dep));
    return cudaGetLastError();
}

cudaError_t batch_gather_spec(const BatchArgs& a, const uint32_t* idx, const uint32_t* count, PathList& P,
                              cudaStream_t s) {
    note_launch();
    k_gather_spec_batch<<<grid_for(a.R_total, 256), 256, 0, s>>>(
        a, idx, count, ptr<float>(P.px), ptr<float>(P.py), ptr<float>(P.pz), ptr<float>(P.dx), ptr<float>(P.dy),
        ptr<float>(P.dz), ptr<float>(P.rhi), ptr<float>(P.rlo), ptr<uint32_t>(P.chain_lo), ptr<uint32_t>(P.chain_hi),
        ptr<uint32_t>(P.meta), ptr<float>(P.dep), a.rec_mask ? ptr<uint64_t>(P.mask) : nullptr);
    return cudaGetLastError();
}

cudaError_t batch_gather_diff(const BatchArgs& a, const uint32_t* idx, const uint32_t* count, PathList& P,
                              cudaStream_t s) {
    if (a.K_total <= 0) return cudaSuccess;
    note_launch();
    k_gather_diff_batch<<<grid_for(a.K_total, 256), 256, 0, s>>>(a, idx, count, ptr<float>(P.px), ptr<float>(P.py),
                                                                  ptr<float>(P.pz), ptr<float>(P.rhi),
                                                                  ptr<float>(P.rlo), ptr<uint32_t>(P.meta),
                                                                  ptr<float>(P.dep));
    return cudaGetLastError();
}

}  // namespace st
