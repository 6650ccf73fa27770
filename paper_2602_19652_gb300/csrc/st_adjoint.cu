// Adjoint of the spectrum accumulation (the paper has no gradients; this is the hand-written
// reverse pass of Eq. 2-4, 7-8, 11-12 with the path set frozen).
//
// Given G[m][k] = dL/dRe S + j dL/dIm S, every term T_pmk of the forward sum contributes
// Re(conj(G_mk) dT_pmk/dtheta).  With w = conj(G) T:
//   path length r:  d ln T_k / dr = D0 + (k - kb) D1,  D0 = -2/r - a(kb) + j 2 pi f_kb / c,
//                   D1 = -a_step + j 2 pi df / c  (a = amplitude decay in nepers per metre)
//                   => dL/dr = Re(D0 C0 + D1 C1), C0 = sum_k w, C1 = sum_k (k - kb) w
//   lobe angle:     d ln T_k / dgamma = -2 gamma g_k  => dL/dgamma = -2 gamma sum_k g_k Re w
//   reflection k:   d ln T / d k_band[mat][b] = cnt_mat(p) w_b(k) / k(mat, f_k)
//                   => dL/dk[mat][b] = sum_k V[mat][k] w_b(k) / k(mat, f_k), V[mat][k] = sum_p,m cnt Re w
// and the positions follow through dr/dm = unit(m - P), dgamma/dm = -(d' - cos(gamma) u) / (|m - P| sin gamma),
// dr/ds = -unit(o - s) (diffraction).  The forward's tiling is reused: a thread holds two
// microphones x KT bins of G in registers, the per-(path, mic) sums are reduced over the bin
// subtiles through shared memory, and every reduction runs in a fixed order (deterministic).
#include <math.h>

#include <algorithm>

#include "st_accum_dev.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

using namespace acc;

__device__ __forceinline__ u64 fadd2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fsub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

constexpr int kNV = 4;  // materials whose reflection gradient one launch accumulates

template <int KT, int KIND>
__global__ void __launch_bounds__(256) k_adjoint(const AccumArgs a, const AdjointArgs j, const Geom g) {
    extern __shared__ float4 smem4[];
    const int PT = g.PT, NS = g.NS, TP = g.TP, KB = g.KB, MP = g.MP;
    const Buf B0 = buf_at<KT>(smem4, g, 0), B1 = buf_at<KT>(smem4, g, 1);
    // after the two pipeline buffers: pd [3][PT][12], pv [3][PT], Cbuf [PT][NS][MP][5], Gbuf [PT][MP][6], mt
    float* pdb = reinterpret_cast<float*>(reinterpret_cast<char*>(smem4) + 2 * g.buf_bytes);
    int* pvb = reinterpret_cast<int*>(pdb + 3 * PT * 12);
    float* cbuf = reinterpret_cast<float*>(pvb + 3 * PT);
    float* gbuf = cbuf + (size_t)PT * NS * MP * 5;
    float* mt = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(gbuf + (size_t)PT * MP * 6) + 15) & ~uintptr_t(15));

    const int mb = blockIdx.x % g.n_mb, bb = blockIdx.x / g.n_mb;
    const int mic0 = mb * MP, kb = bb * KB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tp = tid % TP, s = tid / TP;

    const int64_t count = (int64_t)*a.d_count;
    const int64_t n_tiles = (count + PT - 1) / PT;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)blockIdx.y * per, t1 = min(n_tiles, t0 + per);

    // G of the thread's two microphones and KT bins, packed over the microphones
    u64 Gr[KT], Gi[KT];
    {
        const int m1 = mic0 + 2 * tp, m2 = m1 + 1;
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            const int k = kb + s * KT + kk;
            float2 g1 = make_float2(0.f, 0.f), g2 = make_float2(0.f, 0.f);
            if (k < a.F) {
                if (m1 < a.M) g1 = j.G[(int64_t)m1 * a.F + k];
                if (m2 < a.M) g2 = j.G[(int64_t)m2 * a.F + k];
            }
            Gr[kk] = pk2(g1.x, g2.x);
            Gi[kk] = pk2(g1.y, g2.y);
        }
    }
    float V[kNV][KT];
#pragma unroll
    for (int q = 0; q < kNV; ++q)
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) V[q][kk] = 0.0f;
    float dm[3] = {0.f, 0.f, 0.f}, de[3] = {0.f, 0.f, 0.f};  // thread tid < MP: mic mic0 + tid

    const float invNS = 1.0f / (float)NS, invKB = 1.0f / (float)KB;
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
                } else {
                    mt[e] = a.lid[(int64_t)mat * a.F + k];
                }
            }
        }
        load_paths<KIND>(a, PT, t0 * PT, count, pdb, pvb);
        if (t0 + 1 < t1) load_paths<KIND>(a, PT, (t0 + 1) * PT, count, pdb + PT * 12, pvb + PT);
        __syncthreads();
        produce<KT, KIND>(a, g, B0, pdb, pvb, mt, mic0, kb, invNS, invKB);
        __syncthreads();
    }
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int b = (int)((tile - t0) & 1);
        const int pb = (int)((tile - t0) % 3);  // path data of this tile
        const Buf& C = b ? B1 : B0;
        const Buf& Pn = b ? B0 : B1;
        float* pd = pdb + pb * PT * 12;
        const int* pv = pvb + pb * PT;
        // ---- A: tables of the next tile; reverse terms of this tile
        if (tile + 1 < t1) {
            const int nb = (int)((tile + 1 - t0) % 3);
            produce<KT, KIND>(a, g, Pn, pdb + nb * PT * 12, pvb + nb * PT, mt, mic0, kb, invNS, invKB);
        }
        for (int p = 0; p < PT; ++p) {
            const ulonglong2 z0 = C.za[((size_t)p * NS + s) * TP + tp];
            const u64* w = C.wst + ((size_t)p * TP + tp) * 4;
            const u64 w1r = w[0], w1i = w[1], w2r = w[2], w2i = w[3];
            const u64 nw2i = fmul2(w2i, pk2(-1.0f, -1.0f));
            const u64 ng = C.ngp[(size_t)p * TP + tp];
            u64 er = z0.x, ei = z0.y, orr = er, oi = ei;
            cmul2(orr, oi, w1r, w1i, fmul2(w1i, pk2(-1.0f, -1.0f)));
            u64 c0r = 0ull, c0i = 0ull, qr = 0ull, qi = 0ull, cg = 0ull;
            float y[KT];
            const ulonglong2* trow = reinterpret_cast<const ulonglong2*>(C.tab) + (size_t)p * KB + s;
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) {
                const ulonglong2 t = trow[kk * NS];
                u64 E;
                if (KIND == 0) {
                    const float2 arg = up2(ffma2(ng, t.y, t.x));
                    E = pk2(ex2(arg.x), ex2(arg.y));
                } else {
                    E = t.x;
                }
                const u64 zr = (kk & 1) ? orr : er, zi = (kk & 1) ? oi : ei;
                const u64 Tr = fmul2(E, zr), Ti = fmul2(E, zi);
                const u64 wr = ffma2(Gr[kk], Tr, fmul2(Gi[kk], Ti));        // Re(conj(G) T)
                const u64 wi = fsub2(fmul2(Gr[kk], Ti), fmul2(Gi[kk], Tr));  // Im(conj(G) T)
                c0r = fadd2(c0r, wr);
                c0i = fadd2(c0i, wi);
                qr = fadd2(qr, c0r);  // running sum of prefix sums: sum_kk kk w = KT C0 - Q
                qi = fadd2(qi, c0i);
                if (KIND == 0) cg = ffma2(t.y, wr, cg);
                const float2 wr2 = up2(wr);
                y[kk] = wr2.x + wr2.y;
                if (kk & 1) cmul2(orr, oi, w2r, w2i, nw2i); else cmul2(er, ei, w2r, w2i, nw2i);
            }
            // per (path, subtile, mic) partial sums for the position gradients
            if (j.do_pos) {
                const float2 C0r = up2(c0r), C0i = up2(c0i), Qr = up2(qr), Qi = up2(qi), Cg = up2(cg);
                float* cb = cbuf + (((size_t)p * NS + s) * MP + 2 * tp) * 5;
                cb[0] = C0r.x; cb[1] = C0i.x; cb[2] = KT * C0r.x - Qr.x; cb[3] = KT * C0i.x - Qi.x; cb[4] = Cg.x;
                cb[5] = C0r.y; cb[6] = C0i.y; cb[7] = KT * C0r.y - Qr.y; cb[8] = KT * C0i.y - Qi.y; cb[9] = Cg.y;
            }
            // reflection-coefficient sums for the materials of the path's chain
            if (KIND == 0 && j.do_k && pv[p]) {
                const uint32_t meta = __float_as_uint(pd[p * 12 + 8]);
                const int len = meta & 15, matj = (meta >> 8) & 255;
                const uint32_t c0 = __float_as_uint(pd[p * 12 + 9]), c1 = __float_as_uint(pd[p * 12 + 10]);
                float cnt[kNV] = {0.f, 0.f, 0.f, 0.f};
                if (a.reflection_mode == 1) {
                    const int q = matj - j.mat_base;
                    if (q >= 0 && q < kNV) cnt[q] = 1.0f;
                } else {
                    for (int q = 0; q < len; ++q) {
                        const int mq = ((q < 4 ? (c0 >> (8 * q)) : (c1 >> (8 * (q - 4)))) & 255) - j.mat_base;
#pragma unroll
                        for (int u = 0; u < kNV; ++u)
                            if (mq == u) cnt[u] += 1.0f;
                    }
                }
#pragma unroll
                for (int u = 0; u < kNV; ++u)
                    if (cnt[u] != 0.0f) {
#pragma unroll
                        for (int kk = 0; kk < KT; ++kk) V[u][kk] = fmaf(cnt[u], y[kk], V[u][kk]);
                    }
            }
        }
        __syncthreads();
        // ---- B: per (path, mic) gradient contributions; path data of tile + 2
        if (j.do_pos) {
            for (int e = tid; e < PT * MP; e += nthr) {
                const int p = e / MP, ml = e - p * MP;
                const int m = mic0 + ml;
                float* gb = gbuf + ((size_t)p * MP + ml) * 6;
                gb[0] = gb[1] = gb[2] = gb[3] = gb[4] = gb[5] = 0.0f;
                if (!pv[p] || m >= a.M) continue;
                // sums over the subtiles; C1 relative to kb
                float c0r = 0.f, c0i = 0.f, c1r = 0.f, c1i = 0.f, cgs = 0.f;
                for (int s_ = 0; s_ < NS; ++s_) {
                    const float* cb = cbuf + (((size_t)p * NS + s_) * MP + ml) * 5;
                    const float off = (float)(s_ * KT);
                    c0r += cb[0];
                    c0i += cb[1];
                    c1r += cb[2] + off * cb[0];
                    c1i += cb[3] + off * cb[1];
                    cgs += cb[4];
                }
                const float* d = pd + p * 12;
                const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
                const ff dist = dist_ff(mx, my, mz, d[0], d[1], d[2]);
                const ff rr = ff_add(ff{d[6], d[7]}, dist);
                const float r = rr.hi, inv = 1.0f / dist.hi;
                const float ux = (mx - d[0]) * inv, uy = (my - d[1]) * inv, uz = (mz - d[2]) * inv;
                // dL/dr = Re(D0 C0 + D1 C1)
                const float d0r = -2.0f / r - (j.a_0 + j.a_step * (float)kb), d0i = j.w_0 + j.w_step * (float)kb;
                const float d1r = -j.a_step, d1i = j.w_step;
                const float dLdr = (d0r * c0r - d0i * c0i) + (d1r * c1r - d1i * c1i);
                float gx = dLdr * ux, gy = dLdr * uy, gz = dLdr * uz;
                if (KIND == 0) {
                    const float dx = d[3], dy = d[4], dz = d[5];
                    const float cg = dx * ux + dy * uy + dz * uz;
                    const float cx = dy * uz - dz * uy, cy = dz * ux - dx * uz, cz = dx * uy - dy * ux;
                    const float sg = sqrtf(cx * cx + cy * cy + cz * cz);
                    const float gm = atan2f(sg, cg);
                    const float dLdg = -2.0f * gm * 0.69314718055994531f * cgs;
                    if (sg > 1e-20f) {
                        const float f = -dLdg / (dist.hi * sg);
                        gx += f * (dx - cg * ux);
                        gy += f * (dy - cg * uy);
                        gz += f * (dz - cg * uz);
                    }
                } else {
                    // dr/ds = -unit(o - s)
                    const float vx = d[0] - j.s[0], vy = d[1] - j.s[1], vz = d[2] - j.s[2];
                    const float iv = 1.0f / d[6];
                    gb[3] = -dLdr * vx * iv;
                    gb[4] = -dLdr * vy * iv;
                    gb[5] = -dLdr * vz * iv;
                }
                gb[0] = gx;
                gb[1] = gy;
                gb[2] = gz;
            }
        }
        if (tile + 2 < t1) {
            const int nb2 = (int)((tile + 2 - t0) % 3);
            load_paths<KIND>(a, PT, (tile + 2) * PT, count, pdb + nb2 * PT * 12, pvb + nb2 * PT);
        }
        __syncthreads();
        // ---- C: each microphone's thread accumulates its contributions in path order
        if (j.do_pos && tid < MP) {
            for (int p = 0; p < PT; ++p) {
                const float* gb = gbuf + ((size_t)p * MP + tid) * 6;
                for (int c = 0; c < 3; ++c) {
                    dm[c] += gb[c];
                    de[c] += gb[3 + c];
                }
            }
        }
    }
    // ---- outputs of this CTA
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    if (j.do_pos) {
        if (tid < MP && mic0 + tid < a.M) {
            float* o = j.mic_part + ((size_t)(blockIdx.y * g.n_bb + bb) * a.M + mic0 + tid) * 3;
            o[0] = dm[0];
            o[1] = dm[1];
            o[2] = dm[2];
        }
        __syncthreads();
        // emitter: fixed-order sum over the CTA's microphones
        float* red = cbuf;
        if (tid < MP) {
            red[tid * 3 + 0] = de[0];
            red[tid * 3 + 1] = de[1];
            red[tid * 3 + 2] = de[2];
        }
        __syncthreads();
        if (tid < 3) {
            float acc = 0.0f;
            for (int ml = 0; ml < MP; ++ml) acc += red[ml * 3 + tid];
            j.emit_part[(size_t)cta * 3 + tid] = acc;
        }
        __syncthreads();
    }
    if (KIND == 0 && j.do_k) {
        // V of the CTA's bins: fixed-order sum over the thread's microphone pairs
        float* vt = reinterpret_cast<float*>(smem4);  // [kNV][KT][NS][TP]
#pragma unroll
        for (int u = 0; u < kNV; ++u)
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) vt[(((size_t)u * KT + kk) * NS + s) * TP + tp] = V[u][kk];
        __syncthreads();
        for (int e = tid; e < kNV * KB; e += nthr) {
            const int u = e / KB, i = e - u * KB;
            const int kk = i / NS, s_ = i - kk * NS;
            const int k = kb + s_ * KT + kk;
            float acc = 0.0f;
            for (int q = 0; q < TP; ++q) acc += vt[(((size_t)u * KT + kk) * NS + s_) * TP + q];
            if (k < a.F) j.v_part[((size_t)(blockIdx.y * g.n_mb + mb) * kNV + u) * a.F + k] = acc;
        }
    }
}

// direct path: one thread per microphone, sequential over bins
__global__ void k_direct_adjoint(const DirectAccumArgs a, const float* qhi, const float* qlo, const float2* G,
                                 float* mic_out, float* emit_out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.M) return;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (a.vis[m]) {
        const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
        const ff r = dist_ff(mx, my, mz, a.s[0], a.s[1], a.s[2]);
        float dLdr = 0.0f;
        for (int k = 0; k < a.F; ++k) {
            const double f = a.F == 1 ? a.f_lo : a.f_lo + (double)k * a.df;
            const float alpha = (float)(a.a0 + a.a1 * (f / 1000.0));
            const float L = log2f(a.gain) - 2.0f * log2_ff(r) - alpha * r.hi * (3.3219280948873623f / 20.0f);
            const ff x = ff_mul(r, ff{qhi[k], qlo[k]});
            float sn, cs;
            sincospif(2.0f * ff_frac(x), &sn, &cs);
            const float A = exp2f(L);
            const float Tr = A * cs, Ti = A * sn;
            const float2 gk = G[(int64_t)m * a.F + k];
            const float wr = gk.x * Tr + gk.y * Ti, wi = gk.x * Ti - gk.y * Tr;
            const float dr = -2.0f / r.hi - alpha * (2.302585092994046f / 20.0f);
            const float di = (float)(2.0 * 3.141592653589793 * f / a.c);
            dLdr += dr * wr - di * wi;
        }
        const float iv = 1.0f / r.hi;
        gx = dLdr * (mx - a.s[0]) * iv;
        gy = dLdr * (my - a.s[1]) * iv;
        gz = dLdr * (mz - a.s[2]) * iv;
    }
    mic_out[3 * m] = gx;
    mic_out[3 * m + 1] = gy;
    mic_out[3 * m + 2] = gz;
    emit_out[3 * m] = -gx;
    emit_out[3 * m + 1] = -gy;
    emit_out[3 * m + 2] = -gz;
}

// V[u][k] = sum of the partial slices in order (one thread per (u, k)), written to slice 0's place
__global__ void k_v_reduce(float* v_part, int n_slices, int F) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kNV * F) return;
    float acc = 0.0f;
    for (int sl = 0; sl < n_slices; ++sl) acc += v_part[(size_t)sl * kNV * F + idx];
    v_part[idx] = acc;
}

// dk[mat][b] = sum_k V[mat][k] w_b(k) / k(mat, f_k) over the bins whose interpolation uses band b
__global__ void k_dk_contract(const float* V, int F, int mat_base, int n_mat_launch, int n_bands,
                              const float* band_hz, const float* kb_tab, double f_lo, double df, float* dk) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_mat_launch * n_bands) return;
    const int u = idx / n_bands, b = idx % n_bands;
    const int mat = mat_base + u;
    double acc = 0.0;
    for (int k = 0; k < F; ++k) {
        const double v = (double)V[(size_t)u * F + k];
        if (v == 0.0) continue;
        const double f = F == 1 ? f_lo : f_lo + (double)k * df;
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
                while (b0 + 1 < n_bands && (double)band_hz[b0 + 1] <= f) ++b0;
                if (b0 >= n_bands - 1) b0 = n_bands - 2;
                w = (f - (double)band_hz[b0]) / ((double)band_hz[b0 + 1] - (double)band_hz[b0]);
            }
        }
        double wb = 0.0;
        if (n_bands == 1) wb = 1.0;
        else if (b == b0) wb = 1.0 - w;
        else if (b == b0 + 1) wb = w;
        if (wb == 0.0) continue;
        const float* kr = kb_tab + (size_t)mat * n_bands;
        const double kv = n_bands == 1 ? (double)kr[0] : (1.0 - w) * (double)kr[b0] + w * (double)kr[b0 + 1];
        if (!(kv > 0.0)) continue;
        acc += v * wb / kv;
    }
    dk[(size_t)mat * n_bands + b] = (float)acc;
}

// positions: dmic[m] = sum of all partial slices in order; demit = sum of emitter slices in order
__global__ void k_pos_reduce(const float* mic_parts, int n_mic_slices, const float* emit_parts, int n_emit_slices,
                             int M, float* dmic, float* demit) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < 3 * M) {
        float acc = 0.0f;
        for (int sl = 0; sl < n_mic_slices; ++sl) acc += mic_parts[(size_t)sl * M * 3 + idx];
        if (dmic) dmic[idx] = acc;
    } else if (idx < 3 * M + 3) {
        const int c = idx - 3 * M;
        float acc = 0.0f;
        for (int sl = 0; sl < n_emit_slices; ++sl) acc += emit_parts[(size_t)sl * 3 + c];
        if (demit) demit[c] = acc;
    }
}

template <int KT, int KIND>
cudaError_t launch_adjoint(const AccumArgs& a, const AdjointArgs& j, const Geom& g, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_adjoint<KT, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)(g.n_mb * g.n_bb), (unsigned)a.n_chunks);
    note_launch();
    k_adjoint<KT, KIND><<<grid, g.TP * g.NS, adjoint_smem(g), s>>>(a, j, g);
    return cudaGetLastError();
}

}  // namespace

size_t adjoint_smem(const acc::Geom& g) {
    const size_t extra = 3 * (size_t)g.PT * 52 + (size_t)g.PT * g.NS * g.MP * 20 + (size_t)g.PT * g.MP * 24 + 16;
    const size_t vt = (size_t)kNV * g.KB * g.TP * 4;  // end-of-kernel reduction reuses the start of shared memory
    const size_t total = 2 * g.buf_bytes + extra + (g.mat_cached ? g.mat_bytes : 0) + 64;
    return std::max(total, vt + 64);
}

acc::Geom adjoint_geom(int M, int F, int n_mat) {
    // tile shape of the forward (8 bins per thread, 16 microphone pairs per CTA); paths per tile chosen
    // so the pipeline buffers plus the reduction buffers fit about 96 KB
    acc::Geom g = acc::make_geom(M, F, 8, n_mat, 16, 200 * 1024);
    const size_t per_path = (size_t)g.KB * 16 + (size_t)g.NS * g.TP * 16 + (size_t)g.TP * 40;
    const size_t per_tile = 2 * per_path + 3 * 52 + (size_t)g.NS * g.MP * 20 + (size_t)g.MP * 24;
    const size_t fixed = (g.mat_cached ? g.mat_bytes : 0) + 16 + 64 + 256;
    const size_t budget = 96 * 1024;
    g.PT = (int)std::max<size_t>(1, std::min<size_t>(8, budget > fixed ? (budget - fixed) / per_tile : 1));
    g.buf_bytes = (per_path * g.PT + 255) & ~size_t(255);
    g.smem = adjoint_smem(g);
    return g;
}

cudaError_t adjoint_launch(const AccumArgs& a, const AdjointArgs& j, const acc::Geom& g, cudaStream_t s) {
    return a.kind == 0 ? launch_adjoint<8, 0>(a, j, g, s) : launch_adjoint<8, 1>(a, j, g, s);
}

cudaError_t adjoint_direct(const DirectAccumArgs& a, const float* qhi, const float* qlo, const float2* G,
                           float* mic_out, float* emit_out, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    note_launch();
    k_direct_adjoint<<<(a.M + 63) / 64, 64, 0, s>>>(a, qhi, qlo, G, mic_out, emit_out);
    return cudaGetLastError();
}

cudaError_t adjoint_dk(const float* v_part, int n_slices, int F, int mat_base, int n_mat_launch, int n_bands,
                       const float* band_hz_dev, const float* k_dev, double f_lo, double df, float* dk, int n_mat,
                       cudaStream_t s) {
    (void)n_mat;
    const int n = n_mat_launch * n_bands;
    if (n <= 0) return cudaSuccess;
    float* v = const_cast<float*>(v_part);
    note_launch();
    k_v_reduce<<<(kNV * F + 127) / 128, 128, 0, s>>>(v, n_slices, F);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launch();
    k_dk_contract<<<(n + 63) / 64, 64, 0, s>>>(v, F, mat_base, n_mat_launch, n_bands, band_hz_dev, k_dev, f_lo, df, dk);
    return cudaGetLastError();
}

cudaError_t adjoint_pos(const float* mic_parts, int n_mic_slices, const float* emit_parts, int n_emit_slices, int M,
                        float* dmic, float* demit, cudaStream_t s) {
    note_launch();
    k_pos_reduce<<<(3 * M + 3 + 127) / 128, 128, 0, s>>>(mic_parts, n_mic_slices, emit_parts, n_emit_slices, M, dmic,
                                                        demit);
    return cudaGetLastError();
}

}  // namespace st
