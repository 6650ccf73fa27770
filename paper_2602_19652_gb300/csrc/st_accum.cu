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
// The phase never loses precision: only frac(f r / c) enters FP32, and the recurrence runs at most
// KT steps from an exactly reduced anchor.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>

#include "st_internal.cuh"

namespace st {

namespace {

// ---------------------------------------------------------------- float-float arithmetic
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return ff{s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = a + b;
    float e = b - (s - a);
    return ff{s, e};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = a * b;
    float e = fmaf(a, b, -p);
    return ff{p, e};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    float e = s.lo + (x.lo + y.lo);
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    ff p = two_prod(x.hi, y.hi);
    float e = p.lo + fmaf(x.hi, y.lo, x.lo * y.hi);
    return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.hi > 0.0f)) return ff{0.0f, 0.0f};
    float s = sqrtf(x.hi);
    ff p = two_prod(s, s);
    float d = (((x.hi - p.hi) - p.lo) + x.lo) / (2.0f * s);
    return fast_two_sum(s, d);
}
// |a - b| for float32 points, ~2^-44 relative
__device__ __forceinline__ ff dist_ff(float ax, float ay, float az, float bx, float by, float bz) {
    ff dx = two_sum(ax, -bx), dy = two_sum(ay, -by), dz = two_sum(az, -bz);
    ff sx = two_prod(dx.hi, dx.hi);
    sx.lo = fmaf(2.0f * dx.hi, dx.lo, sx.lo);
    ff sy = two_prod(dy.hi, dy.hi);
    sy.lo = fmaf(2.0f * dy.hi, dy.lo, sy.lo);
    ff sz = two_prod(dz.hi, dz.hi);
    sz.lo = fmaf(2.0f * dz.hi, dz.lo, sz.lo);
    return ff_sqrt(ff_add(ff_add(sx, sy), sz));
}
// fractional part in [-0.5, 0.5] of a non-negative float-float
__device__ __forceinline__ float ff_frac(ff x) {
    float n = rintf(x.hi);
    return (x.hi - n) + x.lo;
}
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float log2_ff(ff r) { return log2f(r.hi) + r.lo / (r.hi * 0.69314718055994531f); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

constexpr float kNegInf = -__builtin_huge_valf();

// ---------------------------------------------------------------- per-bin material tables
__global__ void k_tables(int32_t F, int32_t n_mat, int32_t n_bands, const float* band_hz, const float* kb,
                         const float* beta, const float* diff, double f_lo, double df, double c, float* lk, float* g2,
                         float* lid, float* qhi, float* qlo) {
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
    }
}

// ---------------------------------------------------------------- accumulator
// Packed FP32 pairs (fma/mul .f32x2, sm_100 and later): one 64-bit register holds the same
// quantity for two microphones, so every inner-loop instruction advances two terms.
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk2(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up2(u64 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 fmul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// (zr, zi) *= (wr, wi) for two microphones at once; nwi = -wi
__device__ __forceinline__ void cmul2(u64& zr, u64& zi, u64 wr, u64 wi, u64 nwi) {
    const u64 t1 = fmul2(zr, wr), t2 = fmul2(zi, wr);
    const u64 r = ffma2(zi, nwi, t1);
    zi = ffma2(zr, wi, t2);
    zr = r;
}

struct Geom {
    int TP, NS, MP, KB, PT;  // mic pairs per CTA (threads along x), subtiles, mics per CTA, bins per CTA, paths/tile
    int n_mb, n_bb;
    int mat_cached;          // material tables held in shared memory (n_mat small enough)
    size_t buf_bytes;        // one pipeline buffer (tables + anchors of PT paths)
    size_t smem;
};

// Shared memory: two pipeline buffers, each
//   tab [PT][KB] float4      per (path, bin): (log2 X, log2 X, g, g) specular, (X, X, -, -) diffraction,
//                            bin kb + s*KT + kk stored at i = kk*NS + s
//   za  [PT][NS][TP] ulonglong2  phasor at bin kb + s*KT of the two mics of pair tp (re pair, im pair)
//   wst [PT][TP][4] u64      one-bin step (re, im) and two-bin step (re, im) of the pair
//   ngp [PT][TP] u64         -gamma^2 of the pair
// then two path-data buffers pd [PT][12] + valid [PT], then the per-CTA material tables.
struct Buf {
    float4* tab;
    ulonglong2* za;
    u64* wst;
    u64* ngp;
};

template <int KT>
__device__ __forceinline__ Buf buf_at(float4* base, const Geom& g, int b) {
    Buf B;
    char* p = reinterpret_cast<char*>(base) + (size_t)b * g.buf_bytes;
    B.tab = reinterpret_cast<float4*>(p);
    B.za = reinterpret_cast<ulonglong2*>(B.tab + (size_t)g.PT * g.KB);
    B.wst = reinterpret_cast<u64*>(B.za + (size_t)g.PT * g.NS * g.TP);
    B.ngp = B.wst + (size_t)g.PT * g.TP * 4;
    return B;
}

// path data of one tile into pd / pv
template <int KIND>
__device__ __forceinline__ void load_paths(const AccumArgs& a, int PT, int64_t pbase, int64_t count, float* pd, int* pv) {
    for (int p = threadIdx.x; p < PT; p += blockDim.x) {
        const int64_t pi = pbase + p;
        const bool ok = pi < count;
        pv[p] = ok;
        float* d = pd + p * 12;
        if (ok) {
            d[0] = a.px[pi];
            d[1] = a.py[pi];
            d[2] = a.pz[pi];
            d[6] = a.rhi[pi];
            d[7] = a.rlo[pi];
            d[8] = __uint_as_float(a.meta[pi]);
            d[11] = a.dep ? a.dep[pi] : -1.0f;
            if (KIND == 0) {
                d[3] = a.dx[pi];
                d[4] = a.dy[pi];
                d[5] = a.dz[pi];
                d[9] = __uint_as_float(a.chain_lo[pi]);
                d[10] = __uint_as_float(a.chain_hi[pi]);
            }
        }
    }
}

// tables and anchors of one tile (reads pd / pv, writes buffer B)
template <int KT, int KIND>
__device__ __forceinline__ void produce(const AccumArgs& a, const Geom& g, const Buf& B, const float* pd, const int* pv,
                                        const float* mt, int mic0, int kb, float invNS, float invKB) {
    const int PT = g.PT, NS = g.NS, TP = g.TP, KB = g.KB, MP = g.MP;
    const bool cached = g.mat_cached > 0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    // 1a: per (path, bin) factors, written in table order.  With NS % 4 == 0 and the material tables in
    // shared memory, a thread builds four adjacent entries (same path and kk, subtiles s..s+3): one chain
    // decode, 128-bit loads of the material rows and four conflict-free 128-bit stores.
    if (cached && (NS & 3) == 0 && !a.etab) {
        const int KB4 = KB >> 2;
        const float invKB4 = 1.0f / (float)KB4;
        for (int e = tid; e < PT * KB4; e += nthr) {
            const int p = __float2int_rz(((float)e + 0.5f) * invKB4), i = (e - p * KB4) * 4;
            const int kk = __float2int_rz(((float)i + 0.5f) * invNS), s_ = i - kk * NS;
            float4 lx4 = make_float4(kNegInf, kNegInf, kNegInf, kNegInf), g4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (pv[p]) {
                const float* d = pd + p * 12;
                const uint32_t meta = __float_as_uint(d[8]);
                const int matj = (meta >> 8) & 255;
                if (KIND == 0) {
                    if (a.reflection_mode == 1) {
                        lx4 = *reinterpret_cast<const float4*>(mt + matj * KB + i);
                    } else {
                        const int len = meta & 15;
                        const uint32_t c0 = __float_as_uint(d[9]), c1 = __float_as_uint(d[10]);
                        lx4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        for (int q = 0; q < len; ++q) {
                            const int mq = (q < 4 ? (c0 >> (8 * q)) : (c1 >> (8 * (q - 4)))) & 255;
                            const float4 v = *reinterpret_cast<const float4*>(mt + mq * KB + i);
                            lx4.x += v.x;
                            lx4.y += v.y;
                            lx4.z += v.z;
                            lx4.w += v.w;
                        }
                    }
                    g4 = *reinterpret_cast<const float4*>(mt + a.n_mat_tab * KB + matj * KB + i);
                } else {
                    lx4 = *reinterpret_cast<const float4*>(mt + matj * KB + i);
                }
                // bins beyond the grid contribute nothing
                const int k0 = kb + s_ * KT + kk;
                if (k0 >= a.F) lx4.x = kNegInf;
                if (k0 + KT >= a.F) lx4.y = kNegInf;
                if (k0 + 2 * KT >= a.F) lx4.z = kNegInf;
                if (k0 + 3 * KT >= a.F) lx4.w = kNegInf;
            }
            float4* dst = B.tab + (size_t)p * KB + i;
            if (KIND == 0) {
                dst[0] = make_float4(lx4.x, lx4.x, g4.x, g4.x);
                dst[1] = make_float4(lx4.y, lx4.y, g4.y, g4.y);
                dst[2] = make_float4(lx4.z, lx4.z, g4.z, g4.z);
                dst[3] = make_float4(lx4.w, lx4.w, g4.w, g4.w);
            } else {
                const float x0 = ex2(lx4.x), x1 = ex2(lx4.y), x2 = ex2(lx4.z), x3 = ex2(lx4.w);
                dst[0] = make_float4(x0, x0, 0.f, 0.f);
                dst[1] = make_float4(x1, x1, 0.f, 0.f);
                dst[2] = make_float4(x2, x2, 0.f, 0.f);
                dst[3] = make_float4(x3, x3, 0.f, 0.f);
            }
        }
    } else {
        for (int e = tid; e < PT * KB; e += nthr) {
            const int p = __float2int_rz(((float)e + 0.5f) * invKB), i = e - p * KB;
            const int kk = __float2int_rz(((float)i + 0.5f) * invNS), s_ = i - kk * NS;
            const int k = kb + s_ * KT + kk;
            float lx = kNegInf, gg = 0.0f;
            if (pv[p] && k < a.F) {
                const float* d = pd + p * 12;
                const uint32_t meta = __float_as_uint(d[8]);
                const int matj = (meta >> 8) & 255;
                const int nm = a.n_mat_tab;
                if (KIND == 0) {
                    if (a.reflection_mode == 1) {
                        lx = cached ? mt[matj * KB + i] : a.lk[(int64_t)matj * a.F + k];
                    } else {
                        const int len = meta & 15;
                        const uint32_t c0 = __float_as_uint(d[9]), c1 = __float_as_uint(d[10]);
                        float acc = 0.0f;
                        for (int q = 0; q < len; ++q) {
                            const int mq = (q < 4 ? (c0 >> (8 * q)) : (c1 >> (8 * (q - 4)))) & 255;
                            acc += cached ? mt[mq * KB + i] : a.lk[(int64_t)mq * a.F + k];
                        }
                        lx = acc;
                    }
                    gg = cached ? mt[nm * KB + matj * KB + i] : a.g2[(int64_t)matj * a.F + k];
                } else {
                    lx = cached ? mt[matj * KB + i] : a.lid[(int64_t)matj * a.F + k];
                }
                if (a.etab && d[11] >= 0.0f) {
                    const float x = d[11];
                    const int it = min((int)x, a.n_theta - 2);
                    const float w = x - (float)it;
                    const float de = (1.0f - w) * a.etab[(int64_t)it * a.F + k] + w * a.etab[(int64_t)(it + 1) * a.F + k];
                    lx += de > 0.0f ? log2f(de) : kNegInf;
                }
            }
            if (KIND == 0) {
                B.tab[(size_t)p * KB + i] = make_float4(lx, lx, gg, gg);
            } else {
                const float x = ex2(lx);
                B.tab[(size_t)p * KB + i] = make_float4(x, x, 0.0f, 0.0f);
            }
        }
    }
    // 1b: per (path, mic) anchors
    for (int e = tid; e < PT * MP; e += nthr) {
        const int p = e / MP, ml = e - p * MP;
        const int pair = ml >> 1, half = ml & 1;
        const int m = mic0 + ml;
        float* zf = reinterpret_cast<float*>(B.za + (size_t)p * NS * TP + pair);
        float* wf = reinterpret_cast<float*>(B.wst + ((size_t)p * TP + pair) * 4);
        float* nf = reinterpret_cast<float*>(B.ngp + (size_t)p * TP + pair);
        if (!pv[p] || m >= a.M) {
            for (int s_ = 0; s_ < NS; ++s_) {
                zf[(size_t)s_ * TP * 4 + half] = 0.0f;
                zf[(size_t)s_ * TP * 4 + 2 + half] = 0.0f;
            }
            for (int q = 0; q < 4; ++q) wf[2 * q + half] = 0.0f;
            nf[half] = 0.0f;
            continue;
        }
        const float* d = pd + p * 12;
        const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
        const ff dist = dist_ff(mx, my, mz, d[0], d[1], d[2]);
        const ff r = ff_add(ff{d[6], d[7]}, dist);
        float gam2 = 0.0f;
        if (KIND == 0) {
            const float inv = 1.0f / dist.hi;
            const float ux = (mx - d[0]) * inv, uy = (my - d[1]) * inv, uz = (mz - d[2]) * inv;
            const float cg = d[3] * ux + d[4] * uy + d[5] * uz;
            const float cx = d[4] * uz - d[5] * uy, cy = d[5] * ux - d[3] * uz, cz = d[3] * uy - d[4] * ux;
            const float gm = atan2f(sqrtf(cx * cx + cy * cy + cz * cz), cg);
            gam2 = gm * gm;
        }
        const float rh = r.hi;
        const float L0 = -2.0f * log2_ff(r) + rh * (a.atm2_0 + a.atm2_step * (float)kb);
        const ff x0 = ff_mul(r, ff{a.qhi[min(kb, a.F - 1)], a.qlo[min(kb, a.F - 1)]});
        float s0, c0;
        sincospif(2.0f * ff_frac(x0), &s0, &c0);
        const float A0 = ex2(L0);
        float2 z = make_float2(A0 * c0, A0 * s0);
        const ff xs = ff_mul(r, ff{a.dq_hi, a.dq_lo});
        float s1, c1;
        sincospif(2.0f * ff_frac(xs), &s1, &c1);
        const float a1 = ex2(rh * a.atm2_step);
        const float2 W1 = make_float2(a1 * c1, a1 * s1);
        const float2 W2 = cmul(W1, W1);  // two bins
        wf[0 + half] = W1.x;
        wf[2 + half] = W1.y;
        wf[4 + half] = W2.x;
        wf[6 + half] = W2.y;
        nf[half] = -gam2;
        float2 WK = W2;  // KT bins by repeated squaring (KT is a power of two)
        for (int q = 2; q < KT; q *= 2) WK = cmul(WK, WK);
        for (int s_ = 0; s_ < NS; ++s_) {
            zf[(size_t)s_ * TP * 4 + half] = z.x;
            zf[(size_t)s_ * TP * 4 + 2 + half] = z.y;
            z = cmul(z, WK);
        }
    }
}

template <int KT, int KIND>
__global__ void __launch_bounds__(256) k_accum(const AccumArgs a, const Geom g) {
    static_assert((KT & (KT - 1)) == 0 && KT >= 2, "KT must be a power of two");
    extern __shared__ float4 smem4[];
    const int PT = g.PT, NS = g.NS, TP = g.TP, KB = g.KB, MP = g.MP;
    const Buf B0 = buf_at<KT>(smem4, g, 0), B1 = buf_at<KT>(smem4, g, 1);
    float* pdb = reinterpret_cast<float*>(reinterpret_cast<char*>(smem4) + 2 * g.buf_bytes);  // [2][PT][12]
    int* pvb = reinterpret_cast<int*>(pdb + 2 * PT * 12);                                       // [2][PT]
    // material tables: 16-byte aligned for the 128-bit loads of phase 1a
    float* mt = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(pvb + 2 * PT) + 15) & ~uintptr_t(15));

    const int mb = blockIdx.x % g.n_mb, bb = blockIdx.x / g.n_mb;
    const int mic0 = mb * MP, kb = bb * KB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tp = tid % TP, s = tid / TP;

    const int64_t count = (int64_t)*a.d_count;
    const int64_t n_tiles = (count + PT - 1) / PT;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)blockIdx.y * per, t1 = min(n_tiles, t0 + per);

    u64 Sr[KT], Si[KT];
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) Sr[kk] = Si[kk] = 0ull;

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
    // software pipeline: consume tile t from buffer b while producing tile t+1 into buffer b^1
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int b = (int)((tile - t0) & 1);
        const Buf& C = b ? B1 : B0;
        const Buf& Pn = b ? B0 : B1;
        if (tile + 1 < t1) {
            const int nb = b ^ 1;  // path data of tile+1 sits in pd buffer nb
            produce<KT, KIND>(a, g, Pn, pdb + nb * PT * 12, pvb + nb * PT, mt, mic0, kb, invNS, invKB);
        }
        for (int p = 0; p < PT; ++p) {
            const ulonglong2 z0 = C.za[((size_t)p * NS + s) * TP + tp];
            const u64* w = C.wst + ((size_t)p * TP + tp) * 4;
            const u64 w1r = w[0], w1i = w[1], w2r = w[2], w2i = w[3];
            const u64 nw2i = fmul2(w2i, pk2(-1.0f, -1.0f));
            const u64 ng = C.ngp[(size_t)p * TP + tp];
            u64 er = z0.x, ei = z0.y;  // even chain: bins 0, 2, 4, ...
            u64 orr = er, oi = ei;     // odd chain: bins 1, 3, 5, ...
            cmul2(orr, oi, w1r, w1i, fmul2(w1i, pk2(-1.0f, -1.0f)));
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
        if (tile + 2 < t1) {  // pd buffer b held tile's path data, used by produce(tile) one step ago
            load_paths<KIND>(a, PT, (tile + 2) * PT, count, pdb + b * PT * 12, pvb + b * PT);
        }
        __syncthreads();
    }
    // ---- partial spectra of this chunk
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int m = mic0 + 2 * tp + h;
        if (m >= a.M) continue;
        float2* out = a.partial + ((size_t)blockIdx.y * a.M + m) * a.F;
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            const int k = kb + s * KT + kk;
            const float2 re = up2(Sr[kk]), im = up2(Si[kk]);
            if (k < a.F) out[k] = h == 0 ? make_float2(re.x, im.x) : make_float2(re.y, im.y);
        }
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
__global__ void k_direct_accum(const DirectAccumArgs a, const float* qhi, const float* qlo) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.M * a.F) return;
    const int m = (int)(idx / a.F), k = (int)(idx % a.F);
    float2 v = make_float2(0.0f, 0.0f);
    if (a.vis[m]) {
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
        const float A = exp2f(L);
        v = make_float2(A * cs, A * sn);
    }
    a.out[idx] = v;
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
                              float* rhi, float* rlo, uint32_t* chl, uint32_t* chh, uint32_t* meta, float* dep) {
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
            const uint32_t mq = (uint32_t)g.tri_mat[g.rec_tri[ray * g.B + q]] & 255u;
            if (q < 4) lo |= mq << (8 * q); else hi |= mq << (8 * (q - 4));
            matj = (int)mq;
        }
        chl[c] = lo;
        chh[c] = hi;
        meta[c] = (uint32_t)(j + 1) | ((uint32_t)matj << 8);
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
        meta[c] = ((uint32_t)g.tri_mat[g.cand_tri[i]] & 255u) << 8;
        if (g.has_etab) {
            const float vx = ox - g.s[0], vy = oy - g.s[1], vz = oz - g.s[2];
            const float cth = (g.fwd[0] * vx + g.fwd[1] * vy + g.fwd[2] * vz) / r.hi;
            dep[c] = acosf(fminf(1.0f, fmaxf(-1.0f, cth))) * g.inv_dtheta;
        } else {
            dep[c] = -1.0f;
        }
    }
}

// tp_max: mic pairs per CTA at most; budget: shared-memory bytes per CTA
Geom make_geom(int M, int F, int KT, int n_mat, int tp_max = 8, size_t budget = 96 * 1024) {
    Geom g;
    const int pairs = (M + 1) / 2;
    const int ns_need = (F + KT - 1) / KT;
    g.TP = std::max(1, std::min(pairs, tp_max));
    g.NS = std::max(1, std::min(ns_need, 256 / g.TP));
    g.TP = std::max(1, std::min(pairs, 256 / g.NS));
    g.MP = 2 * g.TP;
    g.KB = g.NS * KT;
    g.n_mb = (M + g.MP - 1) / g.MP;
    g.n_bb = (F + g.KB - 1) / g.KB;
    const size_t per_path = (size_t)g.KB * 16 + (size_t)g.NS * g.TP * 16 + (size_t)g.TP * 40;
    const size_t mat_bytes = (size_t)2 * n_mat * g.KB * 4;
    g.mat_cached = mat_bytes <= 24 * 1024 ? 1 : 0;
    const size_t fixed = g.mat_cached ? mat_bytes : 0;
    const size_t avail = budget > fixed + 4096 ? budget - fixed : 4096;
    g.PT = (int)std::min<size_t>(8, std::max<size_t>(1, avail / (2 * per_path + 2 * 52)));
    g.buf_bytes = (per_path * g.PT + 255) & ~size_t(255);
    g.smem = 2 * g.buf_bytes + 2 * (size_t)g.PT * 52 + 16 + fixed + 64;  // 16: alignment of the material tables
    return g;
}

// accumulator tile shape: mic pairs per CTA and shared-memory budget (set by the tuner or ST_ACCUM_TILE="tp,kb")
int g_tile_tp = 16;
size_t g_tile_budget = 96 * 1024;
int g_tile_kt = 16;
bool g_tile_env_read = false;

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
    }
}

template <int KT, int KIND>
cudaError_t launch_accum(const AccumArgs& a, cudaStream_t s) {
    read_tile_env();
    const Geom g = make_geom(a.M, a.F, KT, a.n_mat_tab, g_tile_tp, g_tile_budget);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_accum<KT, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)(g.n_mb * g.n_bb), (unsigned)a.n_chunks);
    note_launch();
    k_accum<KT, KIND><<<grid, g.TP * g.NS, g.smem, s>>>(a, g);
    return cudaGetLastError();
}

}  // namespace

int32_t accum_chunks(int64_t n_paths_hint, int32_t M, int32_t F, int32_t n_mat) {
    read_tile_env();
    const Geom g = make_geom(M, F, g_tile_kt, n_mat, g_tile_tp, g_tile_budget);
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
                                                    ptr<float>(T.qlo));
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(s);  // the staging buffer is freed below
    release(mt);
    if (e != cudaSuccess) return e;
    if (e2 != cudaSuccess) return e2;
    T.F = F;
    T.n_mat = n_mat;
    T.f_lo = f_lo;
    T.df = df;
    T.c = c;
    T.a0 = a0;
    T.a1 = a1;
    return cudaSuccess;
}

cudaError_t accumulate(const AccumArgs& a, cudaStream_t s) {
    read_tile_env();
    if (g_tile_kt == 8) return a.kind == 0 ? launch_accum<8, 0>(a, s) : launch_accum<8, 1>(a, s);
    return a.kind == 0 ? launch_accum<16, 0>(a, s) : launch_accum<16, 1>(a, s);
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

cudaError_t gather_specular(const GatherArgs& g, cudaStream_t s) {
    PathList& P = *g.out;
    note_launch();
    k_gather_spec<<<grid_for(g.N * g.B, 256), 256, 0, s>>>(
        g, ptr<float>(P.px), ptr<float>(P.py), ptr<float>(P.pz), ptr<float>(P.dx), ptr<float>(P.dy), ptr<float>(P.dz),
        ptr<float>(P.rhi), ptr<float>(P.rlo), ptr<uint32_t>(P.chain_lo), ptr<uint32_t>(P.chain_hi),
        ptr<uint32_t>(P.meta), ptr<float>(P.dep));
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

}  // namespace st
