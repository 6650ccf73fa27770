// Device code shared by the spectrum accumulator and its adjoint: float-float arithmetic, packed
// FP32 pairs, the CTA tile geometry and the producer of per-tile tables and anchors.
#pragma once

#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "st_internal.cuh"

namespace st {
namespace acc {

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
    // the correction is ~2^-24 of s: a reciprocal good to a few ulp keeps the sum to ~2^-46
    float d = (((x.hi - p.hi) - p.lo) + x.lo) * __fdividef(0.5f, s);
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
__device__ __forceinline__ float log2_ff(ff r) { return log2f(r.hi) + __fdividef(r.lo, r.hi * 0.69314718055994531f); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

constexpr float kNegInf = -__builtin_huge_valf();

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
    int NB;                  // receiver directivity bands held per (path, mic); 0 = omni receivers
    int ADJ;                 // adjoint layout: per (path, pair) position-gradient vectors after ngp
    int mat_cached;          // material tables held in shared memory (n_mat small enough)
    int mat_direct;          // diffraction without an emitter table: the term loop reads the per-(material, bin)
                             // factor from the cached material table, at the row offset the producer leaves in
                             // ngp; no per-(path, bin) table (tab has no space in the buffers)
    size_t mat_bytes;        // their size
    size_t buf_bytes;        // one pipeline buffer (tables + anchors of PT paths)
    size_t smem;
};

// Shared memory: two pipeline buffers, each
//   tab [PT][KB] float2      per (path, bin): (log2 X, g) specular, (X, X) diffraction,
//                            bin kb + s*KT + kk stored at i = kk*NS + s
//   za  [PT][NS][TP] ulonglong2  phasor at bin kb + s*KT of the two mics of pair tp (re pair, im pair)
//   wst [PT][4][TP] u64      one-bin step re, im and two-bin step re, im of the pair (component-major)
//   ngp [PT][TP] u64         -gamma^2 of the pair (diffraction, mat_direct: the path's material row offset)
//   adj [PT][TP][7] u64      (adjoint only) unit(m - P) xyz, lobe-angle vector xyz (specular) or
//                            -unit(o - s) xyz (diffraction), 1 / r of the pair
// then two path-data buffers pd [PT][12] + valid [PT], then the per-CTA material tables.
struct Buf {
    float4* tab;
    ulonglong2* za;
    u64* wst;
    u64* ngp;
    u64* adj;
    float* dband;  // [PT][MP][NB] receiver directivity band values (directional receivers only)
};

template <int KT>
__device__ __forceinline__ Buf buf_at(float4* base, const Geom& g, int b) {
    Buf B;
    char* p = reinterpret_cast<char*>(base) + (size_t)b * g.buf_bytes;
    B.tab = reinterpret_cast<float4*>(p);
    B.za = reinterpret_cast<ulonglong2*>(p + (g.mat_direct ? (size_t)0 : (size_t)g.PT * g.KB * 8));
    B.wst = reinterpret_cast<u64*>(B.za + (size_t)g.PT * g.NS * g.TP);
    B.ngp = B.wst + (size_t)g.PT * g.TP * 4;
    B.adj = B.ngp + (size_t)g.PT * g.TP;
    B.dband = reinterpret_cast<float*>(B.adj + (g.ADJ ? (size_t)g.PT * g.TP * 7 : 0));
    return B;
}

// Receiver directivity: band values of microphone m's table for the arrival direction v (world frame,
// from the microphone towards the point the sound comes from): rotate into the microphone frame by the
// conjugate of its orientation, azimuth atan2(y, x) on the periodic grid -pi + 2 pi i / n_az, elevation
// asin(z) on -pi/2 + pi j / (n_el - 1), bilinear in (az, el).
// (out[b * stride] for band b)
__device__ __forceinline__ void mic_bands(const AccumArgs& a, int m, float vx, float vy, float vz, float* out, int NB,
                                          int stride = 1) {
    const float l = sqrtf(vx * vx + vy * vy + vz * vz);
    float x = vx / l, y = vy / l, z = vz / l;
    if (a.mic_q) {
        const float* q = a.mic_q + 4 * m;
        const float qw = q[0], qx = -q[1], qy = -q[2], qz = -q[3];
        const float tx = 2.0f * (qy * z - qz * y), ty = 2.0f * (qz * x - qx * z), tz = 2.0f * (qx * y - qy * x);
        const float rx = x + qw * tx + (qy * tz - qz * ty), ry = y + qw * ty + (qz * tx - qx * tz),
                    rz = z + qw * tz + (qx * ty - qy * tx);
        x = rx;
        y = ry;
        z = rz;
    }
    const float az = atan2f(y, x), el = asinf(fminf(1.0f, fmaxf(-1.0f, z)));
    const float gx = (az + 3.14159265358979f) * (0.15915494309189535f * (float)a.n_az);
    const float fx = floorf(gx);
    const float wa = gx - fx;
    int i0 = (int)fx % a.n_az;
    if (i0 < 0) i0 += a.n_az;
    const int i1 = (i0 + 1) % a.n_az;
    const float gy = (el + 1.5707963267948966f) * (0.3183098861837907f * (float)(a.n_el - 1));
    int j0 = (int)floorf(gy);
    j0 = max(0, min(j0, a.n_el - 2));
    const float wb = gy - (float)j0;
    const float* T = a.mic_tab + (size_t)m * a.n_el * a.n_az * NB;
    const float* t00 = T + ((size_t)j0 * a.n_az + i0) * NB;
    const float* t01 = T + ((size_t)j0 * a.n_az + i1) * NB;
    const float* t10 = T + ((size_t)(j0 + 1) * a.n_az + i0) * NB;
    const float* t11 = T + ((size_t)(j0 + 1) * a.n_az + i1) * NB;
    for (int b = 0; b < NB; ++b) {
        const float lo = (1.0f - wa) * t00[b] + wa * t01[b];
        const float hi = (1.0f - wa) * t10[b] + wa * t11[b];
        out[b * stride] = (1.0f - wb) * lo + wb * hi;
    }
}

// path data of one tile into pd / pv
template <int KIND>
__device__ __forceinline__ void load_paths(const AccumArgs& a, int PT, int64_t pbase, int64_t count, float* pd, int* pv) {
    const int64_t base = a.d_base ? (int64_t)*a.d_base : 0;  // first path of this launch
    for (int p = threadIdx.x; p < PT; p += blockDim.x) {
        const int64_t rel = pbase + p;
        const bool ok = rel < count;
        const int64_t pi = base + rel;
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

// asynchronous 4-byte global -> shared copies (cp.async): the issuing thread does not wait for the data;
// cp_async_wait_all before the barrier that publishes the tile
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// path data of one tile into pd / pv as load_paths does, one thread per path, copied asynchronously: the
// copies are in flight while the tile phase runs; cp_async_wait_all before the barrier that publishes them
template <int KIND>
__device__ __forceinline__ void load_paths_cp(const AccumArgs& a, int PT, int64_t pbase, int64_t count, float* pd,
                                              int* pv) {
    const int64_t base = a.d_base ? (int64_t)*a.d_base : 0;
    for (int p = threadIdx.x; p < PT; p += blockDim.x) {
        const int64_t rel = pbase + p;
        const bool ok = rel < count;
        pv[p] = ok;
        if (!ok) continue;
        const int64_t pi = base + rel;
        float* d = pd + p * 12;
        cp_async4(d + 0, a.px + pi);
        cp_async4(d + 1, a.py + pi);
        cp_async4(d + 2, a.pz + pi);
        cp_async4(d + 6, a.rhi + pi);
        cp_async4(d + 7, a.rlo + pi);
        cp_async4(d + 8, a.meta + pi);
        if (a.dep) cp_async4(d + 11, a.dep + pi); else d[11] = -1.0f;
        if (KIND == 0) {
            cp_async4(d + 3, a.dx + pi);
            cp_async4(d + 4, a.dy + pi);
            cp_async4(d + 5, a.dz + pi);
            cp_async4(d + 9, a.chain_lo + pi);
            cp_async4(d + 10, a.chain_hi + pi);
        }
    }
    cp_async_commit();
}

// path data of one tile into pd / pv as load_paths does, with the words spread over the CTA's threads
// and copied asynchronously (the copies overlap the tile phase that issues them)
template <int KIND>
__device__ __forceinline__ void load_paths_async(const AccumArgs& a, int PT, int64_t pbase, int64_t count, float* pd,
                                                 int* pv) {
    const int64_t base = a.d_base ? (int64_t)*a.d_base : 0;
    for (int e = threadIdx.x; e < PT * 12; e += blockDim.x) {
        const int p = e / 12, k = e - p * 12;
        const int64_t rel = pbase + p;
        const bool ok = rel < count;
        if (k == 0) pv[p] = ok;
        if (!ok) continue;  // the words of an invalid path are never read
        const int64_t pi = base + rel;
        float* d = pd + p * 12 + k;
        const float* src = nullptr;
        switch (k) {
            case 0: src = a.px + pi; break;
            case 1: src = a.py + pi; break;
            case 2: src = a.pz + pi; break;
            case 3: src = KIND == 0 ? a.dx + pi : nullptr; break;
            case 4: src = KIND == 0 ? a.dy + pi : nullptr; break;
            case 5: src = KIND == 0 ? a.dz + pi : nullptr; break;
            case 6: src = a.rhi + pi; break;
            case 7: src = a.rlo + pi; break;
            case 8: src = reinterpret_cast<const float*>(a.meta + pi); break;
            case 9: src = KIND == 0 ? reinterpret_cast<const float*>(a.chain_lo + pi) : nullptr; break;
            case 10: src = KIND == 0 ? reinterpret_cast<const float*>(a.chain_hi + pi) : nullptr; break;
            default:
                if (a.dep) src = a.dep + pi; else *d = -1.0f;
                break;
        }
        if (src) cp_async4(d, src);
    }
    cp_async_commit();
}

// Scalar values of microphone mic0 + ml for path p of the tile: writes its half of the pair's step words, lobe
// (or material row) word, receiver band values and, in the adjoint, gradient vectors; returns its phasor at the
// CTA's first bin and the step over one subtile (KT bins), both zero for a microphone the path does not reach.
template <int KT, int KIND, int ADJ>
__device__ __forceinline__ void anchor_mic(const AccumArgs& a, const Geom& g, const Buf& B, const float* pd,
                                           const int* pv, int p, int ml, int mic0, int kb, const float* es,
                                           int64_t pglob, float2* z_out, float2* wk_out) {
    const int TP = g.TP, KB = g.KB, MP = g.MP;
    const int pair = ml >> 1, half = ml & 1;
    const int m = mic0 + ml;
    float* wf = reinterpret_cast<float*>(B.wst + (size_t)p * 4 * TP + pair);  // component c at wf[2 TP c]
    float* nf = reinterpret_cast<float*>(B.ngp + (size_t)p * TP + pair);
    // (per-microphone receiver test: a microphone that does not see the path gets a zero anchor)
    if (!pv[p] || m >= a.M || (a.mask && !((a.mask[pglob + p] >> m) & 1ull))) {
        *z_out = make_float2(0.0f, 0.0f);
        *wk_out = make_float2(0.0f, 0.0f);
        for (int q = 0; q < 4; ++q) wf[2 * TP * q + half] = 0.0f;
        nf[half] = 0.0f;
        for (int b = 0; b < g.NB; ++b) B.dband[((size_t)p * MP + ml) * g.NB + b] = 0.0f;
        if (ADJ) {
            float* af = reinterpret_cast<float*>(B.adj + ((size_t)p * TP + pair) * 7);
            for (int q = 0; q < 7; ++q) af[2 * q + half] = 0.0f;
        }
        return;
    }
    const float* d = pd + p * 12;
    const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
    const ff dist = dist_ff(mx, my, mz, d[0], d[1], d[2]);
    const ff r = ff_add(ff{d[6], d[7]}, dist);
    if (g.NB > 0) mic_bands(a, m, d[0] - mx, d[1] - my, d[2] - mz, B.dband + ((size_t)p * MP + ml) * g.NB, g.NB);
    float gam2 = 0.0f;
    if (KIND == 0 || ADJ) {
        const float inv = __fdividef(1.0f, dist.hi);
        const float ux = (mx - d[0]) * inv, uy = (my - d[1]) * inv, uz = (mz - d[2]) * inv;
        float* af = reinterpret_cast<float*>(B.adj + ((size_t)p * TP + pair) * 7);
        if (KIND == 0) {
            const float cg = d[3] * ux + d[4] * uy + d[5] * uz;
            const float cx = d[4] * uz - d[5] * uy, cy = d[5] * ux - d[3] * uz, cz = d[3] * uy - d[4] * ux;
            const float sg = sqrtf(cx * cx + cy * cy + cz * cz);
            const float gm = atan2f(sg, cg);
            gam2 = gm * gm;
            if (ADJ) {
                // d gamma / d m = -(d' - cos(gamma) u) / (|m - P| sin gamma); with dL/dgamma =
                // -2 ln2 gamma sum_k g_k Re w the microphone gradient gains (sum_k g_k Re w) times this vector
                const float f = sg > 1e-20f ? 2.0f * 0.69314718055994531f * gm / (dist.hi * sg) : 0.0f;
                af[6 + half] = f * (d[3] - cg * ux);
                af[8 + half] = f * (d[4] - cg * uy);
                af[10 + half] = f * (d[5] - cg * uz);
            }
        } else if (ADJ) {
            const float iv = 1.0f / d[6];  // -unit(o - s): d r / d s of a diffraction path
            af[6 + half] = -((d[0] - es[0]) * iv);
            af[8 + half] = -((d[1] - es[1]) * iv);
            af[10 + half] = -((d[2] - es[2]) * iv);
        }
        if (ADJ) {
            af[0 + half] = ux;
            af[2 + half] = uy;
            af[4 + half] = uz;
        }
    }
    const float rh = r.hi;
    if (ADJ) reinterpret_cast<float*>(B.adj + ((size_t)p * TP + pair) * 7)[12 + half] = 1.0f / rh;
    const float L0 = -2.0f * log2_ff(r) + rh * (a.atm2_0 + a.atm2_step * (float)kb);
    const ff x0 = ff_mul(r, ff{a.qhi[min(kb, a.F - 1)], a.qlo[min(kb, a.F - 1)]});
    float s0, c0;
    sincospif(2.0f * ff_frac(x0), &s0, &c0);
    const float A0 = ex2(L0);
    const float2 z = make_float2(A0 * c0, A0 * s0);
    const ff xs = ff_mul(r, ff{a.dq_hi, a.dq_lo});
    float s1, c1;
    sincospif(2.0f * ff_frac(xs), &s1, &c1);
    const float a1 = ex2(rh * a.atm2_step);
    const float2 W1 = make_float2(a1 * c1, a1 * s1);
    const float2 W2 = cmul(W1, W1);  // two bins
    wf[0 + half] = W1.x;
    wf[2 * TP + half] = W1.y;
    wf[4 * TP + half] = W2.x;
    wf[6 * TP + half] = W2.y;
    if (KIND == 1 && g.mat_direct) {  // offset of the path's row in the material table (term loop)
        const int matp = min((int)((__float_as_uint(d[8]) >> 8) & 255u), a.n_mat_tab - 1);
        reinterpret_cast<int*>(nf)[half] = matp * KB;
    } else {
        nf[half] = -gam2;
    }
    float2 WK = W2;  // KT bins by repeated squaring (KT is a power of two)
    for (int q = 2; q < KT; q *= 2) WK = cmul(WK, WK);
    *z_out = z;
    *wk_out = WK;
}

// tables and anchors of one tile (reads pd / pv, writes buffer B); ADJ: also the position-gradient
// vectors of the adjoint (es = emitter position, diffraction only); SPLIT: see below
template <int KT, int KIND, int ADJ = 0, int SPLIT = 0>
__device__ __forceinline__ void produce(const AccumArgs& a, const Geom& g, const Buf& B, const float* pd, const int* pv,
                                        const float* mt, int mic0, int kb, float invNS, float invKB,
                                        const float* es = nullptr, int64_t pglob = 0) {
    const int PT = g.PT, NS = g.NS, TP = g.TP, KB = g.KB, MP = g.MP;
    const bool cached = g.mat_cached > 0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    // SPLIT (forward specular tiles of the batched work queue): the (path, pair) anchor items, each several
    // times a table entry's work, go to the first warps and the table entries of phase 1a to the others (when
    // at least a warp is left), so that the warps reach the tile's barrier closer together.  (Measured: the
    // 256-pose sweep's specular queue 181 -> 175 ms; the single-pose clutter launch 5.73 -> 5.80 ms, so it
    // keeps the shared mapping.)
    const int n_anc = (KIND == 0 && !ADJ && SPLIT) ? ((PT * TP + 31) & ~31) : 0;
    const bool split = n_anc > 0 && nthr - n_anc >= 32;
    const int t_tab = split ? tid - n_anc : tid, n_tab = split ? nthr - n_anc : nthr;
    // 1a: per (path, bin) factors, written in table order (not needed when the term loop reads the
    // material table directly).  With NS % 4 == 0 and the material tables in
    // shared memory, a thread builds four adjacent entries (same path and kk, subtiles s..s+3): one chain
    // decode, 128-bit loads of the material rows and four conflict-free 128-bit stores.
    if (KIND == 1 && g.mat_direct) {
    } else if (cached && (NS & 3) == 0 && !a.etab) {
        const int KB4 = KB >> 2;
        const float invKB4 = 1.0f / (float)KB4;
        for (int e = t_tab; e >= 0 && e < PT * KB4; e += n_tab) {
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
            // four 8-byte entries (32-byte aligned: i is a multiple of 4)
            float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float2*>(B.tab) + (size_t)p * KB + i);
            if (KIND == 0) {
                dst[0] = make_float4(lx4.x, g4.x, lx4.y, g4.y);
                dst[1] = make_float4(lx4.z, g4.z, lx4.w, g4.w);
            } else {
                const float x0 = ex2(lx4.x), x1 = ex2(lx4.y), x2 = ex2(lx4.z), x3 = ex2(lx4.w);
                dst[0] = make_float4(x0, x0, x1, x1);
                dst[1] = make_float4(x2, x2, x3, x3);
            }
        }
    } else {
        for (int e = t_tab; e >= 0 && e < PT * KB; e += n_tab) {
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
                reinterpret_cast<float2*>(B.tab)[(size_t)p * KB + i] = make_float2(lx, gg);
            } else {
                const float x = ex2(lx);
                reinterpret_cast<float2*>(B.tab)[(size_t)p * KB + i] = make_float2(x, x);
            }
        }
    }
    // 1b: per (path, mic) anchors and the phasors at the subtile starts.  Specular paths of the forward go by
    // microphone pair (the two microphones' values, then one packed complex step per subtile and a 128-bit
    // store); diffraction and the adjoint by microphone (more items in flight: this phase is latency-bound
    // when the tile has fewer (path, pair) items than threads).
    if (KIND == 0 && !ADJ) {
        for (int e = tid; e < PT * TP && (!split || tid < n_anc); e += split ? n_anc : nthr) {
            const int p = e / TP, pair = e - p * TP;
            float2 zz[2], wk[2];
#pragma unroll
            for (int half = 0; half < 2; ++half)
                anchor_mic<KT, KIND, ADJ>(a, g, B, pd, pv, p, 2 * pair + half, mic0, kb, es, pglob, &zz[half],
                                                &wk[half]);
            u64 zr = pk2(zz[0].x, zz[1].x), zi = pk2(zz[0].y, zz[1].y);
            const u64 kr = pk2(wk[0].x, wk[1].x), ki = pk2(wk[0].y, wk[1].y), nki = pk2(-wk[0].y, -wk[1].y);
            ulonglong2* zo = B.za + (size_t)p * NS * TP + pair;
            for (int s_ = 0; s_ < NS; ++s_) {
                zo[(size_t)s_ * TP] = make_ulonglong2(zr, zi);
                cmul2(zr, zi, kr, ki, nki);
            }
        }
    } else {
        for (int e = tid; e < PT * MP; e += nthr) {
            const int p = e / MP, ml = e - p * MP;
            const int pair = ml >> 1, half = ml & 1;
            float2 z, wk;
            anchor_mic<KT, KIND, ADJ>(a, g, B, pd, pv, p, ml, mic0, kb, es, pglob, &z, &wk);
            float* zf = reinterpret_cast<float*>(B.za + (size_t)p * NS * TP + pair);
            for (int s_ = 0; s_ < NS; ++s_) {
                zf[(size_t)s_ * TP * 4 + half] = z.x;
                zf[(size_t)s_ * TP * 4 + 2 + half] = z.y;
                z = cmul(z, wk);
            }
        }
    }
}


// tp_max: mic pairs per CTA at most; budget: shared-memory bytes per CTA
// balance: the microphone pairs spread evenly over the microphone blocks with the bin tiling unchanged (40
// microphones: two blocks of 10 pairs instead of 16 + 4; the CTA then has fewer threads, and where it runs as
// 256 threads the spare ones are whole idle warps rather than pairs that compute zeros)
inline Geom make_geom(int M, int F, int KT, int n_mat, int tp_max = 8, size_t budget = 96 * 1024, int dir_nb = 0,
                      int mat_direct = 0, int balance = 0) {
    Geom g;
    g.NB = dir_nb;
    g.ADJ = 0;
    const int pairs = (M + 1) / 2;
    const int ns_need = (F + KT - 1) / KT;
    g.TP = std::max(1, std::min(pairs, tp_max));
    g.NS = std::max(1, std::min(ns_need, 256 / g.TP));
    g.TP = std::max(1, std::min(pairs, 256 / g.NS));
    if (balance) {
        const int nb = (pairs + g.TP - 1) / g.TP;
        g.TP = (pairs + nb - 1) / nb;
    }
    g.MP = 2 * g.TP;
    g.KB = g.NS * KT;
    g.n_mb = (M + g.MP - 1) / g.MP;
    g.n_bb = (F + g.KB - 1) / g.KB;
    const size_t mat_bytes = (size_t)2 * n_mat * g.KB * 4;  // two floats or one packed pair per (material, bin)
    g.mat_cached = mat_bytes <= 24 * 1024 ? 1 : 0;
    g.mat_direct = (mat_direct && g.mat_cached) ? 1 : 0;
    const size_t per_path = (g.mat_direct ? (size_t)0 : (size_t)g.KB * 8) + (size_t)g.NS * g.TP * 16 +
                            (size_t)g.TP * 40 + (size_t)g.MP * dir_nb * 4;
    // fixed region: cached material tables, then (directional receivers) per-bin band interpolation
    g.mat_bytes = (g.mat_cached ? mat_bytes : 0) + (dir_nb ? (size_t)g.KB * 8 : 0);
    const size_t fixed = g.mat_bytes;
    const size_t avail = budget > fixed + 4096 ? budget - fixed : 4096;
    g.PT = (int)std::min<size_t>(8, std::max<size_t>(1, avail / (2 * per_path + 2 * 52)));
    g.buf_bytes = (per_path * g.PT + 255) & ~size_t(255);
    g.smem = 2 * g.buf_bytes + 2 * (size_t)g.PT * 52 + 16 + fixed + 64;  // 16: alignment of the material tables
    return g;
}

}  // namespace acc

// One (job, path kind) accumulation of a batch for the persistent launch: its arguments (a.partial: its chunk
// partials [n_chunks][M][F]), tile shape and output [M][F]; its work items (CTAs) are item0 .. item0 +
// n_mb n_bb n_chunks - 1 of the launch and its outputs out0 .. out0 + M F - 1 of the reduction.
struct AccumTask {
    AccumArgs a;
    acc::Geom g;
    float2* out;
    int64_t item0, out0;
    const uint32_t* mat_off;  // tensor-core diffraction task: first path of each material, then the end
};
// fills t->a, t->g and t->out (the general accumulator's tile shape, 16 bins per thread, omni receivers)
cudaError_t accum_task(const AccumArgs& a, float2* out, AccumTask* t);
// the persistent accumulation of the tasks of one path kind (device table, items numbered from 0); smem = the
// largest tile's shared memory; counter: one device word, reset here
cudaError_t accumulate_queue(int kind, const AccumTask* tasks, int32_t n_tasks, int64_t n_items, size_t smem,
                             unsigned long long* counter, cudaStream_t s);
// fixed-order sums of the tasks' chunk partials into their outputs (outputs numbered from 0 over the tasks)
cudaError_t reduce_tasks(const AccumTask* tasks, int32_t n_tasks, int64_t n_out, cudaStream_t s);
// Batched tensor-core diffraction (st_accum_mma.cu).  batch_material_order sorts the compacted candidate
// indices by (job, material) -- stable, jobs stay contiguous, the material only for jobs with diff_mma set --
// and writes each such job's material offsets mat_off[j * kMatStride + q] (q = 0 .. n_mat; scratch:
// material_order_scratch(cap) bytes).  diffraction_mma_task fills a task (its tile geometry: n_mb, n_bb,
// smem) whose items the queue launch runs, one CTA per item.
cudaError_t batch_material_order(const BatchArgs& a, const uint32_t* count, int64_t cap, uint32_t* idx,
                                 uint32_t* mat_off, void* scratch, cudaStream_t s);
void diffraction_mma_task(const AccumArgs& a, const uint32_t* mat_off, float2* out, AccumTask* t);
cudaError_t accumulate_diffraction_mma_queue(const AccumTask* tasks, int32_t n_tasks, int64_t n_items,
                                             cudaStream_t s);

}  // namespace st
