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

constexpr int kNV = 4;  // materials whose reflection gradient one launch accumulates

// Reduce-scatter of 8 per-bin values over the TP = 2^TPL lanes of a microphone-pair group (TP
// consecutive lanes share a subtile): after it, v[0 .. VR) of lane tp hold the group's sums for bins
// rs_first<TPL>(tp) .. + VR.  Fixed order, so the result does not depend on scheduling.
template <int TPL>
struct RS {
    static constexpr int L = TPL < 3 ? TPL : 3;  // halving steps
    static constexpr int VR = 8 >> L;            // values kept per lane
};
template <int TPL>
__device__ __forceinline__ int rs_first(int tp) {
    int off = 0, n = 8;
#pragma unroll
    for (int i = 0; i < RS<TPL>::L; ++i) {
        const int h = (1 << TPL) >> (i + 1);
        n >>= 1;
        if (tp & h) off += n;
    }
    return off;
}
template <int TPL>
__device__ __forceinline__ void rs_reduce(float (&v)[8], int tp, unsigned wm) {
    int n = 8;
#pragma unroll
    for (int i = 0; i < RS<TPL>::L; ++i) {
        const int h = (1 << TPL) >> (i + 1);
        n >>= 1;
        const bool up = (tp & h) != 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (q < n) {
                const float keep = up ? v[n + q] : v[q];
                const float send = up ? v[q] : v[n + q];
                v[q] = keep + __shfl_xor_sync(wm, send, h);
            }
        }
    }
    if (TPL >= 4) v[0] += __shfl_xor_sync(wm, v[0], 1);  // 16 lanes: tp and tp ^ 1 end with the same sum
}

// One CTA: MP = 2 TP microphones x KB bins, a chunk of the path list in tiles of PT paths (the
// forward's software pipeline: the next tile's tables are produced while this tile's terms are
// reversed; one barrier per tile).  Thread (s, tp) holds G of its two microphones and KT bins and,
// per path, folds its subtile's share of the position gradients into registers (the derivative of
// the path length and of the lobe angle are linear in the per-subtile sums C0, C1, Cg), and its
// share of the reflection sums V into kNV x VR registers after a reduce-scatter over the pair lanes.
template <int KT, int KIND, int TPL, int EMIT>
__global__ void __launch_bounds__(256, (KIND == 1 || TPL >= 3) ? 2 : 1)
    k_adjoint(const AccumArgs a, const AdjointArgs j, const Geom g) {
    static_assert(KIND == 1 || KT == 8, "the reduce-scatter of the reflection sums takes 8 bins per thread");
    constexpr int VR = RS<TPL>::VR;
    extern __shared__ float4 smem4[];
    const int PT = g.PT, NS = g.NS, TP = g.TP, KB = g.KB;
    const Buf B0 = buf_at<KT>(smem4, g, 0), B1 = buf_at<KT>(smem4, g, 1);
    // after the two pipeline buffers: pd [3][PT][12], pv [3][PT], (EMIT) chain jacobians [3][PT][12], material tables
    float* pdb = reinterpret_cast<float*>(reinterpret_cast<char*>(smem4) + 2 * g.buf_bytes);
    int* pvb = reinterpret_cast<int*>(pdb + 3 * PT * 12);
    // (16-byte aligned: each path's 12 floats are read as three float4)
    float* pjb = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(pvb + 3 * PT) + 15) & ~uintptr_t(15));
    // (specular) per path of a tile: how often each of the launch's kNV materials occurs in its reflection chain
    float4* pcb = reinterpret_cast<float4*>(pjb + (EMIT ? 3 * PT * 12 : 0));
    // (specular) and one integer signature of those counts per path (-1: no path), compared between neighbours
    int* psg = reinterpret_cast<int*>(pcb + (KIND == 0 ? 3 * PT : 0));
    float* mt = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(psg + (KIND == 0 ? 3 * PT : 0)) + 15) & ~uintptr_t(15));

    const int mb = blockIdx.x % g.n_mb, bb = blockIdx.x / g.n_mb;
    const int mic0 = mb * g.MP, kb = bb * KB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tp = tid % TP, s = tid / TP;
    // lanes of this warp that exist (the last warp of a small CTA is partial; TP divides 32)
    const int wbase = tid & ~31;
    const unsigned wm = nthr - wbase >= 32 ? 0xffffffffu : ((1u << (nthr - wbase)) - 1u);

    const int64_t count = (int64_t)*a.d_count;
    const int64_t n_tiles = (count + PT - 1) / PT;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)blockIdx.y * per, t1 = min(n_tiles, t0 + per);
    // the emitter variant always computes positions and never lobe widths (constants there, so that the term
    // loop carries no select between the two reflection sums)
    const bool do_pos = EMIT ? true : j.do_pos != 0;
    const bool do_beta = EMIT ? false : j.do_beta != 0;
    // chain jacobians of one tile's paths (EMIT), next to their path data
    auto load_jac = [&](int64_t pbase, float* dst) {
        if (EMIT) {
            for (int e = threadIdx.x; e < PT * 12; e += blockDim.x) {
                const int64_t rel = pbase + e / 12;
                dst[e] = rel < count ? a.jac[rel * 12 + e % 12] : 0.0f;
            }
        }
    };

    // material counts of one tile's paths (slot of its path data), one thread per path
    auto chain_counts = [&](const float* pd, const int* pv, float4* dst, int* sig) {
        if (KIND == 0 && j.do_k)
            for (int p = threadIdx.x; p < PT; p += blockDim.x) {
                float cnt[kNV] = {0.f, 0.f, 0.f, 0.f};
                int code = -1;
                if (pv[p]) {
                    const uint32_t meta = __float_as_uint(pd[p * 12 + 8]);
                    const int len = meta & 15, matj = (meta >> 8) & 255;
                    const uint32_t c0 = __float_as_uint(pd[p * 12 + 9]), c1 = __float_as_uint(pd[p * 12 + 10]);
                    if (a.reflection_mode == 1 || do_beta) {  // one material: the last hit's
                        const int q = matj - j.mat_base;
                        for (int u = 0; u < kNV; ++u)
                            if (q == u) cnt[u] = 1.0f;
                    } else {
                        for (int q = 0; q < len; ++q) {
                            const int mq = ((q < 4 ? (c0 >> (8 * q)) : (c1 >> (8 * (q - 4)))) & 255) - j.mat_base;
                            for (int u = 0; u < kNV; ++u)
                                if (mq == u) cnt[u] += 1.0f;
                        }
                    }
                    code = 0;  // counts of at most 8 hits: base 9
                    for (int u = kNV - 1; u >= 0; --u) code = code * 9 + (int)cnt[u];
                }
                dst[p] = make_float4(cnt[0], cnt[1], cnt[2], cnt[3]);
                sig[p] = code;
            }
    };

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
            // diffraction keeps -Im G: the Horner sums below use conj(G) E directly
            Gi[kk] = KIND == 1 ? pk2(-g1.y, -g2.y) : pk2(g1.y, g2.y);
        }
    }
    float V[kNV][VR];
#pragma unroll
    for (int q = 0; q < kNV; ++q)
#pragma unroll
        for (int v = 0; v < VR; ++v) V[q][v] = 0.0f;

    // position gradients of the thread's two microphones (and the emitter, diffraction), packed
    u64 dmx = 0ull, dmy = 0ull, dmz = 0ull;
    // emitter gradient: its factors (the direction -unit(o - s) of a diffraction path, the chain jacobian of a
    // specular one) are the same for both microphones of a pair, so it is summed over the pair first (three
    // scalar registers instead of three packed pairs)
    float esx = 0.0f, esy = 0.0f, esz = 0.0f;
    // d ln T / dr at this subtile's first bin, without the -2/r spreading term: (-a, w); per bin: (-a_step, w_step)
    const float kbs = (float)(kb + s * KT);
    const float ars = -(j.a_0 + j.a_step * kbs), nais = -(j.w_0 + j.w_step * kbs);
    const u64 ArS = pk2(ars, ars), nAiS = pk2(nais, nais);
    const u64 D1r = pk2(-j.a_step, -j.a_step), nD1i = pk2(-j.w_step, -j.w_step);

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
                } else if (g.mat_direct) {  // the factor itself, as a pair for the two microphones of a thread
                    const float x = (kb + s_ * KT + kk < a.F) ? ex2(a.lid[(int64_t)mat * a.F + k]) : 0.0f;
                    reinterpret_cast<u64*>(mt)[e] = pk2(x, x);
                } else {
                    mt[e] = a.lid[(int64_t)mat * a.F + k];
                }
            }
        }
        load_paths_async<KIND>(a, PT, t0 * PT, count, pdb, pvb);
        load_jac(t0 * PT, pjb);
        if (t0 + 1 < t1) {
            load_paths_async<KIND>(a, PT, (t0 + 1) * PT, count, pdb + PT * 12, pvb + PT);
            load_jac((t0 + 1) * PT, pjb + PT * 12);
        }
        cp_async_wait_all();
        __syncthreads();
        produce<KT, KIND, 1>(a, g, B0, pdb, pvb, mt, mic0, kb, invNS, invKB, j.s, t0 * PT);
        chain_counts(pdb, pvb, pcb, psg);
        __syncthreads();
    }
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int b = (int)((tile - t0) & 1);
        const int pb = (int)((tile - t0) % 3);  // path data of this tile
        const Buf& C = b ? B1 : B0;
        const Buf& Pn = b ? B0 : B1;
        const float* pd = pdb + pb * PT * 12;
        const int* pv = pvb + pb * PT;
        if (tile + 2 < t1) {  // slot of tile-1, free: in flight during this phase
            const int nb2 = (int)((tile + 2 - t0) % 3);
            load_paths_async<KIND>(a, PT, (tile + 2) * PT, count, pdb + nb2 * PT * 12, pvb + nb2 * PT);
            load_jac((tile + 2) * PT, pjb + nb2 * PT * 12);
        }
        if (tile + 1 < t1) {
            const int nb = (int)((tile + 1 - t0) % 3);
            produce<KT, KIND, 1>(a, g, Pn, pdb + nb * PT * 12, pvb + nb * PT, mt, mic0, kb, invNS, invKB, j.s,
                                 (tile + 1) * PT);
            chain_counts(pdb + nb * PT * 12, pvb + nb * PT, pcb + nb * PT, psg + nb * PT);
        }
        // per-bin values of the current run of paths with equal material counts (specular; flushed by the
        // tile's last path at the latest, so that they are not live across the producer phase)
        float Y[KT];
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) Y[kk] = 0.0f;
        for (int p = 0; p < PT; ++p) {
            const ulonglong2 z0 = C.za[((size_t)p * NS + s) * TP + tp];
            const u64* w = C.wst + (size_t)p * 4 * TP + tp;  // component-major: conflict-free 64-bit loads
            const u64 w1r = w[0], w1i = w[TP], w2r = w[2 * TP], w2i = w[3 * TP];
            const u64 nw2i = fmul2(w2i, pk2(-1.0f, -1.0f));
            const u64 ng = C.ngp[(size_t)p * TP + tp];
            u64 er = z0.x, ei = z0.y, orr = er, oi = ei;
            cmul2(orr, oi, w1r, w1i, fmul2(w1i, pk2(-1.0f, -1.0f)));
            u64 c0r = 0ull, c0i = 0ull, qr = 0ull, qi = 0ull, cg = 0ull;
            u64 c1r = 0ull, c1i = 0ull;  // diffraction: C1 = sum_kk kk conj(G) T directly
            const float2 ngv = up2(ng);  // -gamma^2 of the two microphones (lobe sums)
            const float2* trow = reinterpret_cast<const float2*>(C.tab) + (size_t)p * KB + s;
            // diffraction with the material table read directly: row offset left by the producer in ngp
            const u64* mrow = reinterpret_cast<const u64*>(mt) + s;
            if (KIND == 1 && g.mat_direct) mrow += (int)(uint32_t)ng;
            if (KIND == 1) {
                // Diffraction (positions only): with u_kk = conj(G_kk) E_kk and z_kk = z0 W^kk,
                //   C0 = z0 P(W), C1 = z0 W P'(W),  P(W) = sum_kk u_kk W^kk,
                // P and P' by Horner's scheme from the top bin (no explicit phasor chain).
                const u64 nw1i = fmul2(w1i, pk2(-1.0f, -1.0f));
                auto Eat = [&](int kk) -> u64 {
                    return g.mat_direct ? mrow[kk * NS] : reinterpret_cast<const u64*>(trow)[kk * NS];
                };
                u64 E = Eat(KT - 1);
                u64 pr = fmul2(Gr[KT - 1], E), pim = fmul2(Gi[KT - 1], E), dpr = 0ull, dpi = 0ull;
#pragma unroll
                for (int kk = KT - 2; kk >= 0; --kk) {
                    E = Eat(kk);
                    const u64 ur = fmul2(Gr[kk], E), ui = fmul2(Gi[kk], E);
                    const u64 ndr = ffma2(dpr, w1r, ffma2(dpi, nw1i, pr));  // P' <- P' W + P
                    const u64 ndi = ffma2(dpr, w1i, ffma2(dpi, w1r, pim));
                    const u64 npr = ffma2(pr, w1r, ffma2(pim, nw1i, ur));  // P <- P W + u
                    const u64 npi = ffma2(pr, w1i, ffma2(pim, w1r, ui));
                    dpr = ndr;
                    dpi = ndi;
                    pr = npr;
                    pim = npi;
                }
                c0r = ffma2(er, pr, fmul2(fmul2(ei, pk2(-1.0f, -1.0f)), pim));
                c0i = ffma2(er, pim, fmul2(ei, pr));
                const u64 tr = ffma2(w1r, dpr, fmul2(nw1i, dpi)), ti = ffma2(w1r, dpi, fmul2(w1i, dpr));
                c1r = ffma2(er, tr, fmul2(fmul2(ei, pk2(-1.0f, -1.0f)), ti));
                c1i = ffma2(er, ti, fmul2(ei, tr));
            } else {
#pragma unroll
                for (int kk = 0; kk < KT; ++kk) {  // specular
                    const float2 t = trow[kk * NS];  // (log2 X, g)
                    const u64 E = pk2(ex2(fmaf(ngv.x, t.y, t.x)), ex2(fmaf(ngv.y, t.y, t.x)));
                    const u64 zr = (kk & 1) ? orr : er, zi = (kk & 1) ? oi : ei;
                    const u64 Tr = fmul2(E, zr), Ti = fmul2(E, zi);
                    const u64 wr = ffma2(Gr[kk], Tr, fmul2(Gi[kk], Ti));        // Re(conj(G) T)
                    const u64 wi = fsub2(fmul2(Gr[kk], Ti), fmul2(Gi[kk], Tr));  // Im(conj(G) T)
                    c0r = fadd2(c0r, wr);
                    c0i = fadd2(c0i, wi);
                    qr = fadd2(qr, c0r);  // running sum of prefix sums: sum_kk kk w = KT C0 - Q
                    qi = fadd2(qi, c0i);
                    if (KIND == 0) cg = ffma2(pk2(t.y, t.y), wr, cg);
                    const float2 wr2 = up2(wr);
                    Y[kk] += do_beta ? fmaf(wr2.x, ngv.x, wr2.y * ngv.y) : wr2.x + wr2.y;
                    if (kk & 1) cmul2(orr, oi, w2r, w2i, nw2i); else cmul2(er, ei, w2r, w2i, nw2i);
                }
            }
            if (do_pos) {
                const u64* ad = C.adj + ((size_t)p * TP + tp) * 7;
                // C1 relative to the subtile's first bin
                const u64 q1r = KIND == 1 ? c1r : fsub2(fmul2(pk2((float)KT, (float)KT), c0r), qr);
                const u64 q1i = KIND == 1 ? c1i : fsub2(fmul2(pk2((float)KT, (float)KT), c0i), qi);
                const u64 d0r = ffma2(pk2(-2.0f, -2.0f), ad[6], ArS);  // -2/r - a(kb_s)
                // dL/dr share: Re(D0 C0 + D1 C1), D0 = d0r + j w(kb_s), D1 = -a_step + j w_step
                u64 dl = fmul2(d0r, c0r);
                dl = ffma2(nAiS, c0i, dl);
                dl = ffma2(D1r, q1r, dl);
                dl = ffma2(nD1i, q1i, dl);
                if (KIND == 0 && EMIT) {
                    // microphone share g = dl u + cg v'; emitter through the hit point and the path length:
                    // dL/ds += (dr/ds) dl - J^T g  (J = dP/ds, both per path, frozen chain)
                    const u64 gx = ffma2(cg, ad[3], fmul2(dl, ad[0]));
                    const u64 gy = ffma2(cg, ad[4], fmul2(dl, ad[1]));
                    const u64 gz = ffma2(cg, ad[5], fmul2(dl, ad[2]));
                    dmx = fadd2(dmx, gx);
                    dmy = fadd2(dmy, gy);
                    dmz = fadd2(dmz, gz);
                    const float* jp = pjb + pb * PT * 12 + p * 12;
                    const float4 j0 = *reinterpret_cast<const float4*>(jp);      // J00 J01 J02 J10
                    const float4 j1 = *reinterpret_cast<const float4*>(jp + 4);  // J11 J12 J20 J21
                    const float4 j2 = *reinterpret_cast<const float4*>(jp + 8);  // J22 drx dry drz
                    const float2 dl2 = up2(dl), gx2 = up2(gx), gy2 = up2(gy), gz2 = up2(gz);
                    const float sl = dl2.x + dl2.y, sx = gx2.x + gx2.y, sy = gy2.x + gy2.y, sz = gz2.x + gz2.y;
                    esx = fmaf(j2.y, sl, esx);
                    esx = fmaf(-j0.x, sx, esx);
                    esx = fmaf(-j0.w, sy, esx);
                    esx = fmaf(-j1.z, sz, esx);
                    esy = fmaf(j2.z, sl, esy);
                    esy = fmaf(-j0.y, sx, esy);
                    esy = fmaf(-j1.x, sy, esy);
                    esy = fmaf(-j1.w, sz, esy);
                    esz = fmaf(j2.w, sl, esz);
                    esz = fmaf(-j0.z, sx, esz);
                    esz = fmaf(-j1.y, sy, esz);
                    esz = fmaf(-j2.x, sz, esz);
                } else {
                    dmx = ffma2(dl, ad[0], dmx);
                    dmy = ffma2(dl, ad[1], dmy);
                    dmz = ffma2(dl, ad[2], dmz);
                }
                if (KIND == 0) {  // lobe angle
                    if (!EMIT) {
                        dmx = ffma2(cg, ad[3], dmx);
                        dmy = ffma2(cg, ad[4], dmy);
                        dmz = ffma2(cg, ad[5], dmz);
                    }
                } else {  // emitter: dr/ds = -unit(o - s)
                    const float2 d2 = up2(dl);
                    const float dsum = d2.x + d2.y;
                    esx = fmaf(dsum, up2(ad[3]).x, esx);
                    esy = fmaf(dsum, up2(ad[4]).x, esy);
                    esz = fmaf(dsum, up2(ad[5]).x, esz);
                }
            }
            // reflection-coefficient sums for the materials of the path's chain: V += cnt (x) Y.  Consecutive
            // paths with the same material counts (the backward orders its path list by them) share one
            // reduce-scatter: Y sums their per-bin values until the counts change or the tile ends (the
            // decision is the same for every thread of the CTA).  An invalid path adds zeros to Y.
            if constexpr (KIND == 0) if (j.do_k) {
                if (p == PT - 1 || psg[pb * PT + p] != psg[pb * PT + p + 1]) {
                    rs_reduce<TPL>(Y, tp, wm);
                    const float4 c4 = pcb[pb * PT + p];  // the chain's material counts, from the producer
                    const float cnt[kNV] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                    for (int u = 0; u < kNV; ++u)
#pragma unroll
                        for (int v = 0; v < VR; ++v) V[u][v] = fmaf(cnt[u], Y[v], V[u][v]);
#pragma unroll
                    for (int kk = 0; kk < KT; ++kk) Y[kk] = 0.0f;
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
    // ---- outputs of this CTA (shared memory reused)
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    if (do_pos) {
        float* red = reinterpret_cast<float*>(smem4);  // [NS][TP][2][3] microphones, then [nthr][3] emitter
        float* rede = red + (size_t)nthr * 6;
        __syncthreads();
        {
            const float2 x = up2(dmx), y2 = up2(dmy), z = up2(dmz);
            float* o = red + (size_t)tid * 6;
            o[0] = x.x; o[1] = y2.x; o[2] = z.x;
            o[3] = x.y; o[4] = y2.y; o[5] = z.y;
            rede[tid * 3 + 0] = esx;
            rede[tid * 3 + 1] = esy;
            rede[tid * 3 + 2] = esz;
        }
        __syncthreads();
        if (tid < g.MP && mic0 + tid < a.M) {  // microphone mic0 + tid: fixed-order sum over the subtiles
            const int pair = tid >> 1, half = tid & 1;
            float acc[3] = {0.f, 0.f, 0.f};
            for (int s_ = 0; s_ < NS; ++s_) {
                const float* r = red + ((size_t)s_ * TP + pair) * 6 + 3 * half;
                acc[0] += r[0];
                acc[1] += r[1];
                acc[2] += r[2];
            }
            float* o = j.mic_part + ((size_t)(blockIdx.y * g.n_bb + bb) * a.M + mic0 + tid) * 3;
            o[0] = acc[0];
            o[1] = acc[1];
            o[2] = acc[2];
        }
        if (tid < 3) {
            float acc = 0.0f;
            for (int t = 0; t < nthr; ++t) acc += rede[t * 3 + tid];
            j.emit_part[(size_t)cta * 3 + tid] = acc;
        }
    }
    if (KIND == 0 && j.do_k) {
        // each bin's sum sits in one lane (two identical lanes with 16 pairs: the even one writes)
        const bool writer = TPL >= 4 ? (tp & 1) == 0 : true;
        const int k0 = kb + s * KT + rs_first<TPL>(tp);
        if (writer) {
#pragma unroll
            for (int u = 0; u < kNV; ++u)
#pragma unroll
                for (int v = 0; v < VR; ++v)
                    if (k0 + v < a.F) j.v_part[((size_t)(blockIdx.y * g.n_mb + mb) * kNV + u) * a.F + k0 + v] = V[u][v];
        }
    }
}

// per compacted specular path (record id = idx[c] = ray * B + j): dP_j/ds and dr_j/ds along the frozen chain.
// Hit q is the intersection of the line from P_{q-1} along d_q with triangle q's plane:
// dP_q/dP_{q-1} = I - d_q n_q^T / (n_q . d_q), dt_q/dP_{q-1} = -n_q^T / (n_q . d_q), P_{-1} = s.
__global__ void k_chain_jacobians(const uint32_t* idx, const uint32_t* count, int32_t B, const int32_t* rec_tri,
                                  const float* rec_d, const float* nrm, const float* dirs, float4 qv, float* jac) {
    const int64_t n = *count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const int64_t id = idx[c];
        const int64_t ray = id / B;
        const int jj = (int)(id - ray * B);
        // emitted direction: q applied to the ray's local direction
        const float vx = dirs[3 * ray], vy = dirs[3 * ray + 1], vz = dirs[3 * ray + 2];
        const float tx = 2.0f * (qv.z * vz - qv.w * vy), ty = 2.0f * (qv.w * vx - qv.y * vz),
                    tz = 2.0f * (qv.y * vy - qv.z * vx);
        float d[3] = {vx + qv.x * tx + (qv.z * tz - qv.w * ty), vy + qv.x * ty + (qv.w * tx - qv.y * tz),
                      vz + qv.x * tz + (qv.y * ty - qv.z * tx)};
        float J[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f}, dr[3] = {0.f, 0.f, 0.f};
        for (int q = 0; q <= jj; ++q) {
            const int32_t t = rec_tri[ray * B + q];
            const float n0 = nrm[3 * t], n1 = nrm[3 * t + 1], n2 = nrm[3 * t + 2];
            const float inv = 1.0f / (n0 * d[0] + n1 * d[1] + n2 * d[2]);
            float nJ[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) nJ[k] = (n0 * J[k] + n1 * J[3 + k] + n2 * J[6 + k]) * inv;
#pragma unroll
            for (int k = 0; k < 3; ++k) dr[k] -= nJ[k];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) J[3 * r + k] -= d[r] * nJ[k];
            const float* dn = rec_d + 3 * (ray * B + q);
            d[0] = dn[0];
            d[1] = dn[1];
            d[2] = dn[2];
        }
        float* o = jac + c * 12;
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = J[k];
        o[9] = dr[0];
        o[10] = dr[1];
        o[11] = dr[2];
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

// dk[mat][b] = sum_k V[mat][k] w_b(k) / k(mat, f_k) over the bins whose interpolation uses band b.
// One block per (material, band); threads stride over the bins in float64, then a fixed-order tree sum.
constexpr int kDkThreads = 128;
__global__ void __launch_bounds__(kDkThreads) k_dk_contract(const float* V, int F, int mat_base, int n_bands,
                                                           const float* band_hz, const float* kb_tab, double f_lo,
                                                           double df, float* dk) {
    __shared__ double red[kDkThreads];
    const int u = blockIdx.x / n_bands, b = blockIdx.x % n_bands;
    const int mat = mat_base + u;
    const float* kr = kb_tab + (size_t)mat * n_bands;
    double acc = 0.0;
    for (int k = threadIdx.x; k < F; k += kDkThreads) {
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
                int lo = 0, hi = n_bands - 1;  // last band centre <= f
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if ((double)band_hz[mid] <= f) lo = mid; else hi = mid;
                }
                b0 = lo;
                w = (f - (double)band_hz[b0]) / ((double)band_hz[b0 + 1] - (double)band_hz[b0]);
            }
        }
        double wb = 0.0;
        if (n_bands == 1) wb = 1.0;
        else if (b == b0) wb = 1.0 - w;
        else if (b == b0 + 1) wb = w;
        if (wb == 0.0) continue;
        const double kv = n_bands == 1 ? (double)kr[0] : (1.0 - w) * (double)kr[b0] + w * (double)kr[b0 + 1];
        if (!(kv > 0.0)) continue;
        acc += v * wb / kv;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kDkThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) dk[(size_t)mat * n_bands + b] = (float)red[0];
}

// dbeta[mat][b] = sum_k Vg[mat][k] dg_k / dbeta_b, g_k = (1 - w) / (2 beta_b0^2) + w / (2 beta_b1^2), Vg the lobe
// sums dL/dg; one block per (material, band), threads over the bins in float64, fixed-order tree sum
__global__ void __launch_bounds__(kDkThreads) k_dbeta_contract(const float* V, int F, int mat_base, int n_bands,
                                                              const float* band_hz, const float* beta_tab,
                                                              double f_lo, double df, float* dbeta) {
    __shared__ double red[kDkThreads];
    const int u = blockIdx.x / n_bands, b = blockIdx.x % n_bands;
    const int mat = mat_base + u;
    const double be = (double)beta_tab[(size_t)mat * n_bands + b];
    const double dgdb = -1.0 / (be * be * be);
    double acc = 0.0;
    for (int k = threadIdx.x; k < F; k += kDkThreads) {
        const double v = (double)V[(size_t)u * F + k];
        if (v == 0.0) continue;
        const double f = F == 1 ? f_lo : f_lo + (double)k * df;
        double wb = 1.0;
        if (n_bands > 1) {
            int b0;
            double w;
            if (f <= (double)band_hz[0]) {
                b0 = 0;
                w = 0.0;
            } else if (f >= (double)band_hz[n_bands - 1]) {
                b0 = n_bands - 2;
                w = 1.0;
            } else {
                int lo = 0, hi = n_bands - 1;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if ((double)band_hz[mid] <= f) lo = mid; else hi = mid;
                }
                b0 = lo;
                w = (f - (double)band_hz[b0]) / ((double)band_hz[b0 + 1] - (double)band_hz[b0]);
            }
            wb = (b == b0) ? 1.0 - w : (b == b0 + 1 ? w : 0.0);
        }
        if (wb == 0.0) continue;
        acc += v * wb * dgdb;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kDkThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) dbeta[(size_t)mat * n_bands + b] = (float)red[0];
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

template <int KT, int KIND, int TPL, int EMIT = 0>
cudaError_t launch_adjoint(const AccumArgs& a, const AdjointArgs& j, const Geom& g, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_adjoint<KT, KIND, TPL, EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)(g.n_mb * g.n_bb), (unsigned)a.n_chunks);
    const size_t smem =
        g.smem + (EMIT ? (size_t)3 * g.PT * 12 * 4 + 16 : 0) + (KIND == 0 ? (size_t)3 * g.PT * (16 + 4) + 16 : 0);
    note_launch();
    k_adjoint<KT, KIND, TPL, EMIT><<<grid, g.TP * g.NS, smem, s>>>(a, j, g);
    return cudaGetLastError();
}

}  // namespace

namespace {

size_t adjoint_per_path(const acc::Geom& g) {
    return (g.mat_direct ? (size_t)0 : (size_t)g.KB * 8) + (size_t)g.NS * g.TP * 16 + (size_t)g.TP * 40 +
           (size_t)g.TP * 56;
}

}  // namespace

size_t adjoint_smem(const acc::Geom& g) {
    const size_t total = 2 * g.buf_bytes + 3 * (size_t)g.PT * 52 + 16 + (g.mat_cached ? g.mat_bytes : 0) + 64;
    const size_t red = (size_t)g.TP * g.NS * 9 * 4 + 64;  // end-of-kernel reductions reuse the start
    return std::max(total, red);
}

acc::Geom adjoint_geom(int M, int F, int n_mat, int mat_direct, int tp_max, int kt) {
    // tile shape of the forward with kt bins per thread (8 where the reflection sums are reduce-scattered across
    // the pair lanes, 16 for diffraction paths) and up to tp_max microphone pairs per CTA, the pair count a power
    // of two; paths per tile as many as fit about 100 KB, so that two CTAs share an SM
    acc::Geom g = acc::make_geom(M, F, kt, n_mat, tp_max, 200 * 1024, 0, mat_direct);
    int tp2 = 1;
    while (tp2 * 2 <= g.TP) tp2 *= 2;
    g.TP = tp2;
    g.MP = 2 * tp2;
    g.n_mb = (M + g.MP - 1) / g.MP;
    g.ADJ = 1;
    const size_t per_path = adjoint_per_path(g);
    const size_t per_tile = 2 * per_path + 3 * 52;
    const size_t fixed = (g.mat_cached ? g.mat_bytes : 0) + 16 + 64 + 512;
    const size_t budget = 100 * 1024;
    g.PT = (int)std::max<size_t>(1, std::min<size_t>(8, budget > fixed ? (budget - fixed) / per_tile : 1));
    g.buf_bytes = (per_path * g.PT + 255) & ~size_t(255);
    g.smem = adjoint_smem(g);
    return g;
}

cudaError_t adjoint_launch(const AccumArgs& a, const AdjointArgs& j, const acc::Geom& g, cudaStream_t s) {
    if (a.kind == 1) return g.KB == 16 * g.NS ? launch_adjoint<16, 1, 0>(a, j, g, s) : launch_adjoint<8, 1, 0>(a, j, g, s);
    if (a.jac && j.do_pos) {
        switch (g.TP) {
            case 1: return launch_adjoint<8, 0, 0, 1>(a, j, g, s);
            case 2: return launch_adjoint<8, 0, 1, 1>(a, j, g, s);
            case 4: return launch_adjoint<8, 0, 2, 1>(a, j, g, s);
            case 8: return launch_adjoint<8, 0, 3, 1>(a, j, g, s);
            default: return launch_adjoint<8, 0, 4, 1>(a, j, g, s);
        }
    }
    switch (g.TP) {
        case 1: return launch_adjoint<8, 0, 0>(a, j, g, s);
        case 2: return launch_adjoint<8, 0, 1>(a, j, g, s);
        case 4: return launch_adjoint<8, 0, 2>(a, j, g, s);
        case 8: return launch_adjoint<8, 0, 3>(a, j, g, s);
        default: return launch_adjoint<8, 0, 4>(a, j, g, s);
    }
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
    k_dk_contract<<<n, kDkThreads, 0, s>>>(v, F, mat_base, n_bands, band_hz_dev, k_dev, f_lo, df, dk);
    return cudaGetLastError();
}

cudaError_t chain_jacobians(const uint32_t* idx, const uint32_t* count, int64_t n_max, int32_t B, const int32_t* rec_tri,
                            const float* rec_d, const float* nrm, const float* dirs, const float q[4], float* jac,
                            cudaStream_t s) {
    if (n_max <= 0) return cudaSuccess;
    note_launch();
    k_chain_jacobians<<<grid_for(n_max, 256), 256, 0, s>>>(idx, count, B, rec_tri, rec_d, nrm, dirs,
                                                           make_float4(q[0], q[1], q[2], q[3]), jac);
    return cudaGetLastError();
}

cudaError_t adjoint_dbeta(const float* v_part, int n_slices, int F, int mat_base, int n_mat_launch, int n_bands,
                          const float* band_hz_dev, const float* beta_dev, double f_lo, double df, float* dbeta,
                          cudaStream_t s) {
    const int n = n_mat_launch * n_bands;
    if (n <= 0) return cudaSuccess;
    float* v = const_cast<float*>(v_part);
    note_launch();
    k_v_reduce<<<(kNV * F + 127) / 128, 128, 0, s>>>(v, n_slices, F);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launch();
    k_dbeta_contract<<<n, kDkThreads, 0, s>>>(v, F, mat_base, n_bands, band_hz_dev, beta_dev, f_lo, df, dbeta);
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
