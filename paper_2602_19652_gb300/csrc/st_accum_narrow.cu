// Spectrum accumulation (Eq. 2-4, 7-8) for narrow receiver arrays: one microphone pair (M <= 2, the
// two ears of the bat workloads) over many bins.
//
// The general accumulator spreads a CTA over microphone pairs x bin subtiles and shares per-(path, bin)
// factor tables between the pairs; with a single pair there is nothing to share, its CTAs shrink to one
// thread per 16 bins and the tables (16 bytes per path and bin) fill shared memory.  Here instead:
//  - thread s of a path group takes the interleaved bins kb + s + NS kk (kk < 16), both microphones
//    packed in f32x2 registers, so a warp's loads of material rows and tables are consecutive;
//  - PG groups of NS threads take different paths of a tile (256 threads per CTA), their partial
//    spectra summed in a fixed order at the end;
//  - the per-(path, bin) factor (reflection product, lobe, emitter directivity) is formed in the term
//    loop from the CTA's material rows in shared memory;
//  - per (path, microphone) the tile producer computes the phasor at the CTA's first bin and the bin
//    step raised to 2^e (e = 0 .. log2 NS + 1), each directly from the float-float path length; a
//    thread's own first phasor is the product of the powers selected by the bits of s.
// Work items and reductions are in fixed order: results do not depend on scheduling.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "st_accum_dev.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

using namespace acc;

constexpr int kNKT = 16;      // bins per thread
constexpr int kNThreads = 256;

struct NGeom {
    int NS, LNS;   // threads per path group (a power of two) and its log2
    int PG, PPG;   // path groups per CTA, paths per group per tile
    int PT;        // paths per tile
    int KB;        // bins per CTA = NS * kNKT
    int n_bb;      // CTAs along the bins
    int NB;        // receiver directivity bands (0 = omni)
    int mat_cached;
    size_t buf_bytes, mat_bytes, smem;
};

// one pipeline buffer: zb [PT] ulonglong2, pw [PT][LNS + 2] ulonglong2, ngp [PT] u64, dband [PT][NB][2] f32 (the
// two microphones' values of a band side by side, read as one packed pair)
struct NBuf {
    ulonglong2* zb;
    ulonglong2* pw;
    u64* ngp;
    float* dband;
};

__host__ __device__ inline size_t n_per_path(int LNS, int NB) { return 16 + (size_t)16 * (LNS + 2) + 8 + (size_t)8 * NB; }

__device__ __forceinline__ NBuf nbuf_at(char* base, const NGeom& g, int b) {
    NBuf B;
    char* p = base + (size_t)b * g.buf_bytes;
    B.zb = reinterpret_cast<ulonglong2*>(p);
    B.pw = B.zb + g.PT;
    B.ngp = reinterpret_cast<u64*>(B.pw + (size_t)g.PT * (g.LNS + 2));
    B.dband = reinterpret_cast<float*>(B.ngp + g.PT);
    return B;
}

// per (path, microphone, item): item 0 = phasor at bin kb (+ lobe exponent, receiver bands),
// item 1 + e = bin step raised to 2^e
template <int KIND>
__device__ __forceinline__ void nproduce(const AccumArgs& a, const NGeom& g, const NBuf& B, const float* pd,
                                         const int* pv, int kb, int64_t pglob) {
    const int items = g.LNS + 3;
    for (int e = threadIdx.x; e < g.PT * 2 * items; e += blockDim.x) {
        const int p = e / (2 * items), rem = e - p * 2 * items;
        const int half = rem / items, it = rem - half * items;
        const int m = half;
        float* zf = reinterpret_cast<float*>(it == 0 ? B.zb + p : B.pw + (size_t)p * (g.LNS + 2) + (it - 1));
        // (per-microphone receiver test: a microphone that does not see the path gets a zero anchor)
        if (!pv[p] || m >= a.M || (a.mask && !((a.mask[pglob + p] >> m) & 1ull))) {
            zf[half] = 0.0f;
            zf[2 + half] = 0.0f;
            if (it == 0) {
                reinterpret_cast<float*>(B.ngp + p)[half] = 0.0f;
                for (int b = 0; b < g.NB; ++b) B.dband[((size_t)p * g.NB + b) * 2 + half] = 0.0f;
            }
            continue;
        }
        const float* d = pd + p * 12;
        const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
        const ff dist = dist_ff(mx, my, mz, d[0], d[1], d[2]);
        const ff r = ff_add(ff{d[6], d[7]}, dist);
        const float rh = r.hi;
        if (it == 0) {
            float gam2 = 0.0f;
            if (KIND == 0) {
                const float inv = 1.0f / dist.hi;
                const float ux = (mx - d[0]) * inv, uy = (my - d[1]) * inv, uz = (mz - d[2]) * inv;
                const float cg = d[3] * ux + d[4] * uy + d[5] * uz;
                const float cx = d[4] * uz - d[5] * uy, cy = d[5] * ux - d[3] * uz, cz = d[3] * uy - d[4] * ux;
                const float gm = atan2f(sqrtf(cx * cx + cy * cy + cz * cz), cg);
                gam2 = gm * gm;
            }
            reinterpret_cast<float*>(B.ngp + p)[half] = -gam2;
            if (g.NB > 0) mic_bands(a, m, d[0] - mx, d[1] - my, d[2] - mz, B.dband + (size_t)p * 2 * g.NB + half, g.NB, 2);
            const float L0 = -2.0f * log2_ff(r) + rh * (a.atm2_0 + a.atm2_step * (float)kb);
            const ff x0 = ff_mul(r, ff{a.qhi[min(kb, a.F - 1)], a.qlo[min(kb, a.F - 1)]});
            float s0, c0;
            sincospif(2.0f * ff_frac(x0), &s0, &c0);
            const float A0 = ex2(L0);
            zf[half] = A0 * c0;
            zf[2 + half] = A0 * s0;
        } else {
            const float sc = (float)(1 << (it - 1));  // exact scaling of the float-float step
            const ff xs = ff_mul(r, ff{a.dq_hi * sc, a.dq_lo * sc});
            float s1, c1;
            sincospif(2.0f * ff_frac(xs), &s1, &c1);
            const float am = ex2(rh * (a.atm2_step * sc));
            zf[half] = am * c1;
            zf[2 + half] = am * s1;
        }
    }
}

template <int KIND, int DIR>
__global__ void __launch_bounds__(kNThreads, 2) k_accum_narrow(const AccumArgs a, const NGeom g) {
    extern __shared__ float4 smem4[];
    char* base = reinterpret_cast<char*>(smem4);
    const NBuf B0 = nbuf_at(base, g, 0), B1 = nbuf_at(base, g, 1);
    const int PT = g.PT, NS = g.NS, KB = g.KB;
    float* pdb = reinterpret_cast<float*>(base + 2 * g.buf_bytes);  // [3][PT][12]
    int* pvb = reinterpret_cast<int*>(pdb + 3 * PT * 12);            // [3][PT]
    float* mt = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(pvb + 3 * PT) + 15) & ~uintptr_t(15));
    const int nm = a.n_mat_tab;
    // material rows of the CTA's bins: lk, g2 (specular) or lid (diffraction), [n_mat][KB] each; then
    // the per-bin band interpolation (directional receivers)
    float2* bwt = reinterpret_cast<float2*>(mt + (g.mat_cached ? (KIND == 0 ? 2 : 1) * nm * KB : 0));

    const int bb = blockIdx.x, kb = bb * KB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int s = tid % NS, grp = tid / NS;

    const int64_t count = (int64_t)*a.d_count;
    const int64_t pb0 = a.d_base ? (int64_t)*a.d_base : 0;  // global index of this launch's first path
    const int64_t n_tiles = (count + PT - 1) / PT;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)blockIdx.y * per, t1 = min(n_tiles, t0 + per);

    // material row pointers: shared memory (index i) or the global tables (index kb + i)
    const float* lkp = g.mat_cached ? mt : (KIND == 0 ? a.lk : a.lid) + kb;
    const float* g2p = g.mat_cached ? mt + nm * KB : a.g2 + kb;
    const int rs = g.mat_cached ? KB : a.F;

    u64 Sr[kNKT], Si[kNKT];
#pragma unroll
    for (int kk = 0; kk < kNKT; ++kk) Sr[kk] = Si[kk] = 0ull;

    if (t0 < t1) {
        if (g.mat_cached) {
            for (int e = tid; e < nm * KB; e += nthr) {
                const int mat = e / KB, i = e - mat * KB;
                const int k = min(kb + i, a.F - 1);
                if (KIND == 0) {
                    mt[e] = a.lk[(int64_t)mat * a.F + k];
                    mt[nm * KB + e] = a.g2[(int64_t)mat * a.F + k];
                } else {
                    mt[e] = a.lid[(int64_t)mat * a.F + k];
                }
            }
        }
        if (DIR)
            for (int i = tid; i < KB; i += nthr) bwt[i] = a.bw[min(kb + i, a.F - 1)];
        load_paths_async<KIND>(a, PT, t0 * PT, count, pdb, pvb);
        if (t0 + 1 < t1) load_paths_async<KIND>(a, PT, (t0 + 1) * PT, count, pdb + PT * 12, pvb + PT);
        cp_async_wait_all();
        __syncthreads();
        nproduce<KIND>(a, g, B0, pdb, pvb, kb, pb0 + t0 * PT);
        __syncthreads();
    }
    const u64 one = pk2(1.0f, 1.0f), zero = 0ull, neg = pk2(-1.0f, -1.0f);
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int b = (int)((tile - t0) & 1);
        const int pb = (int)((tile - t0) % 3);
        const NBuf& C = b ? B1 : B0;
        const NBuf& Pn = b ? B0 : B1;
        const float* pd = pdb + pb * PT * 12;
        const int* pv = pvb + pb * PT;
        if (tile + 2 < t1) {  // slot of tile-1, free: in flight during this phase
            const int nb2 = (int)((tile + 2 - t0) % 3);
            load_paths_async<KIND>(a, PT, (tile + 2) * PT, count, pdb + nb2 * PT * 12, pvb + nb2 * PT);
        }
        if (tile + 1 < t1) {
            const int nb = (int)((tile + 1 - t0) % 3);
            nproduce<KIND>(a, g, Pn, pdb + nb * PT * 12, pvb + nb * PT, kb, pb0 + (tile + 1) * PT);
        }
        for (int q = 0; q < g.PPG; ++q) {
            const int p = grp * g.PPG + q;
            if (!pv[p]) continue;  // uniform over the group
            const float* d = pd + p * 12;
            // this thread's first phasor: z(kb) times the bin step to the power s (bits of s)
            const ulonglong2 z0 = C.zb[p];
            u64 er = z0.x, ei = z0.y;
            const ulonglong2* pw = C.pw + (size_t)p * (g.LNS + 2);
            for (int e = 0; e < g.LNS; ++e) {
                const ulonglong2 w = pw[e];
                const bool on = (s >> e) & 1;
                const u64 wr = on ? w.x : one, wi = on ? w.y : zero;
                cmul2(er, ei, wr, wi, fmul2(wi, neg));
            }
            u64 orr = er, oi = ei;  // odd chain: one interleave step (NS bins) further
            {
                const ulonglong2 w = pw[g.LNS];
                cmul2(orr, oi, w.x, w.y, fmul2(w.y, neg));
            }
            const ulonglong2 st2 = pw[g.LNS + 1];  // chain step: 2 NS bins
            const u64 s2r = st2.x, s2i = st2.y, ns2i = fmul2(st2.y, neg);
            const u64 ng = C.ngp[p];
            // reflection chain: row offsets of the path's materials
            const uint32_t meta = __float_as_uint(d[8]);
            const int len = (KIND == 0 && a.reflection_mode == 0) ? (int)(meta & 15) : 1;
            const int matj = (meta >> 8) & 255;
            // (the first four in registers; hits 5 .. 8 are decoded where they are used)
            int off[4];
            uint32_t c1 = 0;
            if (KIND == 0 && a.reflection_mode == 0) {
                const uint32_t c0 = __float_as_uint(d[9]);
                c1 = __float_as_uint(d[10]);
#pragma unroll
                for (int u = 0; u < 4; ++u) off[u] = (int)((c0 >> (8 * u)) & 255) * rs;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) off[u] = matj * rs;
            }
            const int goff = matj * rs;
            // emitter directivity: row pair of the path's angle
            const float* e0 = nullptr;
            float ew = 0.0f;
            if (a.etab && d[11] >= 0.0f) {
                const float x = d[11];
                const int itn = min((int)x, a.n_theta - 2);
                ew = x - (float)itn;
                e0 = a.etab + (int64_t)itn * a.F;
            }
            const u64* dp = reinterpret_cast<const u64*>(C.dband) + (size_t)p * g.NB;
            // the term loop, specialised on the emitter table (its loads then carry no condition)
            auto terms = [&](auto has_e) {
                constexpr bool HE = decltype(has_e)::value;
#pragma unroll
                for (int kk = 0; kk < kNKT; ++kk) {
                    const int i = s + NS * kk;
                    const int k = kb + i;
                    float lx, de = 1.0f;
                    if (HE) {  // emitter directivity, a factor of the amplitude (zero where the table is)
                        const int kc = min(k, a.F - 1);
                        de = fmaxf((1.0f - ew) * __ldg(e0 + kc) + ew * __ldg(e0 + a.F + kc), 0.0f);
                    }
                    if (k < a.F) {
                        lx = lkp[off[0] + i];
#pragma unroll
                        for (int u = 1; u < 4; ++u)
                            if (u < len) lx += lkp[off[u] + i];
                        for (int u = 4; u < len; ++u) lx += lkp[(int)((c1 >> (8 * (u - 4))) & 255) * rs + i];
                    } else {
                        lx = kNegInf;
                    }
                    u64 E;
                    if (KIND == 0) {
                        const float gg = k < a.F ? g2p[goff + i] : 0.0f;
                        const float2 arg = up2(ffma2(ng, pk2(gg, gg), pk2(lx, lx)));
                        E = pk2(ex2(arg.x), ex2(arg.y));
                    } else {
                        const float x = ex2(lx);
                        E = pk2(x, x);
                    }
                    if (DIR) {  // both microphones' bands at once
                        const float2 bwv = bwt[i];
                        const int b0 = (int)bwv.x;
                        u64 D = dp[b0];
                        if (g.NB > 1) D = ffma2(pk2(bwv.y, bwv.y), fsub2(dp[b0 + 1], D), D);
                        E = fmul2(E, HE ? fmul2(D, pk2(de, de)) : D);
                    } else if (HE) {
                        E = fmul2(E, pk2(de, de));
                    }
                    if ((kk & 1) == 0) {
                        Sr[kk] = ffma2(E, er, Sr[kk]);
                        Si[kk] = ffma2(E, ei, Si[kk]);
                        cmul2(er, ei, s2r, s2i, ns2i);
                    } else {
                        Sr[kk] = ffma2(E, orr, Sr[kk]);
                        Si[kk] = ffma2(E, oi, Si[kk]);
                        cmul2(orr, oi, s2r, s2i, ns2i);
                    }
                }
            };
            if (e0) terms(std::true_type{}); else terms(std::false_type{});
        }
        cp_async_wait_all();
        __syncthreads();
    }
    // ---- partial spectra of this chunk: sum of the path groups in order, 4 bins per pass
    float4* red = reinterpret_cast<float4*>(smem4);  // [4][PG][NS]: (re m0, re m1, im m0, im m1)
#pragma unroll
    for (int pass = 0; pass < kNKT / 4; ++pass) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int kk = pass * 4 + q;
            const float2 re = up2(Sr[kk]), im = up2(Si[kk]);
            red[((size_t)q * g.PG + grp) * NS + s] = make_float4(re.x, re.y, im.x, im.y);
        }
        __syncthreads();
        for (int e = tid; e < 4 * NS; e += nthr) {
            const int q = e / NS, s_ = e - q * NS;
            float4 acc = red[((size_t)q * g.PG) * NS + s_];
            for (int gi = 1; gi < g.PG; ++gi) {
                const float4 v = red[((size_t)q * g.PG + gi) * NS + s_];
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
            }
            const int k = kb + s_ + NS * (pass * 4 + q);
            if (k < a.F) {
                float2* out = a.partial + (size_t)blockIdx.y * a.M * a.F;
                out[k] = make_float2(acc.x, acc.z);
                if (a.M > 1) out[(size_t)a.F + k] = make_float2(acc.y, acc.w);
            }
        }
    }
}

NGeom make_ngeom(int M, int F, int n_mat, int dir_nb, int kind) {
    NGeom g;
    (void)M;
    g.NB = dir_nb;
    const int need = (F + kNKT - 1) / kNKT;
    g.NS = 1;
    g.LNS = 0;
    while (g.NS < need && g.NS < kNThreads) {
        g.NS *= 2;
        g.LNS++;
    }
    g.PG = kNThreads / g.NS;
    g.KB = g.NS * kNKT;
    g.n_bb = (F + g.KB - 1) / g.KB;
    g.PPG = std::max(1, 16 / g.PG);
    g.PT = g.PG * g.PPG;
    const size_t per_path = n_per_path(g.LNS, g.NB);
    g.buf_bytes = (per_path * g.PT + 255) & ~size_t(255);
    g.mat_bytes = (size_t)(kind == 0 ? 2 : 1) * n_mat * g.KB * 4;
    g.mat_cached = g.mat_bytes <= 64 * 1024 ? 1 : 0;
    const size_t fixed = (g.mat_cached ? g.mat_bytes : 0) + (dir_nb ? (size_t)g.KB * 8 : 0);
    const size_t red = (size_t)4 * g.PG * g.NS * 16;
    g.smem = std::max(2 * g.buf_bytes + 3 * (size_t)g.PT * 52 + 16 + fixed + 64, red + 64);
    return g;
}

template <int KIND, int DIR>
cudaError_t launch_narrow(const AccumArgs& a, cudaStream_t s) {
    const NGeom g = make_ngeom(a.M, a.F, a.n_mat_tab, DIR ? a.n_bands_tab : 0, KIND);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_accum_narrow<KIND, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)g.n_bb, (unsigned)a.n_chunks);
    note_launch();
    k_accum_narrow<KIND, DIR><<<grid, kNThreads, g.smem, s>>>(a, g);
    return cudaGetLastError();
}

}  // namespace

bool narrow_accum(int32_t M) { return M <= 2; }

int32_t narrow_chunks(int64_t n_paths_hint, int32_t M, int32_t F, int32_t n_mat, int32_t dir_nb) {
    const NGeom g = make_ngeom(M, F, n_mat, dir_nb, 0);
    const int resident = std::max(1, std::min(2, (int)((220 * 1024) / std::max<size_t>(g.smem, 1))));
    int64_t want = (int64_t)152 * resident / std::max(g.n_bb, 1);
    const int64_t tiles = (n_paths_hint + g.PT - 1) / g.PT;
    want = std::min<int64_t>(want, std::max<int64_t>(tiles, 1));
    return (int32_t)std::max<int64_t>(1, want);
}

cudaError_t accumulate_narrow(const AccumArgs& a, cudaStream_t s) {
    if (a.mic_tab) return a.kind == 0 ? launch_narrow<0, 1>(a, s) : launch_narrow<1, 1>(a, s);
    return a.kind == 0 ? launch_narrow<0, 0>(a, s) : launch_narrow<1, 0>(a, s);
}

}  // namespace st
