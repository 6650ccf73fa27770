// Diffraction accumulation (Eq. 7-8) as a complex matrix product on the tensor cores.
//
// With an omni emitter and omni receivers the per-bin factor of a diffraction path depends only on its
// material q and the bin k (the diffraction table I_d), so with the paths of one material
//     T_q[m][k] = sum_p z_pm W_pm^k,        S[m][k] = sum_q E_q[k] T_q[m][k],
// where z_pm is path p's phasor at microphone m and the block's first bin (spreading, air absorption and
// phase) and W_pm its one-bin step.  Writing k = 32 k1 + k2 (k1 < 16, k2 < 32) splits W^k = (W^32)^k1 W^k2:
//     T_q[m][32 k1 + k2] = sum_p U[k1][p] V[p][k2],   U[k1][p] = z_pm (W_pm^32)^k1,   V[p][k2] = W_pm^k2,
// a 16 x P times P x 32 complex product over the paths for each microphone.
//
// A CTA takes four microphones (one warp each) and 512 bins, and walks its share of the material-ordered
// path list in tiles of 32 paths.  Per tile every thread forms U and V of one (path, microphone) in float32
// -- two chains from anchors computed directly from the float-float path length -- and stores them as
// bf16 pairs x = hi + lo (16 significant bits); each warp then multiplies its microphone's tile with
// mma.sync (bf16 inputs, float32 accumulation), hi*hi + hi*lo + lo*hi for each of the four real products
// of the complex one (the dropped lo*lo is below 2^-16 of a product; relative L2 error of the spectra
// a few 1e-6).  When the material changes, every kFlushTiles tiles, and at the end, a warp adds E_q[k] times
// its accumulators to its spectrum registers (float32 fma, rounded to nearest: the tensor cores' own float32
// accumulation is not, and its error would grow with the tiles summed into one accumulator).  Results are in
// fixed order for a given launch shape.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "st_accum_dev.cuh"
#include "st_internal.cuh"

namespace st {

namespace {

using namespace acc;

constexpr int kMmaMics = 4;     // microphones (warps) per CTA
constexpr int kMmaPaths = 32;   // paths per tile
constexpr int kK1 = 16, kK2 = 32, kMmaBins = kK1 * kK2;
constexpr int kFlushTiles = 4;  // tiles summed into the matrix-product accumulators between flushes
constexpr int kURow = 24;       // bf16 per U row (16 + 8 padding: conflict-free ldmatrix rows)
constexpr int kVRow = 40;       // bf16 per V row (32 + 8)
constexpr size_t kUBytes = (size_t)kMmaMics * 4 * kMmaPaths * kURow * 2;
constexpr size_t kVBytes = (size_t)kMmaMics * 4 * kMmaPaths * kVRow * 2;
constexpr size_t kMmaSmem = kUBytes + kVBytes + kMmaPaths * 8 * 4 + kMmaPaths * 4;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// D += A B: m16n8k16, bf16 inputs, float32 accumulation (registers only: not volatile, so that the compiler
// interleaves products on independent accumulators)
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// (x0, x1) -> bf16 high parts and the bf16 low parts of the remainders, each as one packed word
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - __low2float(h), x1 - __high2float(h));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Two phasor chains at once, as (re, re) and (im, im) pairs: (zr, zi) *= (wr, wi) with the rounding of cmul
// (re = fma(zr, wr, -(zi wi)), im = fma(zr, wi, zi wr)), so the pairs hold exactly the scalar chains' values;
// nwi = -wi
__device__ __forceinline__ void cmul2_as_scalar(u64& zr, u64& zi, u64 wr, u64 wi, u64 nwi) {
    const u64 tn = fmul2(zi, nwi), t2 = fmul2(zi, wr);
    const u64 r = ffma2(zr, wr, tn);
    zi = ffma2(zr, wi, t2);
    zr = r;
}

// tile of the material-ordered path list: material q, first path and path count
struct MTile {
    int q;
    int64_t first;
    int n;
};

__device__ __forceinline__ MTile tile_at(const uint32_t* mat_off, int n_mat, int64_t t) {
    for (int q = 0; q < n_mat; ++q) {
        const int64_t cnt = (int64_t)mat_off[q + 1] - mat_off[q];
        const int64_t nt = (cnt + kMmaPaths - 1) / kMmaPaths;
        if (t < nt) {
            const int64_t left = cnt - t * kMmaPaths;
            return MTile{q, (int64_t)mat_off[q] + t * kMmaPaths, (int)(left < kMmaPaths ? left : kMmaPaths)};
        }
        t -= nt;
    }
    return MTile{-1, 0, 0};
}

// One CTA's work: microphone block mb, bin block bb, chunk `chunk` of a.n_chunks (its share of the tiles)
__device__ __forceinline__ void diff_mma_cta(const AccumArgs& a, const uint32_t* mat_off, int mb, int bb, int chunk,
                                             char* base) {
    __nv_bfloat16* Us = reinterpret_cast<__nv_bfloat16*>(base);            // [mic][part][path][kURow]
    __nv_bfloat16* Vs = reinterpret_cast<__nv_bfloat16*>(base + kUBytes);  // [mic][part][path][kVRow]
    float* pd = reinterpret_cast<float*>(base + kUBytes + kVBytes);        // [path][8]: point, r hi, r lo
    int* pq = reinterpret_cast<int*>(pd + kMmaPaths * 8);                  // [path] valid

    const int mic0 = mb * kMmaMics, kb = bb * kMmaBins;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_mat = a.n_mat_tab;

    int64_t n_tiles = 0;
    for (int q = 0; q < n_mat; ++q) n_tiles += ((int64_t)mat_off[q + 1] - mat_off[q] + kMmaPaths - 1) / kMmaPaths;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)chunk * per, t1 = min(n_tiles, t0 + per);

    // this warp's accumulators: T (current material) and S (spectrum), fragment layout of m16n8 blocks:
    // element i of n-block nb is (k1 = g + 8 (i >> 1), k2 = 8 nb + 2 t + (i & 1))
    float Tr[4][4], Ti[4][4], Sr[4][4], Si[4][4];
#pragma unroll
    for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int i = 0; i < 4; ++i) Tr[nb][i] = Ti[nb][i] = Sr[nb][i] = Si[nb][i] = 0.0f;
    const int g = lane >> 2, t4 = lane & 3;
    const int m_w = mic0 + warp;
    int q_cur = -1, n_acc = 0;

    auto flush = [&]() {
        if (q_cur < 0) return;
#pragma unroll
        for (int nb = 0; nb < 4; ++nb)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = kb + kK2 * (g + 8 * (i >> 1)) + 8 * nb + 2 * t4 + (i & 1);
                const float E = k < a.F ? ex2(__ldg(a.lid + (int64_t)q_cur * a.F + k)) : 0.0f;
                Sr[nb][i] = fmaf(E, Tr[nb][i], Sr[nb][i]);
                Si[nb][i] = fmaf(E, Ti[nb][i], Si[nb][i]);
                Tr[nb][i] = 0.0f;
                Ti[nb][i] = 0.0f;
            }
    };

    const int kq = min(kb, a.F - 1);
    const ff qk{a.qhi[kq], a.qlo[kq]};
    for (int64_t tile = t0; tile < t1; ++tile) {
        const MTile T = tile_at(mat_off, n_mat, tile);
        // path data of the tile
        if (tid < kMmaPaths) {
            const bool ok = tid < T.n;
            const int64_t i = T.first + tid;
            pq[tid] = ok ? 1 : 0;
            float* d = pd + tid * 8;
            d[0] = ok ? a.px[i] : 0.0f;
            d[1] = ok ? a.py[i] : 0.0f;
            d[2] = ok ? a.pz[i] : 0.0f;
            d[3] = ok ? a.rhi[i] : 1.0f;
            d[4] = ok ? a.rlo[i] : 0.0f;
        }
        __syncthreads();  // (also: the previous tile's fragments have been read)
        // U and V of one (path, microphone) per thread
        {
            const int p = tid % kMmaPaths, ml = tid / kMmaPaths, m = mic0 + ml;
            float2 z = make_float2(0.0f, 0.0f), w1 = make_float2(0.0f, 0.0f), w32 = make_float2(0.0f, 0.0f);
            if (pq[p] && m < a.M) {
                const float* d = pd + p * 8;
                const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
                const ff r = ff_add(ff{d[3], d[4]}, dist_ff(mx, my, mz, d[0], d[1], d[2]));
                const float rh = r.hi;
                const float L0 = -2.0f * log2_ff(r) + rh * (a.atm2_0 + a.atm2_step * (float)kb);
                float s, c;
                sincospif(2.0f * ff_frac(ff_mul(r, qk)), &s, &c);
                const float A0 = ex2(L0);
                z = make_float2(A0 * c, A0 * s);
                sincospif(2.0f * ff_frac(ff_mul(r, ff{a.dq_hi, a.dq_lo})), &s, &c);
                const float a1 = ex2(rh * a.atm2_step);
                w1 = make_float2(a1 * c, a1 * s);
                // (32 = 2^5: the float-float step scales exactly)
                sincospif(2.0f * ff_frac(ff_mul(r, ff{a.dq_hi * 32.0f, a.dq_lo * 32.0f})), &s, &c);
                const float a32 = ex2(rh * (a.atm2_step * 32.0f));
                w32 = make_float2(a32 * c, a32 * s);
            }
            // U row: z (W^32)^k1, k1 = 0 .. 15, parts re hi, re lo, im hi, im lo (even and odd k1 as two
            // independent chains of step W^64)
            uint32_t* ur = reinterpret_cast<uint32_t*>(Us + (((size_t)ml * 4) * kMmaPaths + p) * kURow);
            const size_t upart = (size_t)kMmaPaths * kURow / 2;  // words between parts
            const float2 w64 = cmul(w32, w32);
            const float2 zo = cmul(z, w32);
            // the even and odd chains as one packed pair
            u64 ur2 = pk2(z.x, zo.x), ui2 = pk2(z.y, zo.y);
            const u64 w64r = pk2(w64.x, w64.x), w64i = pk2(w64.y, w64.y), nw64i = pk2(-w64.y, -w64.y);
#pragma unroll
            for (int j = 0; j < kK1 / 8; ++j) {
                uint32_t rh4[4], rl4[4], ih4[4], il4[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 ur = up2(ur2), ui = up2(ui2);
                    cmul2_as_scalar(ur2, ui2, w64r, w64i, nw64i);
                    split2(ur.x, ur.y, rh4[e], rl4[e]);
                    split2(ui.x, ui.y, ih4[e], il4[e]);
                }
                reinterpret_cast<uint4*>(ur + 0 * upart)[j] = make_uint4(rh4[0], rh4[1], rh4[2], rh4[3]);
                reinterpret_cast<uint4*>(ur + 1 * upart)[j] = make_uint4(rl4[0], rl4[1], rl4[2], rl4[3]);
                reinterpret_cast<uint4*>(ur + 2 * upart)[j] = make_uint4(ih4[0], ih4[1], ih4[2], ih4[3]);
                reinterpret_cast<uint4*>(ur + 3 * upart)[j] = make_uint4(il4[0], il4[1], il4[2], il4[3]);
            }
            // V row: W^k2, k2 = 0 .. 31 (zero for an invalid path or microphone)
            uint32_t* vr = reinterpret_cast<uint32_t*>(Vs + (((size_t)ml * 4) * kMmaPaths + p) * kVRow);
            const size_t vpart = (size_t)kMmaPaths * kVRow / 2;
            // (four independent chains of step W^4: k2 = 4 e + c)
            float2 vc[4];
            vc[0] = (pq[p] && m < a.M) ? make_float2(1.0f, 0.0f) : make_float2(0.0f, 0.0f);
            vc[1] = cmul(vc[0], w1);
            vc[2] = cmul(vc[1], w1);
            vc[3] = cmul(vc[2], w1);
            const float2 w4 = cmul(cmul(w1, w1), cmul(w1, w1));
            // chains 0, 1 and chains 2, 3 as two packed pairs
            u64 r01 = pk2(vc[0].x, vc[1].x), i01 = pk2(vc[0].y, vc[1].y);
            u64 r23 = pk2(vc[2].x, vc[3].x), i23 = pk2(vc[2].y, vc[3].y);
            const u64 w4r = pk2(w4.x, w4.x), w4i = pk2(w4.y, w4.y), nw4i = pk2(-w4.y, -w4.y);
#pragma unroll
            for (int j = 0; j < kK2 / 8; ++j) {
                uint32_t rh4[4], rl4[4], ih4[4], il4[4];
#pragma unroll
                for (int e2 = 0; e2 < 2; ++e2) {
                    const float2 a01 = up2(r01), b01 = up2(i01), a23 = up2(r23), b23 = up2(i23);
                    split2(a01.x, a01.y, rh4[2 * e2], rl4[2 * e2]);
                    split2(b01.x, b01.y, ih4[2 * e2], il4[2 * e2]);
                    split2(a23.x, a23.y, rh4[2 * e2 + 1], rl4[2 * e2 + 1]);
                    split2(b23.x, b23.y, ih4[2 * e2 + 1], il4[2 * e2 + 1]);
                    cmul2_as_scalar(r01, i01, w4r, w4i, nw4i);
                    cmul2_as_scalar(r23, i23, w4r, w4i, nw4i);
                }
                reinterpret_cast<uint4*>(vr + 0 * vpart)[j] = make_uint4(rh4[0], rh4[1], rh4[2], rh4[3]);
                reinterpret_cast<uint4*>(vr + 1 * vpart)[j] = make_uint4(rl4[0], rl4[1], rl4[2], rl4[3]);
                reinterpret_cast<uint4*>(vr + 2 * vpart)[j] = make_uint4(ih4[0], ih4[1], ih4[2], ih4[3]);
                reinterpret_cast<uint4*>(vr + 3 * vpart)[j] = make_uint4(il4[0], il4[1], il4[2], il4[3]);
            }
        }
        __syncthreads();
        if (m_w < a.M) {
            // the accumulators go into the spectrum registers when the material changes, and at least every
            // kFlushTiles tiles: the tensor cores' float32 accumulation does not round to nearest, so its error
            // grows with the number of products summed into one accumulator; the spectrum sums round to nearest
            if (T.q != q_cur || n_acc == kFlushTiles) {
                flush();
                q_cur = T.q;
                n_acc = 0;
            }
            ++n_acc;
            const __nv_bfloat16* Uw = Us + (size_t)warp * 4 * kMmaPaths * kURow;
            const __nv_bfloat16* Vw = Vs + (size_t)warp * 4 * kMmaPaths * kVRow;
            const int mi = lane >> 3, rr = lane & 7;
#pragma unroll
            for (int ks = 0; ks < kMmaPaths / 16; ++ks) {
                // A fragments (16 k1 x 16 paths) of the four parts, from U rows [path][k1] transposed
                uint32_t A[4][4];
                const int pa = ks * 16 + rr + (mi >> 1) * 8, ca = (mi & 1) * 8;
#pragma unroll
                for (int part = 0; part < 4; ++part)
                    ldsm_x4_t(smem_u32(Uw + ((size_t)part * kMmaPaths + pa) * kURow + ca), A[part][0], A[part][1],
                              A[part][2], A[part][3]);
                uint32_t nI[2][4];  // -(U im): the real part takes - Ui Vi
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    nI[0][e] = A[2][e] ^ 0x80008000u;
                    nI[1][e] = A[3][e] ^ 0x80008000u;
                }
                const int pb = ks * 16 + rr + (mi & 1) * 8;
                // B fragments (16 paths x 8 k2) of the four n-blocks, from V rows [path][k2]: Bf[part][nb][0..1]
                uint32_t Bf[4][4][2];
#pragma unroll
                for (int nb2 = 0; nb2 < 2; ++nb2) {
                    const int cb = nb2 * 16 + (mi >> 1) * 8;
#pragma unroll
                    for (int part = 0; part < 4; ++part)
                        ldsm_x4_t(smem_u32(Vw + ((size_t)part * kMmaPaths + pb) * kVRow + cb), Bf[part][2 * nb2][0],
                                  Bf[part][2 * nb2][1], Bf[part][2 * nb2 + 1][0], Bf[part][2 * nb2 + 1][1]);
                }
                // real: Ur Vr - Ui Vi; imaginary: Ur Vi + Ui Vr -- each product over the four n-blocks in turn
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Tr[nb], A[0], Bf[0][nb][0], Bf[0][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Ti[nb], A[0], Bf[2][nb][0], Bf[2][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Tr[nb], A[0], Bf[1][nb][0], Bf[1][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Ti[nb], A[0], Bf[3][nb][0], Bf[3][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Tr[nb], A[1], Bf[0][nb][0], Bf[0][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Ti[nb], A[1], Bf[2][nb][0], Bf[2][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Tr[nb], nI[0], Bf[2][nb][0], Bf[2][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Ti[nb], A[2], Bf[0][nb][0], Bf[0][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Tr[nb], nI[0], Bf[3][nb][0], Bf[3][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Ti[nb], A[2], Bf[1][nb][0], Bf[1][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Tr[nb], nI[1], Bf[2][nb][0], Bf[2][nb][1]);
#pragma unroll
                for (int nb = 0; nb < 4; ++nb) mma_bf16(Ti[nb], A[3], Bf[0][nb][0], Bf[0][nb][1]);
            }
        }
    }
    flush();
    // this chunk's partial spectrum of the warp's microphone
    if (m_w < a.M) {
        float2* out = a.partial + ((size_t)chunk * a.M + m_w) * a.F;
#pragma unroll
        for (int nb = 0; nb < 4; ++nb)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = kb + kK2 * (g + 8 * (i >> 1)) + 8 * nb + 2 * t4 + (i & 1);
                if (k < a.F) out[k] = make_float2(Sr[nb][i], Si[nb][i]);
            }
    }
}

__global__ void __launch_bounds__(kMmaMics * 32, 3) k_accum_diff_mma(const AccumArgs a, const uint32_t* mat_off,
                                                                    int n_mb) {
    extern __shared__ float4 smem4[];
    diff_mma_cta(a, mat_off, blockIdx.x % n_mb, blockIdx.x / n_mb, blockIdx.y, reinterpret_cast<char*>(smem4));
}

// The diffraction tasks of a batch (one per job, each with its material offsets): CTA i runs item i of the
// table, items numbered as in the single-job grid (microphone block fastest, then bin block, then chunk).
__global__ void __launch_bounds__(kMmaMics * 32, 3) k_accum_diff_mma_queue(const AccumTask* tasks, int32_t n_tasks) {
    extern __shared__ float4 smem4[];
    const int64_t it = blockIdx.x;
    int lo = 0, hi = n_tasks - 1;  // last task whose first item is <= it
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].item0 <= it) lo = mid; else hi = mid - 1;
    }
    const AccumTask& T = tasks[lo];
    const int n_mb = T.g.n_mb, nxy = n_mb * T.g.n_bb;
    const int local = (int)(it - T.item0);
    diff_mma_cta(T.a, T.mat_off, (local % nxy) % n_mb, (local % nxy) / n_mb, local / nxy,
                 reinterpret_cast<char*>(smem4));
}

// ---------------------------------------------------------------- the diffraction adjoint (positions)
// The reverse pass needs per (path, microphone) C0 = sum_k c_k z_k and C1 = sum_k (k - kb) c_k z_k with
// c_k = conj(G_k) E_q[k] (G: dL/dS of the diffraction component, E_q: the material's factor).  With
// z_k = z0 (W^32)^k1 W^k2 (k - kb = 32 k1 + k2):
//     C0 = z0 sum_k1 (W^32)^k1 Y[k1],                 Y[k1]  = sum_k2 W^k2 c[k1][k2]
//     C1 = z0 sum_k1 (W^32)^k1 (32 k1 Y[k1] + Y'[k1]), Y'[k1] = sum_k2 W^k2 k2 c[k1][k2]
// so for the paths of one material and one microphone [Y | Y'] = V (P x 32) times B (32 x 32) with
// B[k2][k1] = c[k1][k2] and B[k2][16 + k1] = k2 c[k1][k2]: the gradient is the operand shared by all paths,
// rebuilt when the material changes.  Per tile each warp multiplies its microphone's V by its B on the tensor
// cores (bf16 high and low parts as in the forward), then finishes C0 and C1 with the 16-term sums above
// (float32, the powers (W^32)^k1 kept from the tile's producer), forms dL/dr = Re(D0 C0 + D1 C1) and adds
// dL/dr times d r / d m and d r / d s to its microphone and emitter gradient registers.
constexpr int kBRow = 40;  // bf16 per B row: 32 k2 + 8
constexpr size_t kAdjV = (size_t)kMmaMics * 4 * kMmaPaths * kVRow * 2;
constexpr size_t kAdjB = (size_t)kMmaMics * 4 * 32 * kBRow * 2;
// per-path rows of the epilogue's operands, padded against bank conflicts: the lanes of a quad read one path,
// eight paths at once
constexpr int kUpRow = kK1 + 1;  // float2 per (W^32)^k1 row
constexpr int kPmRow = 9;        // floats per (path, microphone) record
constexpr size_t kAdjU = (size_t)kMmaMics * kMmaPaths * kUpRow * 8;
constexpr size_t kAdjPM = (size_t)kMmaMics * kMmaPaths * kPmRow * 4;
constexpr size_t kAdjSmem = kAdjV + kAdjB + kAdjU + kAdjPM + kMmaPaths * 8 * 4 + kMmaPaths * 4 + kMmaMics * 4 * 4;

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__global__ void __launch_bounds__(kMmaMics * 32, 2) k_adjoint_diff_mma(const AccumArgs a, const AdjointArgs j,
                                                                      const uint32_t* mat_off, int n_mb, int n_bb) {
    extern __shared__ float4 smem4[];
    char* base = reinterpret_cast<char*>(smem4);
    __nv_bfloat16* Vs = reinterpret_cast<__nv_bfloat16*>(base);                 // [mic][part][path][kVRow]
    __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(base + kAdjV);         // [mic][part][n][kBRow]
    float2* Up = reinterpret_cast<float2*>(base + kAdjV + kAdjB);               // [mic][path][kUpRow]: (W^32)^k1
    float* pm = reinterpret_cast<float*>(base + kAdjV + kAdjB + kAdjU);         // [mic][path][kPmRow]
    float* pd = pm + (size_t)kMmaMics * kMmaPaths * kPmRow;                     // [path][8]
    int* pq = reinterpret_cast<int*>(pd + kMmaPaths * 8);                       // [path] valid
    float* ered = reinterpret_cast<float*>(pq + kMmaPaths);                     // [mic][4] emitter sums

    const int mb = blockIdx.x % n_mb, bb = blockIdx.x / n_mb;
    const int mic0 = mb * kMmaMics, kb = bb * kMmaBins;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t4 = lane & 3;
    const int n_mat = a.n_mat_tab;
    const int m_w = mic0 + warp;

    int64_t n_tiles = 0;
    for (int q = 0; q < n_mat; ++q) n_tiles += ((int64_t)mat_off[q + 1] - mat_off[q] + kMmaPaths - 1) / kMmaPaths;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)blockIdx.y * per, t1 = min(n_tiles, t0 + per);

    // dL/dr = Re(D0 C0 + D1 C1): D0 = -2/r - a(kb) + j w(kb), D1 = -a_step + j w_step
    const float akb = j.a_0 + j.a_step * (float)kb, wkb = j.w_0 + j.w_step * (float)kb;
    float gmx = 0.0f, gmy = 0.0f, gmz = 0.0f, gex = 0.0f, gey = 0.0f, gez = 0.0f;
    int q_cur = -1;
    const int kq = min(kb, a.F - 1);
    const ff qk{a.qhi[kq], a.qlo[kq]};
    for (int64_t tile = t0; tile < t1; ++tile) {
        const MTile T = tile_at(mat_off, n_mat, tile);
        __syncthreads();  // the previous tile's epilogue has read the path data and the per-(path, mic) values
        if (tid < kMmaPaths) {
            const bool ok = tid < T.n;
            const int64_t i = T.first + tid;
            pq[tid] = ok ? 1 : 0;
            float* d = pd + tid * 8;
            d[0] = ok ? a.px[i] : 0.0f;
            d[1] = ok ? a.py[i] : 0.0f;
            d[2] = ok ? a.pz[i] : 0.0f;
            d[3] = ok ? a.rhi[i] : 1.0f;
            d[4] = ok ? a.rlo[i] : 0.0f;
            // d r / d s = -unit(o - s) (the emitter-to-point length is r hi + r lo)
            const float iv = 1.0f / d[3];
            d[5] = -((d[0] - j.s[0]) * iv);
            d[6] = -((d[1] - j.s[1]) * iv);
            d[7] = -((d[2] - j.s[2]) * iv);
        }
        if (T.q != q_cur) {
            // B of the four microphones for the new material: rows n < 16 c[n][k2], rows 16 + n k2 c[n][k2]
            for (int e = tid; e < kMmaMics * kK1 * kK2; e += blockDim.x) {
                const int ml = e / (kK1 * kK2), rem = e - ml * kK1 * kK2, k1 = rem / kK2, k2 = rem - k1 * kK2;
                const int m = mic0 + ml, k = kb + kK2 * k1 + k2;
                float cr = 0.0f, ci = 0.0f;
                if (m < a.M && k < a.F) {
                    const float2 G = j.G[(int64_t)m * a.F + k];
                    const float E = ex2(__ldg(a.lid + (int64_t)T.q * a.F + k));
                    cr = G.x * E;  // conj(G) E
                    ci = -G.y * E;
                }
                const float cw[2][2] = {{cr, ci}, {(float)k2 * cr, (float)k2 * ci}};
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int n = half * kK1 + k1;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const __nv_bfloat16 h = __float2bfloat16_rn(cw[half][c]);
                        const __nv_bfloat16 l = __float2bfloat16_rn(cw[half][c] - __bfloat162float(h));
                        Bs[(((size_t)ml * 4 + 2 * c) * 32 + n) * kBRow + k2] = h;
                        Bs[(((size_t)ml * 4 + 2 * c + 1) * 32 + n) * kBRow + k2] = l;
                    }
                }
            }
            q_cur = T.q;
        }
        __syncthreads();
        // per (path, microphone): V row, the powers (W^32)^k1, z0, D0's real part and d r / d m
        {
            const int p = tid % kMmaPaths, ml = tid / kMmaPaths, m = mic0 + ml;
            float2 z = make_float2(0.0f, 0.0f), w1 = make_float2(0.0f, 0.0f), w32 = make_float2(0.0f, 0.0f);
            float* o = pm + ((size_t)ml * kMmaPaths + p) * kPmRow;
            const bool ok = pq[p] && m < a.M;
            if (ok) {
                const float* d = pd + p * 8;
                const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
                const ff dist = dist_ff(mx, my, mz, d[0], d[1], d[2]);
                const ff r = ff_add(ff{d[3], d[4]}, dist);
                const float rh = r.hi;
                const float L0 = -2.0f * log2_ff(r) + rh * (a.atm2_0 + a.atm2_step * (float)kb);
                float s, c;
                sincospif(2.0f * ff_frac(ff_mul(r, qk)), &s, &c);
                const float A0 = ex2(L0);
                z = make_float2(A0 * c, A0 * s);
                sincospif(2.0f * ff_frac(ff_mul(r, ff{a.dq_hi, a.dq_lo})), &s, &c);
                const float a1 = ex2(rh * a.atm2_step);
                w1 = make_float2(a1 * c, a1 * s);
                sincospif(2.0f * ff_frac(ff_mul(r, ff{a.dq_hi * 32.0f, a.dq_lo * 32.0f})), &s, &c);
                const float a32 = ex2(rh * (a.atm2_step * 32.0f));
                w32 = make_float2(a32 * c, a32 * s);
                const float inv = 1.0f / dist.hi;
                o[0] = z.x;
                o[1] = z.y;
                o[2] = -2.0f / rh - akb;
                o[3] = (mx - d[0]) * inv;  // d r / d m = unit(m - P)
                o[4] = (my - d[1]) * inv;
                o[5] = (mz - d[2]) * inv;
                o[6] = 1.0f;
            } else {
                o[0] = o[1] = o[2] = o[3] = o[4] = o[5] = o[6] = 0.0f;
            }
            float2* up = Up + ((size_t)ml * kMmaPaths + p) * kUpRow;
            const float2 w64 = cmul(w32, w32);
            // the even and odd powers as one packed pair
            u64 ur2 = pk2(1.0f, w32.x), ui2 = pk2(0.0f, w32.y);
            const u64 w64r = pk2(w64.x, w64.x), w64i = pk2(w64.y, w64.y), nw64i = pk2(-w64.y, -w64.y);
#pragma unroll
            for (int k1 = 0; k1 < kK1; k1 += 2) {
                const float2 ur = up2(ur2), ui = up2(ui2);
                up[k1] = make_float2(ur.x, ui.x);
                up[k1 + 1] = make_float2(ur.y, ui.y);
                cmul2_as_scalar(ur2, ui2, w64r, w64i, nw64i);
            }
            uint32_t* vr = reinterpret_cast<uint32_t*>(Vs + (((size_t)ml * 4) * kMmaPaths + p) * kVRow);
            const size_t vpart = (size_t)kMmaPaths * kVRow / 2;
            float2 vc[4];
            vc[0] = ok ? make_float2(1.0f, 0.0f) : make_float2(0.0f, 0.0f);
            vc[1] = cmul(vc[0], w1);
            vc[2] = cmul(vc[1], w1);
            vc[3] = cmul(vc[2], w1);
            const float2 w4 = cmul(cmul(w1, w1), cmul(w1, w1));
            // chains 0, 1 and chains 2, 3 as two packed pairs
            u64 r01 = pk2(vc[0].x, vc[1].x), i01 = pk2(vc[0].y, vc[1].y);
            u64 r23 = pk2(vc[2].x, vc[3].x), i23 = pk2(vc[2].y, vc[3].y);
            const u64 w4r = pk2(w4.x, w4.x), w4i = pk2(w4.y, w4.y), nw4i = pk2(-w4.y, -w4.y);
#pragma unroll
            for (int jj = 0; jj < kK2 / 8; ++jj) {
                uint32_t rh4[4], rl4[4], ih4[4], il4[4];
#pragma unroll
                for (int e2 = 0; e2 < 2; ++e2) {
                    const float2 a01 = up2(r01), b01 = up2(i01), a23 = up2(r23), b23 = up2(i23);
                    split2(a01.x, a01.y, rh4[2 * e2], rl4[2 * e2]);
                    split2(b01.x, b01.y, ih4[2 * e2], il4[2 * e2]);
                    split2(a23.x, a23.y, rh4[2 * e2 + 1], rl4[2 * e2 + 1]);
                    split2(b23.x, b23.y, ih4[2 * e2 + 1], il4[2 * e2 + 1]);
                    cmul2_as_scalar(r01, i01, w4r, w4i, nw4i);
                    cmul2_as_scalar(r23, i23, w4r, w4i, nw4i);
                }
                reinterpret_cast<uint4*>(vr + 0 * vpart)[jj] = make_uint4(rh4[0], rh4[1], rh4[2], rh4[3]);
                reinterpret_cast<uint4*>(vr + 1 * vpart)[jj] = make_uint4(rl4[0], rl4[1], rl4[2], rl4[3]);
                reinterpret_cast<uint4*>(vr + 2 * vpart)[jj] = make_uint4(ih4[0], ih4[1], ih4[2], ih4[3]);
                reinterpret_cast<uint4*>(vr + 3 * vpart)[jj] = make_uint4(il4[0], il4[1], il4[2], il4[3]);
            }
        }
        __syncthreads();
        if (m_w < a.M) {
            const __nv_bfloat16* Vw = Vs + (size_t)warp * 4 * kMmaPaths * kVRow;
            const __nv_bfloat16* Bw = Bs + (size_t)warp * 4 * 32 * kBRow;
            const int mi = lane >> 3, rr = lane & 7;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                // [Y | Y'] rows of paths 16 mt .. 16 mt + 15: fragment element i of n-block nb is
                // (path 16 mt + g + 8 (i >> 1), column 8 nb + 2 t + (i & 1))
                float Yr[4][4], Yi[4][4];
#pragma unroll
                for (int nb = 0; nb < 4; ++nb)
#pragma unroll
                    for (int i = 0; i < 4; ++i) Yr[nb][i] = Yi[nb][i] = 0.0f;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    uint32_t A[4][4];
                    const int pa = 16 * mt + rr + (mi & 1) * 8, ca = 16 * ks + (mi >> 1) * 8;
#pragma unroll
                    for (int part = 0; part < 4; ++part)
                        ldsm_x4(smem_u32(Vw + ((size_t)part * kMmaPaths + pa) * kVRow + ca), A[part][0], A[part][1],
                                A[part][2], A[part][3]);
                    uint32_t nI[2][4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        nI[0][e] = A[2][e] ^ 0x80008000u;
                        nI[1][e] = A[3][e] ^ 0x80008000u;
                    }
                    uint32_t Bf[4][4][2];  // [part][n-block][reg]
#pragma unroll
                    for (int nb2 = 0; nb2 < 2; ++nb2) {
                        const int nrow = 16 * nb2 + rr + (mi >> 1) * 8, cb = 16 * ks + (mi & 1) * 8;
#pragma unroll
                        for (int part = 0; part < 4; ++part)
                            ldsm_x4(smem_u32(Bw + ((size_t)part * 32 + nrow) * kBRow + cb), Bf[part][2 * nb2][0],
                                    Bf[part][2 * nb2][1], Bf[part][2 * nb2 + 1][0], Bf[part][2 * nb2 + 1][1]);
                    }
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yr[nb], A[0], Bf[0][nb][0], Bf[0][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yi[nb], A[0], Bf[2][nb][0], Bf[2][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yr[nb], A[0], Bf[1][nb][0], Bf[1][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yi[nb], A[0], Bf[3][nb][0], Bf[3][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yr[nb], A[1], Bf[0][nb][0], Bf[0][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yi[nb], A[1], Bf[2][nb][0], Bf[2][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yr[nb], nI[0], Bf[2][nb][0], Bf[2][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yi[nb], A[2], Bf[0][nb][0], Bf[0][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yr[nb], nI[0], Bf[3][nb][0], Bf[3][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yi[nb], A[2], Bf[1][nb][0], Bf[1][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yr[nb], nI[1], Bf[2][nb][0], Bf[2][nb][1]);
#pragma unroll
                    for (int nb = 0; nb < 4; ++nb) mma_bf16(Yi[nb], A[3], Bf[0][nb][0], Bf[0][nb][1]);
                }
                // C0 and C1 of the two paths of this thread (rows g and g + 8 of the m-tile): this lane's k1
                // are 2 t, 2 t + 1 (n-block 0) and 8 + 2 t, 9 + 2 t (n-block 1); Y' in n-blocks 2 and 3
#pragma unroll
                for (int hp = 0; hp < 2; ++hp) {
                    const int p = 16 * mt + g + 8 * hp;
                    const float2* up = Up + ((size_t)warp * kMmaPaths + p) * kUpRow;
                    float s0r = 0.0f, s0i = 0.0f, s1r = 0.0f, s1i = 0.0f;
#pragma unroll
                    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const int i = 2 * hp + c, k1 = 8 * nb + 2 * t4 + c;
                            const float2 w = up[k1];
                            const float yr = Yr[nb][i], yi = Yi[nb][i];
                            const float xr = 32.0f * (float)k1 * yr + Yr[nb + 2][i];
                            const float xi = 32.0f * (float)k1 * yi + Yi[nb + 2][i];
                            s0r += w.x * yr - w.y * yi;
                            s0i += w.x * yi + w.y * yr;
                            s1r += w.x * xr - w.y * xi;
                            s1i += w.x * xi + w.y * xr;
                        }
#pragma unroll
                    for (int o = 1; o <= 2; o <<= 1) {
                        s0r += __shfl_xor_sync(0xffffffffu, s0r, o);
                        s0i += __shfl_xor_sync(0xffffffffu, s0i, o);
                        s1r += __shfl_xor_sync(0xffffffffu, s1r, o);
                        s1i += __shfl_xor_sync(0xffffffffu, s1i, o);
                    }
                    const float* q = pm + ((size_t)warp * kMmaPaths + p) * kPmRow;
                    if (t4 == 0 && q[6] != 0.0f) {
                        const float zr = q[0], zi = q[1];
                        const float c0r = zr * s0r - zi * s0i, c0i = zr * s0i + zi * s0r;
                        const float c1r = zr * s1r - zi * s1i, c1i = zr * s1i + zi * s1r;
                        const float dl = q[2] * c0r - wkb * c0i - j.a_step * c1r - j.w_step * c1i;
                        gmx += dl * q[3];
                        gmy += dl * q[4];
                        gmz += dl * q[5];
                        const float* d = pd + p * 8;
                        gex += dl * d[5];
                        gey += dl * d[6];
                        gez += dl * d[7];
                    }
                }
            }
        }
    }
    // the warp's sums (lanes with t = 0 hold them), in a fixed order
#pragma unroll
    for (int o = 4; o <= 16; o <<= 1) {
        gmx += __shfl_xor_sync(0xffffffffu, gmx, o);
        gmy += __shfl_xor_sync(0xffffffffu, gmy, o);
        gmz += __shfl_xor_sync(0xffffffffu, gmz, o);
        gex += __shfl_xor_sync(0xffffffffu, gex, o);
        gey += __shfl_xor_sync(0xffffffffu, gey, o);
        gez += __shfl_xor_sync(0xffffffffu, gez, o);
    }
    if (lane == 0) {
        if (m_w < a.M) {
            float* o = j.mic_part + ((size_t)(blockIdx.y * n_bb + bb) * a.M + m_w) * 3;
            o[0] = gmx;
            o[1] = gmy;
            o[2] = gmz;
        }
        ered[warp * 4 + 0] = gex;
        ered[warp * 4 + 1] = gey;
        ered[warp * 4 + 2] = gez;
    }
    __syncthreads();
    if (tid < 3) {
        float acc = 0.0f;
        for (int w = 0; w < kMmaMics; ++w) acc += ered[w * 4 + tid];
        j.emit_part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 3 + tid] = acc;
    }
}

// material key of every compacted diffraction candidate (past the count: a key above every material)
__global__ void k_mat_keys(const uint32_t* idx, const uint32_t* count, int64_t cap, const int32_t* cand_tri,
                           const int32_t* tri_mat, uint64_t* keys) {
    const int64_t n = *count;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cap; c += (int64_t)gridDim.x * blockDim.x)
        keys[c] = c < n ? (uint64_t)((uint32_t)tri_mat[cand_tri[idx[c]]] & 255u) : 256ull;
}

// first position of each material in the sorted keys, and the count at the end
__global__ void k_mat_offsets(const uint64_t* keys, const uint32_t* count, int n_mat, uint32_t* off) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > n_mat) return;
    const int64_t n = *count;
    if (q == n_mat) {
        off[q] = (uint32_t)n;
        return;
    }
    int64_t lo = 0, hi = n;  // lower bound of key q
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < (uint64_t)q) lo = mid + 1;
        else hi = mid;
    }
    off[q] = (uint32_t)lo;
}

// Batched form: key (job, material) of every compacted diffraction candidate, the material only for the jobs
// accumulated on the tensor cores (0 for the others, whose order then stays the compaction order); past the
// count a key above every job
__global__ void k_mat_keys_batch(const BatchArgs a, const uint32_t* idx, const uint32_t* count, int64_t cap,
                                 uint64_t* keys) {
    const int64_t n = *count;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cap; c += (int64_t)gridDim.x * blockDim.x) {
        if (c >= n) {
            keys[c] = (uint64_t)a.n_jobs << 16;
            continue;
        }
        const int64_t i = idx[c];
        const int job = find_job(a.samp_offs, a.n_jobs, i);
        const JobDev& b = a.jobs[job];
        uint32_t q = 0u;
        if (b.diff_mma) {
            q = (uint32_t)b.tri_mat[a.cand_tri[i]] & 255u;
        } else if (b.etab) {
            // emitter-table row of the candidate (the gather's coordinate, floored): a tile's paths then read the
            // same one or two table rows, which stay in L1
            const float ox = a.cand_p[3 * i], oy = a.cand_p[3 * i + 1], oz = a.cand_p[3 * i + 2];
            const float vx = ox - b.s[0], vy = oy - b.s[1], vz = oz - b.s[2];
            const ff r = dist_ff(ox, oy, oz, b.s[0], b.s[1], b.s[2]);
            const float cth = (b.fwd[0] * vx + b.fwd[1] * vy + b.fwd[2] * vz) / r.hi;
            q = (uint32_t)min((int)(acosf(fminf(1.0f, fmaxf(-1.0f, cth))) * b.inv_dtheta), 0xfffe);
        }
        keys[c] = ((uint64_t)job << 16) | q;
    }
}

// per tensor-core job j: first position of each of its materials and its end, off[j * kMatStride + q]
__global__ void k_mat_offsets_batch(const BatchArgs a, const uint64_t* keys, const uint32_t* count, uint32_t* off) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)a.n_jobs * kMatStride) return;
    const int j = (int)(t / kMatStride), q = (int)(t % kMatStride);
    const JobDev& b = a.jobs[j];
    if (!b.diff_mma || q > b.n_mat) return;
    const uint64_t key = ((uint64_t)j << 16) | (uint64_t)q;  // q = n_mat: the first key past the job's materials
    int64_t lo = 0, hi = *count;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    off[t] = (uint32_t)lo;
}

}  // namespace

bool diffraction_mma_applies(const AccumArgs& a) {
    static const int env = [] {
        const char* e = getenv("ST_DIFF_MMA");
        return e ? atoi(e) : 1;
    }();
    return env != 0 && a.kind == 1 && !a.etab && !a.mic_tab && !narrow_accum(a.M) && a.F >= 128 && a.n_mat_tab <= 255;
}

int32_t diffraction_mma_chunks(int64_t n_paths_hint, int32_t M, int32_t F, int32_t n_mat) {
    const int64_t ctas = (int64_t)((M + kMmaMics - 1) / kMmaMics) * ((F + kMmaBins - 1) / kMmaBins);
    const int64_t tiles = (n_paths_hint + kMmaPaths - 1) / kMmaPaths + n_mat;
    const int64_t want = std::max<int64_t>(1, (152 * 3 * 2) / std::max<int64_t>(ctas, 1));
    return (int32_t)std::max<int64_t>(1, std::min<int64_t>(want, tiles));
}

size_t material_order_scratch(int64_t cap) { return (size_t)std::max<int64_t>(cap, 1) * 8 + sort_scratch_bytes(cap); }

cudaError_t material_order(const uint32_t* count, int64_t cap, const int32_t* cand_tri, const int32_t* tri_mat,
                           int n_mat, uint32_t* idx, uint32_t* mat_off, void* scratch, cudaStream_t s) {
    if (cap <= 0) return cudaSuccess;
    uint64_t* keys = static_cast<uint64_t*>(scratch);
    void* sort_scr = static_cast<char*>(scratch) + (size_t)cap * 8;
    note_launch();
    k_mat_keys<<<grid_for(cap, 256), 256, 0, s>>>(idx, count, cap, cand_tri, tri_mat, keys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = radix_sort_u64(keys, idx, cap, 9, sort_scr, s)) != cudaSuccess) return e;  // stable
    note_launch();
    k_mat_offsets<<<(n_mat + 1 + 127) / 128, 128, 0, s>>>(keys, count, n_mat, mat_off);
    return cudaGetLastError();
}

void adjoint_diffraction_mma_shape(int32_t M, int32_t F, int32_t* n_mb, int32_t* n_bb) {
    *n_mb = (M + kMmaMics - 1) / kMmaMics;
    *n_bb = (F + kMmaBins - 1) / kMmaBins;
}

cudaError_t adjoint_diffraction_mma(const AccumArgs& a, const AdjointArgs& j, const uint32_t* mat_off,
                                    cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_adjoint_diff_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int32_t n_mb, n_bb;
    adjoint_diffraction_mma_shape(a.M, a.F, &n_mb, &n_bb);
    dim3 grid((unsigned)(n_mb * n_bb), (unsigned)a.n_chunks);
    note_launch();
    k_adjoint_diff_mma<<<grid, kMmaMics * 32, kAdjSmem, s>>>(a, j, mat_off, n_mb, n_bb);
    return cudaGetLastError();
}

// (jobs with an emitter table and no tensor-core diffraction are keyed by the emitter-table row of each
// candidate instead of its material, so that their accumulator reads few table rows per tile)
cudaError_t batch_material_order(const BatchArgs& a, const uint32_t* count, int64_t cap, uint32_t* idx,
                                 uint32_t* mat_off, void* scratch, cudaStream_t s) {
    if (cap <= 0) return cudaSuccess;
    uint64_t* keys = static_cast<uint64_t*>(scratch);
    void* sort_scr = static_cast<char*>(scratch) + (size_t)cap * 8;
    note_launch();
    k_mat_keys_batch<<<grid_for(cap, 256), 256, 0, s>>>(a, idx, count, cap, keys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int bits = 16;
    while (((int64_t)1 << (bits - 16)) <= a.n_jobs) ++bits;  // job indices 0 .. n_jobs (the sentinel)
    if ((e = radix_sort_u64(keys, idx, cap, bits, sort_scr, s)) != cudaSuccess) return e;  // stable
    const int64_t nt = (int64_t)a.n_jobs * kMatStride;
    note_launch();
    k_mat_offsets_batch<<<grid_for(nt, 256), 256, 0, s>>>(a, keys, count, mat_off);
    return cudaGetLastError();
}

void diffraction_mma_task(const AccumArgs& a, const uint32_t* mat_off, float2* out, AccumTask* t) {
    t->a = a;
    t->g = acc::Geom{};
    t->g.n_mb = (a.M + kMmaMics - 1) / kMmaMics;
    t->g.n_bb = (a.F + kMmaBins - 1) / kMmaBins;
    t->g.smem = kMmaSmem;
    t->out = out;
    t->mat_off = mat_off;
}

cudaError_t accumulate_diffraction_mma_queue(const AccumTask* tasks, int32_t n_tasks, int64_t n_items,
                                             cudaStream_t s) {
    if (n_tasks <= 0 || n_items <= 0) return cudaSuccess;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_accum_diff_mma_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmaSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    note_launch();
    k_accum_diff_mma_queue<<<(unsigned)n_items, kMmaMics * 32, kMmaSmem, s>>>(tasks, n_tasks);
    return cudaGetLastError();
}

cudaError_t accumulate_diffraction_mma(const AccumArgs& a, const uint32_t* mat_off, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_accum_diff_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmaSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int n_mb = (a.M + kMmaMics - 1) / kMmaMics, n_bb = (a.F + kMmaBins - 1) / kMmaBins;
    dim3 grid((unsigned)(n_mb * n_bb), (unsigned)a.n_chunks);
    note_launch();
    k_accum_diff_mma<<<grid, kMmaMics * 32, kMmaSmem, s>>>(a, mat_off, n_mb);
    return cudaGetLastError();
}

}  // namespace st
