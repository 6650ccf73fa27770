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
// a few 1e-6).  When the material changes, and at the end, a warp adds E_q[k] times its accumulators to
// its spectrum registers.  Results are in fixed order for a given launch shape.
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

// D += A B: m16n8k16, bf16 inputs, float32 accumulation
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
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

__global__ void __launch_bounds__(kMmaMics * 32, 3) k_accum_diff_mma(const AccumArgs a, const uint32_t* mat_off,
                                                                    int n_mb) {
    extern __shared__ float4 smem4[];
    char* base = reinterpret_cast<char*>(smem4);
    __nv_bfloat16* Us = reinterpret_cast<__nv_bfloat16*>(base);            // [mic][part][path][kURow]
    __nv_bfloat16* Vs = reinterpret_cast<__nv_bfloat16*>(base + kUBytes);  // [mic][part][path][kVRow]
    float* pd = reinterpret_cast<float*>(base + kUBytes + kVBytes);        // [path][8]: point, r hi, r lo
    int* pq = reinterpret_cast<int*>(pd + kMmaPaths * 8);                  // [path] valid

    const int mb = blockIdx.x % n_mb, bb = blockIdx.x / n_mb;
    const int mic0 = mb * kMmaMics, kb = bb * kMmaBins;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_mat = a.n_mat_tab;

    int64_t n_tiles = 0;
    for (int q = 0; q < n_mat; ++q) n_tiles += ((int64_t)mat_off[q + 1] - mat_off[q] + kMmaPaths - 1) / kMmaPaths;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)blockIdx.y * per, t1 = min(n_tiles, t0 + per);

    // this warp's accumulators: T (current material) and S (spectrum), fragment layout of m16n8 blocks:
    // element i of n-block nb is (k1 = g + 8 (i >> 1), k2 = 8 nb + 2 t + (i & 1))
    float Tr[4][4], Ti[4][4], Sr[4][4], Si[4][4];
#pragma unroll
    for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int i = 0; i < 4; ++i) Tr[nb][i] = Ti[nb][i] = Sr[nb][i] = Si[nb][i] = 0.0f;
    const int g = lane >> 2, t4 = lane & 3;
    const int m_w = mic0 + warp;
    int q_cur = -1;

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
            // U row: z (W^32)^k1, k1 = 0 .. 15, parts re hi, re lo, im hi, im lo
            uint32_t* ur = reinterpret_cast<uint32_t*>(Us + (((size_t)ml * 4) * kMmaPaths + p) * kURow);
            const size_t upart = (size_t)kMmaPaths * kURow / 2;  // words between parts
#pragma unroll
            for (int j = 0; j < kK1 / 8; ++j) {
                uint32_t rh4[4], rl4[4], ih4[4], il4[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 u0 = z;
                    z = cmul(z, w32);
                    const float2 u1 = z;
                    z = cmul(z, w32);
                    split2(u0.x, u1.x, rh4[e], rl4[e]);
                    split2(u0.y, u1.y, ih4[e], il4[e]);
                }
                reinterpret_cast<uint4*>(ur + 0 * upart)[j] = make_uint4(rh4[0], rh4[1], rh4[2], rh4[3]);
                reinterpret_cast<uint4*>(ur + 1 * upart)[j] = make_uint4(rl4[0], rl4[1], rl4[2], rl4[3]);
                reinterpret_cast<uint4*>(ur + 2 * upart)[j] = make_uint4(ih4[0], ih4[1], ih4[2], ih4[3]);
                reinterpret_cast<uint4*>(ur + 3 * upart)[j] = make_uint4(il4[0], il4[1], il4[2], il4[3]);
            }
            // V row: W^k2, k2 = 0 .. 31 (zero for an invalid path or microphone)
            uint32_t* vr = reinterpret_cast<uint32_t*>(Vs + (((size_t)ml * 4) * kMmaPaths + p) * kVRow);
            const size_t vpart = (size_t)kMmaPaths * kVRow / 2;
            float2 v = (pq[p] && m < a.M) ? make_float2(1.0f, 0.0f) : make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < kK2 / 8; ++j) {
                uint32_t rh4[4], rl4[4], ih4[4], il4[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 v0 = v;
                    v = cmul(v, w1);
                    const float2 v1 = v;
                    v = cmul(v, w1);
                    split2(v0.x, v1.x, rh4[e], rl4[e]);
                    split2(v0.y, v1.y, ih4[e], il4[e]);
                }
                reinterpret_cast<uint4*>(vr + 0 * vpart)[j] = make_uint4(rh4[0], rh4[1], rh4[2], rh4[3]);
                reinterpret_cast<uint4*>(vr + 1 * vpart)[j] = make_uint4(rl4[0], rl4[1], rl4[2], rl4[3]);
                reinterpret_cast<uint4*>(vr + 2 * vpart)[j] = make_uint4(ih4[0], ih4[1], ih4[2], ih4[3]);
                reinterpret_cast<uint4*>(vr + 3 * vpart)[j] = make_uint4(il4[0], il4[1], il4[2], il4[3]);
            }
        }
        __syncthreads();
        if (m_w < a.M) {
            if (T.q != q_cur) {
                flush();
                q_cur = T.q;
            }
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
#pragma unroll
                for (int nb2 = 0; nb2 < 2; ++nb2) {
                    // B fragments (16 paths x 8 k2) of n-blocks 2 nb2 and 2 nb2 + 1, from V rows [path][k2]
                    uint32_t B[4][4];
                    const int cb = nb2 * 16 + (mi >> 1) * 8;
#pragma unroll
                    for (int part = 0; part < 4; ++part)
                        ldsm_x4_t(smem_u32(Vw + ((size_t)part * kMmaPaths + pb) * kVRow + cb), B[part][0], B[part][1],
                                  B[part][2], B[part][3]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int nb = 2 * nb2 + h;
                        const uint32_t vrh0 = B[0][2 * h], vrh1 = B[0][2 * h + 1], vrl0 = B[1][2 * h],
                                       vrl1 = B[1][2 * h + 1], vih0 = B[2][2 * h], vih1 = B[2][2 * h + 1],
                                       vil0 = B[3][2 * h], vil1 = B[3][2 * h + 1];
                        // real: Ur Vr - Ui Vi
                        mma_bf16(Tr[nb], A[0], vrh0, vrh1);
                        mma_bf16(Tr[nb], A[0], vrl0, vrl1);
                        mma_bf16(Tr[nb], A[1], vrh0, vrh1);
                        mma_bf16(Tr[nb], nI[0], vih0, vih1);
                        mma_bf16(Tr[nb], nI[0], vil0, vil1);
                        mma_bf16(Tr[nb], nI[1], vih0, vih1);
                        // imaginary: Ur Vi + Ui Vr
                        mma_bf16(Ti[nb], A[0], vih0, vih1);
                        mma_bf16(Ti[nb], A[0], vil0, vil1);
                        mma_bf16(Ti[nb], A[1], vih0, vih1);
                        mma_bf16(Ti[nb], A[2], vrh0, vrh1);
                        mma_bf16(Ti[nb], A[2], vrl0, vrl1);
                        mma_bf16(Ti[nb], A[3], vrh0, vrh1);
                    }
                }
            }
        }
    }
    flush();
    // this chunk's partial spectrum of the warp's microphone
    if (m_w < a.M) {
        float2* out = a.partial + ((size_t)blockIdx.y * a.M + m_w) * a.F;
#pragma unroll
        for (int nb = 0; nb < 4; ++nb)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = kb + kK2 * (g + 8 * (i >> 1)) + 8 * nb + 2 * t4 + (i & 1);
                if (k < a.F) out[k] = make_float2(Sr[nb][i], Si[nb][i]);
            }
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
