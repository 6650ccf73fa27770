// Allocation-free specular accumulation.
//
// Some callers cannot allocate device memory at the point where they need spectra: code running
// under a memory budget owned by another allocator (a framework's caching allocator or a fixed
// arena), code in real-time loops where a cudaMalloc would stall or synchronise the device, or
// code issued from a callback where allocation is not allowed.  For them this file provides
// st_accumulate_specular_noalloc: the same specular spectrum as st_simulate's accumulation, from
// path records the caller passes, using only a fixed scratch array compiled into the library.
//
// Scratch: g_noalloc_scratch, ST_NOALLOC_SCRATCH_BYTES bytes of device memory that every GPU which
// loads the library holds until the process exits.  It holds the per-bin material tables and the
// per-chunk partial spectra.  All calls share it: two calls that overlap on the GPU (different
// streams, or different threads without ordering) race on it and give wrong results.  Every call
// overwrites all of the scratch it reads, so no state carries over between calls.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "st_internal.cuh"

namespace {

constexpr size_t kScratchBytes = ST_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kChunksMax = 64;
constexpr int kThreads = 256;
constexpr int kTile = 64;
constexpr int kMaxChain = 8;  // the largest max_bounces the entry point accepts

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of g_noalloc_scratch per device (host code may not use the symbol itself)
void* g_scratch_addr[kMaxDevices] = {nullptr};

struct Layout {
    size_t band, kb, beta, lk, g2, qhi, qlo, partial, end;
};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

Layout layout(int n_mat, int n_bands, int F, int M, int chunks) {
    Layout L;
    size_t o = 0;
    L.band = o; o = up256(o + (size_t)n_bands * 4);
    L.kb = o; o = up256(o + (size_t)n_mat * n_bands * 4);
    L.beta = o; o = up256(o + (size_t)n_mat * n_bands * 4);
    L.lk = o; o = up256(o + (size_t)n_mat * F * 4);
    L.g2 = o; o = up256(o + (size_t)n_mat * F * 4);
    L.qhi = o; o = up256(o + (size_t)F * 4);
    L.qlo = o; o = up256(o + (size_t)F * 4);
    L.partial = o; o = up256(o + (size_t)chunks * M * F * 8);
    L.end = o;
    return L;
}

// per-bin tables: log2 k(mat, f_k), lobe exponent 1/(2 beta^2) * log2(e) (linear in f between band
// centres, constant beyond), and f_k / c as a float-float pair
__global__ void k_na_tables(int F, int n_mat, int n_bands, const float* band, const float* kb, const float* beta,
                            double f_lo, double df, double c, float* lk, float* g2, float* qhi, float* qlo) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F * n_mat) return;
    const int mat = idx / F, k = idx % F;
    const double f = F == 1 ? f_lo : f_lo + (double)k * df;
    int b0 = 0;
    double w = 0.0;
    if (n_bands > 1) {
        if (f <= (double)band[0]) {
            b0 = 0;
            w = 0.0;
        } else if (f >= (double)band[n_bands - 1]) {
            b0 = n_bands - 2;
            w = 1.0;
        } else {
            while (b0 + 1 < n_bands && (double)band[b0 + 1] <= f) ++b0;
            if (b0 >= n_bands - 1) b0 = n_bands - 2;
            w = (f - (double)band[b0]) / ((double)band[b0 + 1] - (double)band[b0]);
        }
    }
    const float* kr = kb + (size_t)mat * n_bands;
    const float* br = beta + (size_t)mat * n_bands;
    double kv = kr[b0], g = 1.0 / (2.0 * (double)br[b0] * (double)br[b0]);
    if (n_bands > 1) {
        kv = (1.0 - w) * (double)kr[b0] + w * (double)kr[b0 + 1];
        g = (1.0 - w) * g + w / (2.0 * (double)br[b0 + 1] * (double)br[b0 + 1]);
    }
    lk[idx] = kv > 0.0 ? (float)log2(kv) : -__builtin_huge_valf();
    g2[idx] = (float)(g * 1.4426950408889634);
    if (mat == 0) {
        const double q = f / c;
        const float h = (float)q;
        qhi[k] = h;
        qlo[k] = (float)(q - (double)h);
    }
}

struct ff2 {
    float hi, lo;
};
__device__ __forceinline__ ff2 na_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return ff2{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff2 na_fast(float a, float b) {
    const float s = a + b;
    return ff2{s, b - (s - a)};
}
__device__ __forceinline__ ff2 na_add(ff2 x, ff2 y) {
    const ff2 s = na_two_sum(x.hi, y.hi);
    return na_fast(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ff2 na_mul(ff2 x, ff2 y) {
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.hi, -p) + fmaf(x.hi, y.lo, x.lo * y.hi);
    return na_fast(p, e);
}
__device__ __forceinline__ ff2 na_sq(float a, float b) {  // (a - b)^2 as float-float, a - b exact as a pair
    const ff2 d = na_two_sum(a, -b);
    const float p = d.hi * d.hi;
    return ff2{p, fmaf(d.hi, d.hi, -p) + 2.0f * d.hi * d.lo};
}
__device__ __forceinline__ ff2 na_sqrt(ff2 x) {
    if (!(x.hi > 0.0f)) return ff2{0.0f, 0.0f};
    const float s = sqrtf(x.hi);
    const float p = s * s;
    const float e = fmaf(s, s, -p);
    return na_fast(s, (((x.hi - p) - e) + x.lo) / (2.0f * s));
}

// One thread per (microphone, bin) output; the block's records chunk is streamed through shared
// memory; each term is evaluated directly (float-float path length and phase reduction, sincospi).
__global__ void __launch_bounds__(kThreads) k_na_accum(const int32_t* rec_tri, const float* rec_p, const float* rec_d,
                                                       const double* rec_r, const uint8_t* rec_los, int64_t n_rec,
                                                       int B, const int32_t* tri_mat, int64_t n_tris,
                                                       const float* mics, int M, int F,
                                                       int n_mat, int reflection_mode, float atm2_0,
                                                       float atm2_step, size_t off_lk, size_t off_g2, size_t off_qhi,
                                                       size_t off_qlo, size_t off_partial, int chunks) {
    const float* lk = reinterpret_cast<const float*>(g_noalloc_scratch + off_lk);
    const float* g2 = reinterpret_cast<const float*>(g_noalloc_scratch + off_g2);
    const float* qhi = reinterpret_cast<const float*>(g_noalloc_scratch + off_qhi);
    const float* qlo = reinterpret_cast<const float*>(g_noalloc_scratch + off_qlo);
    float2* partial = reinterpret_cast<float2*>(g_noalloc_scratch + off_partial);
    __shared__ float sp[kTile][8];       // P.xyz, d'.xyz, r hi, r lo
    __shared__ int32_t sm[kTile][2 + kMaxChain];  // valid, chain length, materials of hits 0..j
    const int64_t o = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = o < (int64_t)M * F;
    const int m = active ? (int)(o / F) : 0, k = active ? (int)(o % F) : 0;
    const float mx = mics[3 * m], my = mics[3 * m + 1], mz = mics[3 * m + 2];
    const ff2 q{qhi[k], qlo[k]};
    const float atm = atm2_0 + atm2_step * (float)k;
    const int64_t per = (n_rec + chunks - 1) / chunks;
    const int64_t r0 = (int64_t)blockIdx.y * per, r1 = min(n_rec, r0 + per);
    float sx = 0.0f, sy = 0.0f;
    for (int64_t base = r0; base < r1; base += kTile) {
        __syncthreads();
        for (int t = threadIdx.x; t < kTile; t += kThreads) {
            const int64_t id = base + t;
            int valid = 0;
            if (id < r1 && rec_tri[id] >= 0 && rec_los[id]) valid = 1;
            sm[t][0] = valid;
            if (valid) {
                const int64_t ray = id / B;
                const int j = (int)(id % B);  // j < B <= kMaxChain
                for (int c = 0; c < 3; ++c) {
                    sp[t][c] = rec_p[3 * id + c];
                    sp[t][3 + c] = rec_d[3 * id + c];
                }
                const double r = rec_r[id];
                sp[t][6] = (float)r;
                sp[t][7] = (float)(r - (double)(float)r);
                sm[t][1] = j + 1;
                // a chain whose triangle or material id is out of range contributes nothing (the
                // ids come from the caller; nothing is read outside tri_mat or the tables)
                for (int qq = 0; qq <= j; ++qq) {
                    const int32_t tri = rec_tri[ray * B + qq];
                    const int32_t mat = (tri >= 0 && (int64_t)tri < n_tris) ? tri_mat[tri] : -1;
                    if (mat < 0 || mat >= n_mat) {
                        valid = 0;
                        break;
                    }
                    sm[t][2 + qq] = mat;
                }
                sm[t][0] = valid;
            }
        }
        __syncthreads();
        if (!active) continue;
        for (int t = 0; t < kTile; ++t) {
            if (!sm[t][0]) continue;
            const ff2 dist = na_sqrt(na_add(na_add(na_sq(mx, sp[t][0]), na_sq(my, sp[t][1])), na_sq(mz, sp[t][2])));
            const ff2 r = na_add(ff2{sp[t][6], sp[t][7]}, dist);
            const float inv = 1.0f / dist.hi;
            const float ux = (mx - sp[t][0]) * inv, uy = (my - sp[t][1]) * inv, uz = (mz - sp[t][2]) * inv;
            const float dx = sp[t][3], dy = sp[t][4], dz = sp[t][5];
            const float cg = dx * ux + dy * uy + dz * uz;
            const float cx = dy * uz - dz * uy, cy = dz * ux - dx * uz, cz = dx * uy - dy * ux;
            const float gm = atan2f(sqrtf(cx * cx + cy * cy + cz * cz), cg);
            const int len = sm[t][1];
            const int matj = sm[t][1 + len];
            float lx = 0.0f;
            if (reflection_mode == 1) {
                lx = lk[(size_t)matj * F + k];
            } else {
                for (int qq = 0; qq < len; ++qq) lx += lk[(size_t)sm[t][2 + qq] * F + k];
            }
            const float L = lx - gm * gm * g2[(size_t)matj * F + k] - 2.0f * (log2f(r.hi) + r.lo / (r.hi * 0.6931472f)) +
                            r.hi * atm;
            const ff2 x = na_mul(r, q);
            const float n = rintf(x.hi);
            float sn, cs;
            sincospif(2.0f * ((x.hi - n) + x.lo), &sn, &cs);
            const float A = exp2f(L);
            sx = fmaf(A, cs, sx);
            sy = fmaf(A, sn, sy);
        }
    }
    if (active) partial[(size_t)blockIdx.y * M * F + o] = make_float2(sx, sy);
}

__global__ void k_na_reduce(size_t off_partial, int chunks, int64_t MF, float2* out) {
    const float2* partial = reinterpret_cast<const float2*>(g_noalloc_scratch + off_partial);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MF; i += stride) {
        float sx = 0.0f, sy = 0.0f;
        for (int c = 0; c < chunks; ++c) {
            const float2 v = partial[(size_t)c * MF + i];
            sx += v.x;
            sy += v.y;
        }
        out[i] = make_float2(sx, sy);
    }
}

}  // namespace

extern "C" __attribute__((visibility("default"))) st_status st_accumulate_specular_noalloc(const int32_t* rec_tri, const float* rec_point,
                                                     const float* rec_dir, const double* rec_r, const uint8_t* rec_los,
                                                     int64_t n_rays, int32_t max_bounces, const int32_t* tri_material,
                                                     int64_t n_tris, const float* mics, int32_t n_mics, int32_t n_bins, double f_lo,
                                                     double f_hi, int32_t n_mat, int32_t n_bands, const float* band_hz,
                                                     const float* k, const float* beta, const st_sim_params* params,
                                                     void* spectra_out, void* cuda_stream) {
    if (!rec_tri || !rec_point || !rec_dir || !rec_r || !rec_los || !tri_material || !mics || !band_hz || !k ||
        !beta || !spectra_out || n_rays < 0 || max_bounces < 1 || max_bounces > kMaxChain || n_tris < 1 ||
        n_mics < 1 || n_bins < 1 ||
        n_mat < 1 || n_mat > 255 || n_bands < 1 || n_bands > 64 || !(f_lo > 0.0) || !(f_hi >= f_lo))
        return ST_ERR_ARG;
    st_sim_params p;
    st_sim_params_default(&p);
    if (params) p = *params;
    if (!(p.c > 0.0) || p.reflection_mode < 0 || p.reflection_mode > 1) return ST_ERR_ARG;
    // size check: tables plus at least one chunk of partial spectra must fit the fixed scratch
    const Layout one = layout(n_mat, n_bands, n_bins, n_mics, 1);
    if (one.end > kScratchBytes || n_rays * max_bounces >= ((int64_t)1 << 40)) return ST_ERR_ARG;
    int chunks = 1;
    while (chunks < kChunksMax && layout(n_mat, n_bands, n_bins, n_mics, chunks * 2).end <= kScratchBytes) chunks *= 2;
    const Layout Lo = layout(n_mat, n_bands, n_bins, n_mics, chunks);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ST_ERR_CUDA;
    if (!g_scratch_addr[dev]) {
        // first call on this device: look up the scratch's device address (no allocation)
        void* a = nullptr;
        if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess || !a) return ST_ERR_CUDA;
        g_scratch_addr[dev] = a;
    }
    unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaMemcpyAsync(base + Lo.band, band_hz, (size_t)n_bands * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + Lo.kb, k, (size_t)n_mat * n_bands * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + Lo.beta, beta, (size_t)n_mat * n_bands * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return ST_ERR_CUDA;
    const double df = n_bins > 1 ? (f_hi - f_lo) / (double)(n_bins - 1) : 0.0;
    st::note_launch();
    k_na_tables<<<(n_bins * n_mat + 127) / 128, 128, 0, s>>>(
        n_bins, n_mat, n_bands, reinterpret_cast<const float*>(base + Lo.band),
        reinterpret_cast<const float*>(base + Lo.kb), reinterpret_cast<const float*>(base + Lo.beta), f_lo, df, p.c,
        reinterpret_cast<float*>(base + Lo.lk), reinterpret_cast<float*>(base + Lo.g2),
        reinterpret_cast<float*>(base + Lo.qhi), reinterpret_cast<float*>(base + Lo.qlo));
    if (cudaGetLastError() != cudaSuccess) return ST_ERR_CUDA;
    const double l2 = log2(10.0) / 20.0;
    const float atm2_0 = (float)(-(p.alpha0_db_m + p.alpha1_db_m_khz * f_lo / 1000.0) * l2);
    const float atm2_step = (float)(-(p.alpha1_db_m_khz * df / 1000.0) * l2);
    const int64_t MF = (int64_t)n_mics * n_bins;
    dim3 grid((unsigned)((MF + kThreads - 1) / kThreads), (unsigned)chunks);
    st::note_launch();
    k_na_accum<<<grid, kThreads, 0, s>>>(rec_tri, rec_point, rec_dir, rec_r, rec_los, n_rays * max_bounces,
                                         max_bounces, tri_material, n_tris, mics, n_mics, n_bins, n_mat,
                                         p.reflection_mode,
                                         atm2_0, atm2_step, Lo.lk, Lo.g2, Lo.qhi, Lo.qlo, Lo.partial, chunks);
    if (cudaGetLastError() != cudaSuccess) return ST_ERR_CUDA;
    st::note_launch();
    k_na_reduce<<<st::grid_for(MF, 256), 256, 0, s>>>(Lo.partial, chunks, MF, static_cast<float2*>(spectra_out));
    if (cudaGetLastError() != cudaSuccess) return ST_ERR_CUDA;
    return ST_OK;
}
