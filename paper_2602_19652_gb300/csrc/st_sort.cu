// Device-wide primitives: stable LSD radix sort of (u64 key, u32 value) pairs and scans.
//
// Radix sort: 8-bit digits; per pass one histogram kernel over 4096-key tiles, an exclusive
// scan of the digit-major histogram, and a scatter kernel that ranks keys stably inside the
// tile with warp match masks (lanes with equal digits, ordered by lane, warps by index,
// rounds by position), so equal keys keep their input order.
#include "st_internal.cuh"

namespace st {

namespace {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                         uint32_t* __restrict__ hist, int nb) {
    __shared__ uint32_t h[256];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int r = 0; r < kRsItems; ++r) {
        int64_t i = base + (int64_t)r * kRsThreads + tid;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)tid * nb + blockIdx.x] = h[tid];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin,
                                                            uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                            int64_t n, int shift, const uint32_t* __restrict__ offs,
                                                            int nb) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wc[kRsWarps][257];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_base[tid] = offs[(int64_t)tid * nb + blockIdx.x];
    for (int w = 0; w < kRsWarps; ++w) s_wc[w][tid] = 0;
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t i = base + (int64_t)r * kRsThreads + tid;
        const bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0ull;
        uint32_t v = valid ? vin[i] : 0u;
        const int d = valid ? (int)((k >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt_mask);
        const int leader = __ffs(peers) - 1;
        if (lane == leader && valid) s_wc[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = s_base[d] + (uint32_t)rank;
            for (int w = 0; w < warp; ++w) pos += s_wc[w][d];
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        uint32_t sum = 0;
        for (int w = 0; w < kRsWarps; ++w) {
            sum += s_wc[w][tid];
            s_wc[w][tid] = 0;
        }
        s_base[tid] += sum;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- scan
template <class T>
__device__ T warp_incl(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Scans one tile per block (in may equal out); writes the block-local scan (inclusive or exclusive) and the tile total.
template <class T, bool Inclusive>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const T* in, T* out, int64_t n, T* sums) {
    __shared__ T s_w[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
    T v[kScanItems];
    T acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j;
        v[j] = i < n ? in[i] : T(0);
        acc += v[j];
    }
    T incl = warp_incl<T>(acc);
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kScanThreads / 32 ? s_w[lane] : T(0);
        w = warp_incl<T>(w);
        if (lane < kScanThreads / 32) s_w[lane] = w;
    }
    __syncthreads();
    T run = incl - acc + (warp > 0 ? s_w[warp - 1] : T(0));
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j;
        if (Inclusive) run += v[j];
        if (i < n) out[i] = run;
        if (!Inclusive) run += v[j];
    }
    if (tid == kScanThreads - 1 && sums) sums[blockIdx.x] = s_w[kScanThreads / 32 - 1];
}

template <class T>
__global__ void k_scan_add(T* __restrict__ out, int64_t n, const T* __restrict__ add) {
    const int64_t tile = blockIdx.x;
    if (tile == 0) return;
    const T a = add[tile];
    const int64_t base = tile * kScanTile;
    for (int j = threadIdx.x; j < kScanTile; j += blockDim.x) {
        const int64_t i = base + j;
        if (i < n) out[i] += a;
    }
}

template <class T>
__global__ void k_scan_total(const T* in, const T* scanned, int64_t n, T* total) {
    *total = scanned[n - 1] + in[n - 1];
}

// *total holds the last input (saved before an in-place scan); add the last scanned value.
template <class T>
__global__ void k_scan_total_saved(const T* scanned, int64_t n, T* total) {
    *total += scanned[n - 1];
}

template <class T>
size_t scan_bytes_t(int64_t n) {
    size_t b = 0;
    while (n > 1) {
        n = (n + kScanTile - 1) / kScanTile;
        b += ((size_t)n * sizeof(T) + 255) & ~size_t(255);
    }
    return b + 256;
}

// Exclusive scan at every level (block sums are scanned exclusively, then added).
template <class T, bool Inclusive>
cudaError_t scan_impl(const T* in, T* out, int64_t n, void* scratch, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        note_launch();
        k_scan_tile<T, Inclusive><<<1, kScanThreads, 0, s>>>(in, out, n, (T*)nullptr);
        return cudaGetLastError();
    }
    T* sums = static_cast<T*>(scratch);
    char* rest = static_cast<char*>(scratch) + (((size_t)nb * sizeof(T) + 255) & ~size_t(255));
    note_launch();
    k_scan_tile<T, Inclusive><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    cudaError_t e = scan_impl<T, false>(sums, sums, nb, rest, s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_scan_add<T><<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, sums);
    return cudaGetLastError();
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) { return scan_bytes_t<uint64_t>(n); }

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* scratch,
                               cudaStream_t s) {
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return cudaSuccess;
    }
    // `total` needs the last input, which an in-place scan overwrites: keep it first.
    if (in == out && total) {
        cudaError_t e = cudaMemcpyAsync(total, in + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        e = scan_impl<uint32_t, false>(in, out, n, scratch, s);
        if (e != cudaSuccess) return e;
        note_launch();
        k_scan_total_saved<uint32_t><<<1, 1, 0, s>>>(out, n, total);
        return cudaGetLastError();
    }
    cudaError_t e = scan_impl<uint32_t, false>(in, out, n, scratch, s);
    if (e != cudaSuccess || !total) return e;
    note_launch();
    k_scan_total<uint32_t><<<1, 1, 0, s>>>(in, out, n, total);
    return cudaGetLastError();
}

cudaError_t inclusive_scan_u64(const uint64_t* in, uint64_t* out, int64_t n, void* scratch, cudaStream_t s) {
    return scan_impl<uint64_t, true>(in, out, n, scratch, s);
}

size_t sort_scratch_bytes(int64_t n) {
    const int64_t nb = (n + kRsTile - 1) / kRsTile;
    size_t b = ((size_t)n * sizeof(uint64_t) + 255) & ~size_t(255);
    b += ((size_t)n * sizeof(uint32_t) + 255) & ~size_t(255);
    b += (((size_t)nb * 256 * sizeof(uint32_t)) + 255) & ~size_t(255);
    b += scan_bytes_t<uint32_t>(nb * 256);
    return b + 256;
}

cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, void* scratch, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int64_t nb = (n + kRsTile - 1) / kRsTile;
    char* p = static_cast<char*>(scratch);
    uint64_t* k2 = reinterpret_cast<uint64_t*>(p);
    p += ((size_t)n * sizeof(uint64_t) + 255) & ~size_t(255);
    uint32_t* v2 = reinterpret_cast<uint32_t*>(p);
    p += ((size_t)n * sizeof(uint32_t) + 255) & ~size_t(255);
    uint32_t* hist = reinterpret_cast<uint32_t*>(p);
    p += (((size_t)nb * 256 * sizeof(uint32_t)) + 255) & ~size_t(255);
    void* scan_scratch = p;
    int passes = (bits + 7) / 8;
    if (passes & 1) ++passes;  // even pass count: the result ends in the caller's buffers
    if (passes > 8) passes = 8;
    uint64_t* ka = keys;
    uint32_t* va = vals;
    uint64_t* kb = k2;
    uint32_t* vb = v2;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * 8;
        note_launch();
        k_rs_hist<<<(unsigned)nb, kRsThreads, 0, s>>>(ka, n, shift, hist, (int)nb);
        cudaError_t e = scan_impl<uint32_t, false>(hist, hist, nb * 256, scan_scratch, s);
        if (e != cudaSuccess) return e;
        note_launch();
        k_rs_scatter<<<(unsigned)nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, (int)nb);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint64_t* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    return cudaSuccess;
}

}  // namespace st
