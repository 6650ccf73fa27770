// Impulse responses and received signals (Eq. 5-6, 9-10, 13 and the signal equation of Sec. III-F).
//
// Every path's transfer function is M(f) e^{+j 2 pi f r / c}; summed over paths (linearity) the
// impulse response of a component is the inverse transform of its accumulated spectrum S[c][m][k] on
// the uniform grid f_k = f_lo + k df, and the components add.  With the kernel e^{-j 2 pi f t} (the
// convention that puts an echo at t = r / c) and the spectra holding the positive frequencies of a
// real signal, the band-limited response sampled at fs is
//     y[m][n] = 2 df Re sum_k w_k E_k S[m][k] e^{-j 2 pi f_k n / fs},
//     E_k = (1 / fs) sum_i call[i] e^{+j 2 pi f_k i / fs}  (the emitted call's spectrum; 1 without a call),
// i.e. the impulse response convolved with the call.  Phases are reduced in float64 (f_k n / fs can
// reach 10^5 cycles) and rotated in float32 between anchors 32 bins apart.
#include <math.h>

#include "st_internal.cuh"

namespace st {

namespace {

constexpr int kSigThreads = 256;
constexpr int kAnchor = 32;  // bins between float64 re-anchorings of the per-sample phasor

// one block per bin: E_k = (1/fs) sum_i call[i] e^{+j 2 pi f_k i / fs}; fixed-order reduction
__global__ void __launch_bounds__(kSigThreads) k_call_spectrum(const float* call, int L, double f_lo, double df,
                                                               double fs, float2* E) {
    __shared__ float2 red[kSigThreads];
    const int k = blockIdx.x;
    const double fk = (f_lo + (double)k * df) / fs;  // cycles per sample
    float re = 0.0f, im = 0.0f;
    for (int i = threadIdx.x; i < L; i += kSigThreads) {
        const double x = fk * (double)i;
        const float ph = (float)(x - floor(x));
        float s, c;
        sincospif(2.0f * ph, &s, &c);
        const float v = call[i];
        re = fmaf(v, c, re);
        im = fmaf(v, s, im);
    }
    red[threadIdx.x] = make_float2(re, im);
    __syncthreads();
    for (int h = kSigThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[threadIdx.x].x += red[threadIdx.x + h].x;
            red[threadIdx.x].y += red[threadIdx.x + h].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) E[k] = make_float2((float)(red[0].x / fs), (float)(red[0].y / fs));
}

// G[r][k] = w_k E_k S'[r][k] with S' the component sum (rows = mics) or each component (rows = c M + m)
__global__ void k_sig_combine(const float2* S, int n_comp, int M, int F, const float* w, const float2* E, int per_comp,
                              float2* G) {
    const int rows = per_comp ? n_comp * M : M;
    const int64_t n = (int64_t)rows * F;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const int r = (int)(e / F), k = (int)(e - (int64_t)r * F);
        float2 v;
        if (per_comp) {
            v = S[e];
        } else {
            v = make_float2(0.0f, 0.0f);
            for (int c = 0; c < n_comp; ++c) {
                const float2 u = S[((int64_t)c * M + r) * F + k];
                v.x += u.x;
                v.y += u.y;
            }
        }
        if (w) {
            v.x *= w[k];
            v.y *= w[k];
        }
        if (E) {
            const float2 e2 = E[k];
            v = make_float2(v.x * e2.x - v.y * e2.y, v.x * e2.y + v.y * e2.x);
        }
        G[e] = v;
    }
}

// one thread per output sample n of row blockIdx.y: y = 2 df Re sum_k G_k e^{-j 2 pi f_k n / fs}
__global__ void __launch_bounds__(kSigThreads) k_sig_ir(const float2* G, int F, double f_lo, double df, double fs,
                                                        int n_samples, float scale, float* out) {
    __shared__ float2 g[1024];
    const int row = blockIdx.y;
    const int n = blockIdx.x * kSigThreads + threadIdx.x;
    const double tn = (double)n / fs;
    const double a = f_lo * tn, b = df * tn;  // phase (cycles) at bin 0 and per bin
    const double bf = b - floor(b);
    float sb, cb;
    sincospif(-2.0f * (float)bf, &sb, &cb);  // one-bin rotation
    float acc = 0.0f;
    float zr = 0.0f, zi = 0.0f;
    for (int k0 = 0; k0 < F; k0 += 1024) {
        const int nk = min(1024, F - k0);
        __syncthreads();
        for (int i = threadIdx.x; i < nk; i += kSigThreads) g[i] = G[(int64_t)row * F + k0 + i];
        __syncthreads();
        for (int i = 0; i < nk; ++i) {
            const int k = k0 + i;
            if ((k % kAnchor) == 0) {  // exact phasor from the float64 phase
                const double x = a + (double)k * b;
                sincospif(-2.0f * (float)(x - floor(x)), &zi, &zr);
            }
            const float2 gk = g[i];
            acc = fmaf(gk.x, zr, acc);
            acc = fmaf(-gk.y, zi, acc);
            const float nr = zr * cb - zi * sb;
            zi = fmaf(zr, sb, zi * cb);
            zr = nr;
        }
    }
    if (n < n_samples) out[(int64_t)row * n_samples + n] = scale * acc;
}

}  // namespace

cudaError_t signal_response(const float2* S, int n_comp, int M, int F, double f_lo, double f_hi, double fs,
                            int n_samples, const float* window, const float* call, int call_len, int per_comp,
                            float2* E_buf, float2* G_buf, float* out, cudaStream_t s) {
    const double df = F > 1 ? (f_hi - f_lo) / (double)(F - 1) : 1.0;
    cudaError_t e;
    if (call && call_len > 0) {
        note_launch();
        k_call_spectrum<<<F, kSigThreads, 0, s>>>(call, call_len, f_lo, df, fs, E_buf);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int rows = per_comp ? n_comp * M : M;
    note_launch();
    k_sig_combine<<<grid_for((int64_t)rows * F, 256), 256, 0, s>>>(S, n_comp, M, F, window,
                                                                   (call && call_len > 0) ? E_buf : nullptr, per_comp,
                                                                   G_buf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((unsigned)((n_samples + kSigThreads - 1) / kSigThreads), (unsigned)rows);
    note_launch();
    k_sig_ir<<<grid, kSigThreads, 0, s>>>(G_buf, F, f_lo, df, fs, n_samples, (float)(2.0 * df), out);
    return cudaGetLastError();
}

}  // namespace st
