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
struct Geom {
    int TM, NS, MT, KB, PT;
    int n_mb, n_bb;
    size_t smem;
};

template <int KT, int R>
__global__ void __launch_bounds__(256) k_accum(const AccumArgs a, const Geom g) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const int PT = g.PT, NS = g.NS, MT = g.MT, KB = g.KB, TM = g.TM;
    float2* tab = reinterpret_cast<float2*>(sm);                       // [PT][KT][NS]  (log2 X D_e, g)
    float2* zs = tab + (size_t)PT * KB;                                // [PT][NS][MT]
    float2* Wm = zs + (size_t)PT * NS * MT;                            // [PT][MT]
    float* ngm = reinterpret_cast<float*>(Wm + (size_t)PT * MT);       // [PT][MT]  -gamma^2
    float* pd = ngm + (size_t)PT * MT;                                 // [PT][12] path data
    int* pvalid = reinterpret_cast<int*>(pd + (size_t)PT * 12);        // [PT]

    const int mb = blockIdx.x % g.n_mb, bb = blockIdx.x / g.n_mb;
    const int mic0 = mb * MT, kb = bb * KB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tm = tid % TM, s = tid / TM;

    const int64_t count = (int64_t)*a.d_count;
    const int64_t n_tiles = (count + PT - 1) / PT;
    const int64_t per = (n_tiles + a.n_chunks - 1) / a.n_chunks;
    const int64_t t0 = (int64_t)blockIdx.y * per, t1 = min(n_tiles, t0 + per);

    float2 S[R][KT];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) S[r][kk] = make_float2(0.0f, 0.0f);

    const float dq_hi = a.dq_hi, dq_lo = a.dq_lo;
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t pbase = tile * PT;
        // ---- path data
        for (int p = tid; p < PT; p += nthr) {
            const int64_t pi = pbase + p;
            const bool ok = pi < count;
            pvalid[p] = ok;
            float* d = pd + p * 12;
            if (ok) {
                d[0] = a.px[pi];
                d[1] = a.py[pi];
                d[2] = a.pz[pi];
                d[3] = a.kind == 0 ? a.dx[pi] : 0.0f;
                d[4] = a.kind == 0 ? a.dy[pi] : 0.0f;
                d[5] = a.kind == 0 ? a.dz[pi] : 0.0f;
                d[6] = a.rhi[pi];
                d[7] = a.rlo[pi];
                d[8] = __uint_as_float(a.meta[pi]);
                d[9] = a.kind == 0 ? __uint_as_float(a.chain_lo[pi]) : 0.0f;
                d[10] = a.kind == 0 ? __uint_as_float(a.chain_hi[pi]) : 0.0f;
                d[11] = a.dep ? a.dep[pi] : -1.0f;
            }
        }
        __syncthreads();
        // ---- 1a: per (path, bin) log2 amplitude factors and lobe exponents
        for (int e = tid; e < PT * KB; e += nthr) {
            const int p = e / KB, kl = e % KB;  // kl = s_ * KT + kk
            const int k = kb + kl;
            float lx = kNegInf, gg = 0.0f;
            if (pvalid[p] && k < a.F) {
                const float* d = pd + p * 12;
                const uint32_t meta = __float_as_uint(d[8]);
                const int len = meta & 15, matj = (meta >> 8) & 255;
                if (a.kind == 0) {
                    if (a.reflection_mode == 1) {
                        lx = a.lk[(int64_t)matj * a.F + k];
                    } else {
                        const uint32_t c0 = __float_as_uint(d[9]), c1 = __float_as_uint(d[10]);
                        float acc = 0.0f;
                        for (int q = 0; q < len; ++q) {
                            const int mq = (q < 4 ? (c0 >> (8 * q)) : (c1 >> (8 * (q - 4)))) & 255;
                            acc += a.lk[(int64_t)mq * a.F + k];
                        }
                        lx = acc;
                    }
                    gg = a.g2[(int64_t)matj * a.F + k];
                } else {
                    lx = a.lid[(int64_t)matj * a.F + k];
                }
                if (a.etab && d[11] >= 0.0f) {
                    const float x = d[11];
                    int i = min((int)x, a.n_theta - 2);
                    const float w = x - (float)i;
                    const float de = (1.0f - w) * a.etab[(int64_t)i * a.F + k] + w * a.etab[(int64_t)(i + 1) * a.F + k];
                    lx += de > 0.0f ? log2f(de) : kNegInf;
                }
            }
            const int s_ = kl / KT, kk = kl % KT;
            tab[(p * KT + kk) * NS + s_] = make_float2(lx, gg);
        }
        // ---- 1b: per (path, mic) anchors
        for (int e = tid; e < PT * MT; e += nthr) {
            const int p = e / MT, ml = e % MT;
            const int m = mic0 + ml;
            float2* zrow = zs + (size_t)p * NS * MT + ml;
            if (!pvalid[p] || m >= a.M) {
                for (int s_ = 0; s_ < NS; ++s_) zrow[(size_t)s_ * MT] = make_float2(0.0f, 0.0f);
                Wm[p * MT + ml] = make_float2(0.0f, 0.0f);
                ngm[p * MT + ml] = 0.0f;
                continue;
            }
            const float* d = pd + p * 12;
            const float mx = a.mics[3 * m], my = a.mics[3 * m + 1], mz = a.mics[3 * m + 2];
            const ff dist = dist_ff(mx, my, mz, d[0], d[1], d[2]);
            const ff r = ff_add(ff{d[6], d[7]}, dist);
            float gam2 = 0.0f;
            if (a.kind == 0) {
                const float inv = 1.0f / dist.hi;
                const float ux = (mx - d[0]) * inv, uy = (my - d[1]) * inv, uz = (mz - d[2]) * inv;
                const float cg = d[3] * ux + d[4] * uy + d[5] * uz;
                const float cx = d[4] * uz - d[5] * uy, cy = d[5] * ux - d[3] * uz, cz = d[3] * uy - d[4] * ux;
                const float sg = sqrtf(cx * cx + cy * cy + cz * cz);
                const float gm = atan2f(sg, cg);
                gam2 = gm * gm;
            }
            const float rh = r.hi;
            // amplitude at bin kb: -2 log2 r + r * atm2(kb)
            const float L0 = -2.0f * log2_ff(r) + rh * (a.atm2_0 + a.atm2_step * (float)kb);
            const ff x0 = ff_mul(r, ff{a.qhi[min(kb, a.F - 1)], a.qlo[min(kb, a.F - 1)]});
            float s0, c0;
            sincospif(2.0f * ff_frac(x0), &s0, &c0);
            const float A0 = ex2(L0);
            float2 z = make_float2(A0 * c0, A0 * s0);
            const ff xs = ff_mul(r, ff{dq_hi, dq_lo});
            float s1, c1;
            sincospif(2.0f * ff_frac(xs), &s1, &c1);
            const float a1 = ex2(rh * a.atm2_step);
            Wm[p * MT + ml] = make_float2(a1 * c1, a1 * s1);
            const ff xk = ff_mul(r, ff{dq_hi * (float)KT, dq_lo * (float)KT});
            float s2, c2;
            sincospif(2.0f * ff_frac(xk), &s2, &c2);
            const float a2 = ex2(rh * a.atm2_step * (float)KT);
            const float2 WK = make_float2(a2 * c2, a2 * s2);
            for (int s_ = 0; s_ < NS; ++s_) {
                zrow[(size_t)s_ * MT] = z;
                z = cmul(z, WK);
            }
            ngm[p * MT + ml] = -gam2;
        }
        __syncthreads();
        // ---- 2: terms
        if (s < NS) {
            for (int p = 0; p < PT; ++p) {
                float2 z[R], W[R];
                float ng[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int ml = tm * R + r;
                    z[r] = zs[((size_t)p * NS + s) * MT + ml];
                    W[r] = Wm[p * MT + ml];
                    ng[r] = ngm[p * MT + ml];
                }
                const float2* trow = tab + (size_t)p * KB + s;
#pragma unroll
                for (int kk = 0; kk < KT; ++kk) {
                    const float2 t = trow[kk * NS];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float e = ex2(fmaf(ng[r], t.y, t.x));
                        S[r][kk].x = fmaf(e, z[r].x, S[r][kk].x);
                        S[r][kk].y = fmaf(e, z[r].y, S[r][kk].y);
                        z[r] = cmul(z[r], W[r]);
                    }
                }
            }
        }
        __syncthreads();
    }
    // ---- partial spectra of this chunk
    if (s < NS) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = mic0 + tm * R + r;
            if (m >= a.M) continue;
            float2* out = a.partial + ((size_t)blockIdx.y * a.M + m) * a.F;
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) {
                const int k = kb + s * KT + kk;
                if (k < a.F) out[k] = S[r][kk];
            }
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

Geom make_geom(int M, int F, int KT, int R) {
    Geom g;
    g.TM = std::min((M + R - 1) / R, 32);
    int ns_need = (F + KT - 1) / KT;
    g.NS = std::max(1, std::min(ns_need, 256 / g.TM));
    g.MT = g.TM * R;
    g.KB = g.NS * KT;
    g.n_mb = (M + g.MT - 1) / g.MT;
    g.n_bb = (F + g.KB - 1) / g.KB;
    const size_t per_path = (size_t)g.KB * 8 + (size_t)g.NS * g.MT * 8 + (size_t)g.MT * 12 + 12 * 4 + 4;
    int pt = (int)std::min<size_t>(32, std::max<size_t>(1, (56 * 1024) / per_path));
    g.PT = pt;
    g.smem = per_path * pt + 64;
    return g;
}

template <int KT, int R>
cudaError_t launch_accum(const AccumArgs& a, cudaStream_t s) {
    const Geom g = make_geom(a.M, a.F, KT, R);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_accum<KT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)(g.n_mb * g.n_bb), (unsigned)a.n_chunks);
    note_launch();
    k_accum<KT, R><<<grid, g.TM * g.NS, g.smem, s>>>(a, g);
    return cudaGetLastError();
}

}  // namespace

int32_t accum_chunks(int64_t n_paths_hint, int32_t M, int32_t F) {
    const int R = M >= 2 ? 2 : 1;
    const Geom g = make_geom(M, F, 16, R);
    const int ctas_per_chunk = g.n_mb * g.n_bb;
    const int threads = g.TM * g.NS;
    int resident = std::max(1, std::min(2048 / std::max(threads, 32), (int)((200 * 1024) / std::max<size_t>(g.smem, 1))));
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
    if (a.M >= 2) return launch_accum<16, 2>(a, s);
    return launch_accum<16, 1>(a, s);
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
