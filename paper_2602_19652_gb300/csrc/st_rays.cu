// Emitter ray sets on the device: the spherical Fibonacci lattice and the centre points of the
// recursive zonal equal-area partition of the sphere (Leopardi 2006; the paper's ray set, Sec.
// III-C).  The zone table (cumulative region counts, per-zone colatitude and longitude offset) is
// built on the host in float64; one thread per direction finds its zone and evaluates it in float64,
// rounding to float32 once.  Compiled with -fmad=false (no contraction of the float64 steps).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "st_internal.cuh"

namespace st {

namespace {

__global__ void k_fibonacci(int64_t n, float* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double golden = M_PI * (3.0 - sqrt(5.0));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;
        const double rho = sqrt(fmax(0.0, 1.0 - z * z));
        const double phi = (double)i * golden;
        double s, c;
        sincos(phi, &s, &c);
        out[3 * i] = (float)(rho * c);
        out[3 * i + 1] = (float)(rho * s);
        out[3 * i + 2] = (float)z;
    }
}

// zone z holds regions cum[z] .. cum[z+1]-1 at colatitude with (sin, cos) = zsc[z], longitude offset off[z]
__global__ void k_zonal(int64_t n, int n_zones, const int64_t* cum, const double2* zsc, const double* off,
                        float* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int lo = 0, hi = n_zones;  // last zone with cum[z] <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (cum[mid] <= i) lo = mid; else hi = mid;
        }
        const int64_t m = cum[lo + 1] - cum[lo];
        const double j = (double)(i - cum[lo]);
        double x, y, z;
        if (m == 1 && (lo == 0 || lo == n_zones - 1)) {  // polar caps
            x = 0.0;
            y = 0.0;
            z = lo == 0 ? 1.0 : -1.0;
        } else {
            const double phi = off[lo] + (j + 0.5) * (2.0 * M_PI / (double)m);
            double s, c;
            sincos(phi, &s, &c);
            x = zsc[lo].x * c;
            y = zsc[lo].x * s;
            z = zsc[lo].y;
        }
        out[3 * i] = (float)x;
        out[3 * i + 1] = (float)y;
        out[3 * i + 2] = (float)z;
    }
}

}  // namespace

// zone table of the zonal partition (float64 on the host): cumulative counts, (sin, cos) of the zone's
// centre colatitude, longitude offsets
void zonal_table(int64_t n, std::vector<int64_t>& cum, std::vector<double>& zs, std::vector<double>& zc,
                 std::vector<double>& off) {
    cum.assign(1, 0);
    std::vector<int64_t> counts;
    if (n <= 2) {
        for (int64_t k = 0; k < n; ++k) counts.push_back(1);
    } else {
        const double area = 4.0 * M_PI / (double)n;
        const double theta_c = 2.0 * asin(sqrt(1.0 / (double)n));
        const double ideal = sqrt(area);
        const int64_t n_collars = std::max<int64_t>(1, (int64_t)llround((M_PI - 2.0 * theta_c) / ideal));
        const double fit = (M_PI - 2.0 * theta_c) / (double)n_collars;
        counts.push_back(1);
        double carry = 0.0;
        for (int64_t i = 0; i < n_collars; ++i) {
            const double t0 = theta_c + (double)i * fit, t1 = theta_c + (double)(i + 1) * fit;
            const double y = 2.0 * M_PI * (cos(t0) - cos(t1)) / area;
            const int64_t m = (int64_t)llround(y + carry);
            carry += y - (double)m;
            counts.push_back(m);
        }
        counts.push_back(1);
    }
    for (int64_t m : counts) cum.push_back(cum.back() + m);
    const size_t nz = counts.size();
    zs.assign(nz, 0.0);
    zc.assign(nz, 0.0);
    off.assign(nz, 0.0);
    double offset = 0.0;
    for (size_t z = 0; z < nz; ++z) {
        const double t0 = 2.0 * asin(sqrt(std::min(1.0, (double)cum[z] / (double)n)));
        const double t1 = 2.0 * asin(sqrt(std::min(1.0, (double)cum[z + 1] / (double)n)));
        const double th = 0.5 * (t0 + t1);
        zs[z] = sin(th);
        zc[z] = cos(th);
        if (z >= 2 && z + 1 < nz) offset = fmod(offset + M_PI / (double)counts[z], 2.0 * M_PI);
        off[z] = offset;
    }
}

cudaError_t ray_directions(int kind, int64_t n, float* out, DevBuf& scratch, cudaStream_t s) {
    if (kind == 0) {
        note_launch();
        k_fibonacci<<<grid_for(n, 256), 256, 0, s>>>(n, out);
        return cudaGetLastError();
    }
    std::vector<int64_t> cum;
    std::vector<double> zs, zc, off;
    zonal_table(n, cum, zs, zc, off);
    const int nz = (int)zs.size();
    std::vector<double> packed;  // zsc [nz] double2, then off [nz], then cum [nz+1] (as raw 8-byte words)
    packed.resize((size_t)3 * nz + nz + 1);
    for (int z = 0; z < nz; ++z) {
        packed[2 * z] = zs[z];
        packed[2 * z + 1] = zc[z];
        packed[(size_t)2 * nz + z] = off[z];
    }
    memcpy(&packed[(size_t)3 * nz], cum.data(), (size_t)(nz + 1) * 8);
    cudaError_t e = grow(scratch, packed.size() * 8);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(scratch.p, packed.data(), packed.size() * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;  // the host table is released on return
    const double* base = ptr<double>(scratch);
    note_launch();
    k_zonal<<<grid_for(n, 256), 256, 0, s>>>(n, nz, reinterpret_cast<const int64_t*>(base + 3 * nz),
                                            reinterpret_cast<const double2*>(base), base + 2 * nz, out);
    return cudaGetLastError();
}

}  // namespace st
