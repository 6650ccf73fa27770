// Float32 geometry helpers for the tracing and pre-processing kernels.
//
// These translation units are compiled with -fmad=false and IEEE division/square root: every
// product is rounded on its own and sums of three terms are taken as (a + b) + c, so the
// results are the same bits as any other IEEE-754 implementation taking the same steps.
// Decisions that produce integers (hit triangle, visibility, sampled triangle) therefore do
// not depend on the device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace st {

struct f3 {
    float x, y, z;
};

__device__ __forceinline__ f3 mk(float x, float y, float z) { return f3{x, y, z}; }
__device__ __forceinline__ f3 sub(f3 a, f3 b) { return f3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) {
    float x = a.x * b.x;
    float y = a.y * b.y;
    float z = a.z * b.z;
    return (x + y) + z;
}
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    float x1 = a.y * b.z, x2 = a.z * b.y;
    float y1 = a.z * b.x, y2 = a.x * b.z;
    float z1 = a.x * b.y, z2 = a.y * b.x;
    return f3{x1 - x2, y1 - y2, z1 - z2};
}
// v / |v|, |v| = sqrt((x*x + y*y) + z*z); zero stays zero.  Returns |v| in *len.
__device__ __forceinline__ f3 normalize(f3 v, float* len) {
    float l = sqrtf(dot(v, v));
    *len = l;
    if (l > 0.0f) return f3{v.x / l, v.y / l, v.z / l};
    return f3{0.0f, 0.0f, 0.0f};
}
__device__ __forceinline__ float comp(f3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// One row of an instance's affine map x -> A x + b: ((A_r0 x + A_r1 y) + A_r2 z) + b_r with row = (A_r0, A_r1,
// A_r2, b_r), every product and sum rounded on its own.  The instance expansion and the two-level traversal's
// world-space triangle test both use it, so a triangle reached through either has the same vertices.
__device__ __forceinline__ float affine_row(float4 row, float x, float y, float z) {
    return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(row.x, x), __fmul_rn(row.y, y)), __fmul_rn(row.z, z)), row.w);
}

// q = (w, x, y, z) applied to v: t = 2 (q_v x v); v' = (v + w t) + q_v x t.
__device__ __forceinline__ f3 rotate(const float q[4], f3 v) {
    f3 qv{q[1], q[2], q[3]};
    f3 c = cross(qv, v);
    f3 t{2.0f * c.x, 2.0f * c.y, 2.0f * c.z};
    f3 c2 = cross(qv, t);
    float wx = q[0] * t.x, wy = q[0] * t.y, wz = q[0] * t.z;
    float ax = v.x + wx, ay = v.y + wy, az = v.z + wz;
    return f3{ax + c2.x, ay + c2.y, az + c2.z};
}

// ---------------------------------------------------------------- watertight ray-triangle test
// Woop, Benthin, Wald, "Watertight ray/triangle intersection", JCGT 2(1), 2013: shear the
// triangle into the ray's frame (largest |d| component as z), 2D edge functions U, V, W,
// two-sided sign test, t = T / det.  Float32 only.
struct WRay {
    f3 o;
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

__device__ __forceinline__ WRay wray(f3 o, f3 d) {
    WRay r;
    r.o = o;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax >= ay) ? ((ax >= az) ? 0 : 2) : ((ay >= az) ? 1 : 2);
    int kx = kz + 1;
    if (kx == 3) kx = 0;
    int ky = kx + 1;
    if (ky == 3) ky = 0;
    float dz = comp(d, kz);
    if (dz < 0.0f) {
        int t = kx;
        kx = ky;
        ky = t;
    }
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    r.Sx = comp(d, kx) / dz;
    r.Sy = comp(d, ky) / dz;
    r.Sz = 1.0f / dz;
    return r;
}

__device__ __forceinline__ bool wt_hit(const WRay& r, f3 v0, f3 v1, f3 v2, float* t) {
    f3 A = sub(v0, r.o), B = sub(v1, r.o), C = sub(v2, r.o);
    float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    float p;
    p = r.Sx * Akz; float Ax = comp(A, r.kx) - p;
    p = r.Sy * Akz; float Ay = comp(A, r.ky) - p;
    p = r.Sx * Bkz; float Bx = comp(B, r.kx) - p;
    p = r.Sy * Bkz; float By = comp(B, r.ky) - p;
    p = r.Sx * Ckz; float Cx = comp(C, r.kx) - p;
    p = r.Sy * Ckz; float Cy = comp(C, r.ky) - p;
    float u1 = Cx * By, u2 = Cy * Bx;
    float U = u1 - u2;
    float v1_ = Ax * Cy, v2_ = Ay * Cx;
    float V = v1_ - v2_;
    float w1 = Bx * Ay, w2 = By * Ax;
    float W = w1 - w2;
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    float det = (U + V) + W;
    if (det == 0.0f) return false;
    float Az = r.Sz * Akz, Bz = r.Sz * Bkz, Cz = r.Sz * Ckz;
    float t1 = U * Az, t2 = V * Bz, t3 = W * Cz;
    float T = (t1 + t2) + t3;
    *t = T / det;
    return true;
}

}  // namespace st
