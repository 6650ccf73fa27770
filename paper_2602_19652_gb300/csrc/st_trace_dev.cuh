// Device code shared by the single-pose and batched tracing kernels: BVH traversal (closest and any
// hit), visibility rays and Philox4x32-10.  Included only by translation units compiled with
// -fmad=false (see st_geom.cuh).
#pragma once

#include "st_geom.cuh"
#include "st_internal.cuh"

namespace st {
namespace trv {

struct Trav {
    const float4* __restrict__ nodes;
    const float4* __restrict__ tri_v;
    int32_t root;
    int32_t max_iter;               // 2 * node count + 8: bound on loop iterations of one traversal
    unsigned long long* visits;     // optional [4]: nodes and triangles visited (closest, any-hit)
};

__device__ __forceinline__ float safe_inv(float d) {
    // a zero direction component becomes a huge finite slope so the slab test never forms 0 * inf
    const float big = 1e30f;
    if (fabsf(d) < 1e-30f) return d >= 0.0f ? big : -big;
    return 1.0f / d;
}

// slab test of one box over [tmin, tmax]: true when hit, entry distance in *tn.  tfar is widened
// by (1 + 2 gamma_3) (Ize, "Robust BVH ray traversal", JCGT 2013); boxes are padded as well.
__device__ __forceinline__ bool slab(float lx, float ly, float lz, float hx, float hy, float hz, f3 o, f3 inv,
                                     float tmin, float tmax, float* tn_out) {
    float t0x = (lx - o.x) * inv.x, t1x = (hx - o.x) * inv.x;
    float t0y = (ly - o.y) * inv.y, t1y = (hy - o.y) * inv.y;
    float t0z = (lz - o.z) * inv.z, t1z = (hz - o.z) * inv.z;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), tmin));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
    tf = tf * 1.0000004f;
    *tn_out = tn;
    return tn <= tf;
}

template <bool AnyHit>
__device__ __forceinline__ int32_t traverse(const Trav& T, f3 o, f3 d, int32_t exclude, float t_min, float t_max,
                                            float* t_out, uint32_t* flags) {
    const WRay wr = wray(o, d);
    const f3 inv{safe_inv(d.x), safe_inv(d.y), safe_inv(d.z)};
    int32_t best = -1;
    float tb = t_max;  // closest: +inf; any-hit: the segment end (exclusive)
    int2 stack[kStack];
    int sp = 0;
    int32_t ref = T.root;
    // every node of a proper tree is visited at most once: more iterations than nodes means a
    // malformed hierarchy, reported through the flags instead of looping
    int guard = T.max_iter;
    int n_nodes = 0, n_tris = 0;
    // the search interval for boxes: [-inf, tb]; t_min is enforced on triangles only
    while (true) {
        if (--guard < 0) {
            atomicOr(flags, kFlagBadTree);
            break;
        }
        if (ref >= 0) {
            // 4-wide node: children's bounds as lo.x, hi.x, lo.y, hi.y, lo.z, hi.z rows, then the refs
            const float4* nd = T.nodes + 8 * (size_t)ref;
            const float4 lx = __ldg(nd + 0), hx = __ldg(nd + 1), ly = __ldg(nd + 2), hy = __ldg(nd + 3);
            const float4 lz = __ldg(nd + 4), hz = __ldg(nd + 5), rf = __ldg(nd + 6);
            ++n_nodes;
            // boxes are padded, so a box holding a hit at t > t_min >= 0 exits at t > 0 after rounding
            float t0, t1, t2, t3;
            const int32_t r0 = __float_as_int(rf.x), r1 = __float_as_int(rf.y), r2 = __float_as_int(rf.z),
                          r3 = __float_as_int(rf.w);
            const bool h0 = slab(lx.x, ly.x, lz.x, hx.x, hy.x, hz.x, o, inv, 0.0f, tb, &t0);
            const bool h1 = slab(lx.y, ly.y, lz.y, hx.y, hy.y, hz.y, o, inv, 0.0f, tb, &t1);
            const bool h2 = r2 != kEmptyRef && slab(lx.z, ly.z, lz.z, hx.z, hy.z, hz.z, o, inv, 0.0f, tb, &t2);
            const bool h3 = r3 != kEmptyRef && slab(lx.w, ly.w, lz.w, hx.w, hy.w, hz.w, o, inv, 0.0f, tb, &t3);
            // order the hit children by entry distance (misses last): the nearest is visited next, the
            // others are pushed farthest first
            // (hit keys are clamped below +inf, so the hits sort strictly before the misses)
            const float inf = __int_as_float(0x7f800000), big = 3.0e38f;
            float k0 = h0 ? fminf(t0, big) : inf, k1 = h1 ? fminf(t1, big) : inf;
            float k2 = h2 ? fminf(t2, big) : inf, k3 = h3 ? fminf(t3, big) : inf;
            int32_t c0 = r0, c1 = r1, c2 = r2, c3 = r3;
            auto cx = [](float& ka, int32_t& ca, float& kb, int32_t& cb) {
                if (kb < ka) {
                    const float tk = ka;
                    ka = kb;
                    kb = tk;
                    const int32_t tc = ca;
                    ca = cb;
                    cb = tc;
                }
            };
            cx(k0, c0, k1, c1);
            cx(k2, c2, k3, c3);
            cx(k0, c0, k2, c2);
            cx(k1, c1, k3, c3);
            cx(k1, c1, k2, c2);
            const int nh = (int)h0 + (int)h1 + (int)h2 + (int)h3;
            if (nh > 0) {
                if (sp + nh - 1 > kStack) {
                    atomicOr(flags, kFlagStackOverflow);
                } else {
                    if (nh > 3) stack[sp++] = make_int2(c3, __float_as_int(k3));
                    if (nh > 2) stack[sp++] = make_int2(c2, __float_as_int(k2));
                    if (nh > 1) stack[sp++] = make_int2(c1, __float_as_int(k1));
                }
                ref = c0;
                continue;
            }
        } else {
            const int32_t code = ~ref;
            const int first = code >> 3, cnt = (code & 7) + 1;
            for (int i = first; i < first + cnt; ++i) {
                const float4 v0 = __ldg(&T.tri_v[3 * i + 0]);
                const int32_t id = __float_as_int(v0.w);
                if (id == exclude) continue;
                const float4 v1 = __ldg(&T.tri_v[3 * i + 1]);
                const float4 v2 = __ldg(&T.tri_v[3 * i + 2]);
                ++n_tris;
                float th;
                if (!wt_hit(wr, f3{v0.x, v0.y, v0.z}, f3{v1.x, v1.y, v1.z}, f3{v2.x, v2.y, v2.z}, &th)) continue;
                if (!(th > t_min)) continue;
                if (AnyHit) {
                    if (th < t_max) {
                        *t_out = th;
                        if (T.visits) {
                            atomicAdd(&T.visits[2], (unsigned long long)n_nodes);
                            atomicAdd(&T.visits[3], (unsigned long long)n_tris);
                        }
                        return id;
                    }
                } else if (th < tb || (th == tb && id < best)) {
                    tb = th;
                    best = id;
                }
            }
        }
        // pop, skipping entries whose box starts beyond the best hit
        bool found = false;
        while (sp > 0) {
            const int2 top = stack[--sp];
            if (__int_as_float(top.y) <= tb) {
                ref = top.x;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
    if (T.visits) {
        atomicAdd(&T.visits[AnyHit ? 2 : 0], (unsigned long long)n_nodes);
        atomicAdd(&T.visits[AnyHit ? 3 : 1], (unsigned long long)n_tris);
    }
    *t_out = tb;
    return best;
}

// Visibility of `target` from o: direction normalize(target - o), t in (t_min, |target - o| - eps).
__device__ __forceinline__ bool visible(const Trav& T, f3 o, f3 target, int32_t exclude, float t_min, float eps,
                                        uint32_t* flags) {
    float L;
    const f3 u = normalize(sub(target, o), &L);
    const float tmax = L - eps;
    if (!(tmax > t_min)) return true;
    float th;
    return traverse<true>(T, o, u, exclude, t_min, tmax, &th, flags) < 0;
}

// adds the number of active lanes to a 64-bit counter with one atomic per warp
__device__ __forceinline__ void warp_count(unsigned long long* ctr) {
    const unsigned m = __activemask();
    if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(ctr, (unsigned long long)__popc(m));
}

__device__ __forceinline__ void philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed,
                                         uint32_t out[4]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

}  // namespace trv
}  // namespace st
