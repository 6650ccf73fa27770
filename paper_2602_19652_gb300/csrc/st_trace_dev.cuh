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
    int32_t stack_limit = kStack;   // stack entries a query may use (1..kStack) before it restarts stackless
    unsigned long long* restarts = nullptr;  // optional: queries that restarted from the root
    int32_t refill = 0;  // lanes of a warp waiting for a query before it refills them (0: the kernel's default)
    // Two-level scenes (instances of shared meshes): `nodes` / `root` are then the top-level BVH over the
    // instances' world boxes, whose leaf codes index `tinst` (instance ids in leaf order); every prototype has
    // a 4-wide BVH over its triangles in object space (`bnodes`, `btri`: triangles in leaf order, the
    // prototype-local index in the first `w`).  `inst` holds 8 float4 per instance: the rows (A_r, b_r) of
    // its map, the rows of A^-1 (w: |A^-1|_inf, the prototype's root reference, the first world triangle),
    // and its world box (lo, hi).  Null for flat scenes.
    const float4* __restrict__ bnodes = nullptr;
    const float4* __restrict__ btri = nullptr;
    const float4* __restrict__ inst = nullptr;
    const int32_t* __restrict__ tinst = nullptr;
    // checked build: sizes of nodes, leaf-order triangles, prototype nodes, prototype triangles, instances,
    // world triangles (see ST_CHECK_OR)
    int64_t chk[6] = {0, 0, 0, 0, 0, 0};
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

// Resumable traversal: the state of one query, advanced by one wide node or one leaf triangle per step, so that
// a kernel can give a finished lane a new query while the other lanes of its warp continue.
struct TravState {
    WRay wr;
    f3 o, inv;
    int32_t exclude;
    float t_min, t_max, tb;  // closest: tb = best t so far (+inf at first); any-hit: segment end (exclusive)
    int32_t best, ref;
    int sp, guard, n_nodes, n_tris;
};

__device__ __forceinline__ void trav_init(TravState& S, const Trav& T, f3 o, f3 d, int32_t exclude, float t_min,
                                          float t_max) {
    S.wr = wray(o, d);
    S.o = o;
    S.inv = f3{safe_inv(d.x), safe_inv(d.y), safe_inv(d.z)};
    S.exclude = exclude;
    S.t_min = t_min;
    S.t_max = t_max;
    S.tb = t_max;
    S.best = -1;
    S.ref = T.root;
    S.sp = 0;
    // every node of a proper tree is visited at most once: more iterations than nodes means a
    // malformed hierarchy, reported through the flags instead of looping
    S.guard = T.max_iter;
    S.n_nodes = 0;
    S.n_tris = 0;
}

// one triangle of a leaf (leaf code: first triangle << 3 | triangles left after it); true when an any-hit
// query has found its hit.  S.ref becomes the code of the next triangle, or `after` when the leaf is done.
template <bool AnyHit>
__device__ __forceinline__ bool leaf_step(const Trav& T, TravState& S, int32_t after) {
    const int32_t code = ~S.ref;
    const int i = code >> 3, rest = code & 7;
    const float4 v0 = __ldg(&T.tri_v[3 * i + 0]);
    const int32_t id = __float_as_int(v0.w);
    if (id != S.exclude) {
        const float4 v1 = __ldg(&T.tri_v[3 * i + 1]);
        const float4 v2 = __ldg(&T.tri_v[3 * i + 2]);
        ++S.n_tris;
        float th;
        if (wt_hit(S.wr, f3{v0.x, v0.y, v0.z}, f3{v1.x, v1.y, v1.z}, f3{v2.x, v2.y, v2.z}, &th) && th > S.t_min) {
            if (AnyHit) {
                if (th < S.t_max) {
                    S.tb = th;
                    S.best = id;
                    return true;
                }
            } else if (th < S.tb || (th == S.tb && id < S.best)) {
                S.tb = th;
                S.best = id;
            }
        }
    }
    S.ref = rest > 0 ? ~(((i + 1) << 3) | (rest - 1)) : after;
    return false;
}

// one node or one leaf triangle; true when the query has finished (S.best = hit triangle or -1, S.tb = its t)
template <bool AnyHit>
__device__ __forceinline__ bool trav_step(const Trav& T, TravState& S, int2* stack, uint32_t* flags) {
    if (--S.guard < 0) {
        atomicOr(flags, kFlagBadTree);
        return true;
    }
    if (S.ref >= 0) {
        ST_CHECK_OR(S.ref < T.chk[0], flags, return true);
        // 4-wide node: children's bounds as lo.x, hi.x, lo.y, hi.y, lo.z, hi.z rows, then the refs
        const float4* nd = T.nodes + 8 * (size_t)S.ref;
        const float4 lx = __ldg(nd + 0), hx = __ldg(nd + 1), ly = __ldg(nd + 2), hy = __ldg(nd + 3);
        const float4 lz = __ldg(nd + 4), hz = __ldg(nd + 5), rf = __ldg(nd + 6);
        ++S.n_nodes;
        // boxes are padded, so a box holding a hit at t > t_min >= 0 exits at t > 0 after rounding
        const f3 o = S.o, inv = S.inv;
        const float tb = S.tb;
        float t0, t1, t2, t3;
        const int32_t r0 = __float_as_int(rf.x), r1 = __float_as_int(rf.y), r2 = __float_as_int(rf.z),
                      r3 = __float_as_int(rf.w);
        const bool h0 = slab(lx.x, ly.x, lz.x, hx.x, hy.x, hz.x, o, inv, 0.0f, tb, &t0);
        const bool h1 = slab(lx.y, ly.y, lz.y, hx.y, hy.y, hz.y, o, inv, 0.0f, tb, &t1);
        const bool h2 = r2 != kEmptyRef && slab(lx.z, ly.z, lz.z, hx.z, hy.z, hz.z, o, inv, 0.0f, tb, &t2);
        const bool h3 = r3 != kEmptyRef && slab(lx.w, ly.w, lz.w, hx.w, hy.w, hz.w, o, inv, 0.0f, tb, &t3);
        if (S.sp < 0) {
            // Restart walk of a query whose short stack overflowed: depth first from the root in fixed child
            // order, without a stack.  stack[0] = (this node, first slot still to visit); a node's row 7 holds
            // its parent and its slot there.  A child is entered when its box meets [0, tb] with the best hit so
            // far, so the result is the stack walk's: a subtree skipped for a farther tb holds no triangle
            // nearer than the final tb.
            const int from = stack[0].y;
            const int c = (from <= 0 && h0) ? 0 : (from <= 1 && h1) ? 1 : (from <= 2 && h2) ? 2 : (from <= 3 && h3) ? 3 : -1;
            if (c >= 0) {
                const int32_t ref = c == 0 ? r0 : c == 1 ? r1 : c == 2 ? r2 : r3;
                // into the child node, or through the leaf's triangles and back to the next slot here
                stack[0] = ref >= 0 ? make_int2(ref, 0) : make_int2(S.ref, c + 1);
                S.ref = ref;
                return false;
            }
            if (S.ref == T.root) return true;  // every child of the root done
            const float4 up = __ldg(nd + 7);
            S.ref = __float_as_int(up.x);
            stack[0] = make_int2(S.ref, __float_as_int(up.y) + 1);  // the parent, after this node's slot
            return false;
        }
        // order the hit children by entry distance (misses last): the nearest is visited next, the
        // others are pushed farthest first (hit keys are clamped below +inf, so the hits sort strictly
        // before the misses)
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
            if (S.sp + nh - 1 > T.stack_limit) {
                // the short stack is full: restart from the root with the stackless walk, keeping the best hit
                if (T.restarts) atomicAdd(T.restarts, 1ull);
                S.sp = -1;
                stack[0] = make_int2(T.root, 0);
                S.ref = T.root;
                S.guard = T.max_iter > (1 << 27) ? (1 << 30) : 8 * T.max_iter;  // each node down once, up <= 4 times
                return false;
            } else {
                if (nh > 3) stack[S.sp++] = make_int2(c3, __float_as_int(k3));
                if (nh > 2) stack[S.sp++] = make_int2(c2, __float_as_int(k2));
                if (nh > 1) stack[S.sp++] = make_int2(c1, __float_as_int(k1));
            }
            S.ref = c0;
            return false;
        }
    } else {
        // one triangle of a leaf per step, so lanes in leaves and lanes in inner nodes of the same warp stay
        // in step
        ST_CHECK_OR((int64_t)((~S.ref) >> 3) + ((~S.ref) & 7) < T.chk[1], flags, return true);
        if (leaf_step<AnyHit>(T, S, 1)) return true;
        if (S.ref < 0) return false;
        if (S.sp < 0) {  // restart walk: back to the node that holds the leaf
            S.ref = stack[0].x;
            return false;
        }
    }
    // pop, skipping entries whose box starts beyond the best hit
    while (S.sp > 0) {
        const int2 top = stack[--S.sp];
        if (__int_as_float(top.y) <= S.tb) {
            S.ref = top.x;
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------- two-level scenes
// A query walks the top-level BVH in world space; at an instance whose world box it enters it moves into
// the instance's object space (o' = A^-1 (o - b), d' = A^-1 d: the same ray parameter t in both spaces) and
// walks the prototype's BVH, whose boxes are grown by a bound on the rounding of o' and d' up to the
// instance box's exit distance, so that a box is never rejected where the world-space test would hit.
// Triangles are tested in world space with the world ray: their vertices are mapped by `affine_row`, as
// in the flat expansion, so hits, t and triangle ids (first world triangle of the instance + local index)
// are those of the same scene loaded flat, whatever the two hierarchies look like.
struct TravStateTL : TravState {
    f3 wo, wd, winv;  // the world ray (o and inv hold the object-space ray inside an instance)
    float pad;        // growth of the current instance's object-space boxes (0 at the top level)
    int32_t inst;     // current instance (-1: top level)
    int32_t isp;      // stack depth when the instance was entered (stack walk)
    int32_t broot;    // the current prototype's root reference
    int32_t tbase;    // the current instance's first world triangle
};

__device__ __forceinline__ void trav_init(TravStateTL& S, const Trav& T, f3 o, f3 d, int32_t exclude, float t_min,
                                          float t_max) {
    trav_init(static_cast<TravState&>(S), T, o, d, exclude, t_min, t_max);
    S.wo = o;
    S.wd = d;
    S.winv = S.inv;
    S.pad = 0.0f;
    S.inst = -1;
    S.isp = 0;
    S.broot = 0;
    S.tbase = 0;
}

// slab test of a box grown by g on every side; entry and exit distances
__device__ __forceinline__ bool slab_g(float lx, float ly, float lz, float hx, float hy, float hz, f3 o, f3 inv,
                                       float g, float tmax, float* tn_out, float* tf_out) {
    const float t0x = ((lx - g) - o.x) * inv.x, t1x = ((hx + g) - o.x) * inv.x;
    const float t0y = ((ly - g) - o.y) * inv.y, t1y = ((hy + g) - o.y) * inv.y;
    const float t0z = ((lz - g) - o.z) * inv.z, t1z = ((hz + g) - o.z) * inv.z;
    const float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
    tf = tf * 1.0000004f;
    *tn_out = tn;
    *tf_out = tf;
    return tn <= tf;
}

// into instance i, whose world box the ray leaves at tf
__device__ __forceinline__ void tl_enter(const Trav& T, TravStateTL& S, int32_t i, float tf) {
    const float4* r = T.inst + 8 * (size_t)i;
    const float4 f0 = __ldg(r), f1 = __ldg(r + 1), f2 = __ldg(r + 2);
    const float4 g0 = __ldg(r + 3), g1 = __ldg(r + 4), g2 = __ldg(r + 5);
    const float ux = S.wo.x - f0.w, uy = S.wo.y - f1.w, uz = S.wo.z - f2.w;
    const f3 d = S.wd;
    S.o = f3{(g0.x * ux + g0.y * uy) + g0.z * uz, (g1.x * ux + g1.y * uy) + g1.z * uz,
             (g2.x * ux + g2.y * uy) + g2.z * uz};
    const f3 dd{(g0.x * d.x + g0.y * d.y) + g0.z * d.z, (g1.x * d.x + g1.y * d.y) + g1.z * d.z,
                (g2.x * d.x + g2.y * d.y) + g2.z * d.z};
    S.inv = f3{safe_inv(dd.x), safe_inv(dd.y), safe_inv(dd.z)};
    // |rounding of o' + t d'| <= 4 u |A^-1|_inf (|o - b|_inf + t |d|_inf) for u = 2^-24 and t <= tf; 2^-20
    // leaves a factor 4, and also covers the rounding of the slab differences when |o'| exceeds the
    // prototype's own padding
    const float um = fmaxf(fmaxf(fabsf(ux), fabsf(uy)), fabsf(uz));
    S.pad = 9.5367431640625e-07f * g0.w * (um + fmaxf(tf, 0.0f));
    S.inst = i;
    S.broot = __float_as_int(g1.w);
    S.tbase = __float_as_int(g2.w);
}

__device__ __forceinline__ void tl_exit(TravStateTL& S) {
    S.o = S.wo;
    S.inv = S.winv;
    S.pad = 0.0f;
    S.inst = -1;
}

// stackless walk: stack[0] = resume point of the current level, and inside an instance stack[1].x = the
// top-level leaf's next instance (a leaf code) or 1 when it has none, stack[2] = the top-level resume point
__device__ __forceinline__ void tl_exit_stackless(TravStateTL& S, int2* stack) {
    tl_exit(S);
    stack[0] = stack[2];
    const int32_t cont = stack[1].x;
    S.ref = cont < 0 ? cont : stack[0].x;
}

__device__ __forceinline__ void tl_restart(const Trav& T, TravStateTL& S, int2* stack) {
    if (T.restarts) atomicAdd(T.restarts, 1ull);
    if (S.inst >= 0) tl_exit(S);
    S.sp = -1;
    stack[0] = make_int2(T.root, 0);
    S.ref = T.root;  // a node: two-level scenes always have a top-level root node
    S.guard = T.max_iter > (1 << 27) ? (1 << 30) : 8 * T.max_iter;
}

// one triangle of a prototype leaf, tested in world space
template <bool AnyHit>
__device__ __forceinline__ bool leaf_step_tl(const Trav& T, TravStateTL& S, int32_t after) {
    const int32_t code = ~S.ref;
    const int i = code >> 3, rest = code & 7;
    const float4 v0 = __ldg(&T.btri[3 * i + 0]);
    const int32_t id = S.tbase + __float_as_int(v0.w);
    if (id != S.exclude) {
        const float4 v1 = __ldg(&T.btri[3 * i + 1]);
        const float4 v2 = __ldg(&T.btri[3 * i + 2]);
        const float4* r = T.inst + 8 * (size_t)S.inst;
        const float4 f0 = __ldg(r), f1 = __ldg(r + 1), f2 = __ldg(r + 2);
        ++S.n_tris;
        const f3 w0{affine_row(f0, v0.x, v0.y, v0.z), affine_row(f1, v0.x, v0.y, v0.z), affine_row(f2, v0.x, v0.y, v0.z)};
        const f3 w1{affine_row(f0, v1.x, v1.y, v1.z), affine_row(f1, v1.x, v1.y, v1.z), affine_row(f2, v1.x, v1.y, v1.z)};
        const f3 w2{affine_row(f0, v2.x, v2.y, v2.z), affine_row(f1, v2.x, v2.y, v2.z), affine_row(f2, v2.x, v2.y, v2.z)};
        float th;
        if (wt_hit(S.wr, w0, w1, w2, &th) && th > S.t_min) {
            if (AnyHit) {
                if (th < S.t_max) {
                    S.tb = th;
                    S.best = id;
                    return true;
                }
            } else if (th < S.tb || (th == S.tb && id < S.best)) {
                S.tb = th;
                S.best = id;
            }
        }
    }
    S.ref = rest > 0 ? ~(((i + 1) << 3) | (rest - 1)) : after;
    return false;
}

// one node (either level), one instance of a top-level leaf or one prototype triangle; true when finished
template <bool AnyHit>
__device__ __forceinline__ bool trav_step(const Trav& T, TravStateTL& S, int2* stack, uint32_t* flags) {
    if (--S.guard < 0) {
        atomicOr(flags, kFlagBadTree);
        return true;
    }
    const bool in = S.inst >= 0;
    if (S.ref >= 0) {
        ST_CHECK_OR(S.ref < (in ? T.chk[2] : T.chk[0]), flags, return true);
        const float4* nd = (in ? T.bnodes : T.nodes) + 8 * (size_t)S.ref;
        const float4 lx = __ldg(nd + 0), hx = __ldg(nd + 1), ly = __ldg(nd + 2), hy = __ldg(nd + 3);
        const float4 lz = __ldg(nd + 4), hz = __ldg(nd + 5), rf = __ldg(nd + 6);
        ++S.n_nodes;
        const f3 o = S.o, inv = S.inv;
        const float tb = S.tb, g = S.pad;
        float t0, t1, t2, t3, e;
        const int32_t r0 = __float_as_int(rf.x), r1 = __float_as_int(rf.y), r2 = __float_as_int(rf.z),
                      r3 = __float_as_int(rf.w);
        const bool h0 = slab_g(lx.x, ly.x, lz.x, hx.x, hy.x, hz.x, o, inv, g, tb, &t0, &e);
        const bool h1 = slab_g(lx.y, ly.y, lz.y, hx.y, hy.y, hz.y, o, inv, g, tb, &t1, &e);
        const bool h2 = r2 != kEmptyRef && slab_g(lx.z, ly.z, lz.z, hx.z, hy.z, hz.z, o, inv, g, tb, &t2, &e);
        const bool h3 = r3 != kEmptyRef && slab_g(lx.w, ly.w, lz.w, hx.w, hy.w, hz.w, o, inv, g, tb, &t3, &e);
        if (S.sp < 0) {  // restart walk (see the flat step), one level at a time
            const int from = stack[0].y;
            const int c = (from <= 0 && h0) ? 0 : (from <= 1 && h1) ? 1 : (from <= 2 && h2) ? 2 : (from <= 3 && h3) ? 3 : -1;
            if (c >= 0) {
                const int32_t ref = c == 0 ? r0 : c == 1 ? r1 : c == 2 ? r2 : r3;
                stack[0] = ref >= 0 ? make_int2(ref, 0) : make_int2(S.ref, c + 1);
                S.ref = ref;
                return false;
            }
            if (in && S.ref == S.broot) {  // the prototype's BVH is done: back to the top level
                tl_exit_stackless(S, stack);
                return false;
            }
            if (!in && S.ref == T.root) return true;
            const float4 up = __ldg(nd + 7);
            S.ref = __float_as_int(up.x);
            stack[0] = make_int2(S.ref, __float_as_int(up.y) + 1);
            return false;
        }
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
            if (S.sp + nh - 1 > T.stack_limit) {
                tl_restart(T, S, stack);
                return false;
            }
            if (nh > 3) stack[S.sp++] = make_int2(c3, __float_as_int(k3));
            if (nh > 2) stack[S.sp++] = make_int2(c2, __float_as_int(k2));
            if (nh > 1) stack[S.sp++] = make_int2(c1, __float_as_int(k1));
            S.ref = c0;
            return false;
        }
    } else if (in) {
        ST_CHECK_OR((int64_t)((~S.ref) >> 3) + ((~S.ref) & 7) < T.chk[3], flags, return true);
        if (leaf_step_tl<AnyHit>(T, S, 1)) return true;
        if (S.ref < 0) return false;
        if (S.sp < 0) {
            if (S.broot < 0) tl_exit_stackless(S, stack);  // the prototype's BVH is this one leaf
            else S.ref = stack[0].x;
            return false;
        }
    } else {
        // one instance of a top-level leaf: into its object space when the ray enters its world box
        const int32_t code = ~S.ref;
        const int k = code >> 3, rest = code & 7;
        const int32_t cont = rest > 0 ? ~(((k + 1) << 3) | (rest - 1)) : 1;
        ST_CHECK_OR((int64_t)k + rest < T.chk[4], flags, return true);
        const int32_t i = __ldg(T.tinst + k);
        ST_CHECK_OR(i >= 0 && i < T.chk[4], flags, return true);
        const float4* r = T.inst + 8 * (size_t)i;
        const float4 blo = __ldg(r + 6), bhi = __ldg(r + 7);
        ++S.n_nodes;
        float tn, tf;
        // (w of the box's hi is 1 for an instance of a prototype without triangles: never entered)
        if (bhi.w == 0.0f && slab_g(blo.x, blo.y, blo.z, bhi.x, bhi.y, bhi.z, S.o, S.inv, 0.0f, S.tb, &tn, &tf)) {
            if (S.sp < 0) {
                stack[1] = make_int2(cont, 0);
                stack[2] = stack[0];
                tl_enter(T, S, i, tf);
                if (S.broot >= 0) stack[0] = make_int2(S.broot, 0);
                S.ref = S.broot;
                return false;
            }
            if (cont < 0) {  // the leaf's next instance, resumed when this one is done (key 0: never skipped)
                if (S.sp + 1 > T.stack_limit) {
                    tl_restart(T, S, stack);
                    return false;
                }
                stack[S.sp++] = make_int2(cont, 0);
            }
            S.isp = S.sp;
            tl_enter(T, S, i, tf);
            S.ref = S.broot;
            return false;
        }
        S.ref = cont;
        if (S.ref < 0) return false;
        if (S.sp < 0) {
            S.ref = stack[0].x;
            return false;
        }
    }
    // pop; an instance is left when its entries are used up
    while (true) {
        if (S.inst >= 0 && S.sp == S.isp) tl_exit(S);
        if (S.sp <= 0) return true;
        const int2 top = stack[--S.sp];
        if (__int_as_float(top.y) <= S.tb) {
            S.ref = top.x;
            return false;
        }
    }
}

template <bool TL>
struct TravStateOf {
    using type = TravState;
};
template <>
struct TravStateOf<true> {
    using type = TravStateTL;
};

template <bool AnyHit>
__device__ __forceinline__ void trav_count(const Trav& T, const TravState& S) {
    if (T.visits) {
        atomicAdd(&T.visits[AnyHit ? 2 : 0], (unsigned long long)S.n_nodes);
        atomicAdd(&T.visits[AnyHit ? 3 : 1], (unsigned long long)S.n_tris);
    }
}

template <bool AnyHit, bool TL = false>
__device__ __forceinline__ int32_t traverse(const Trav& T, f3 o, f3 d, int32_t exclude, float t_min, float t_max,
                                            float* t_out, uint32_t* flags) {
    typename TravStateOf<TL>::type S;
    int2 stack[kStack];
    trav_init(S, T, o, d, exclude, t_min, t_max);
    while (!trav_step<AnyHit>(T, S, stack, flags)) {
    }
    trav_count<AnyHit>(T, S);
    *t_out = S.tb;
    return S.best;
}

// Lane refill (persistent traversal kernels): the lanes that need a query claim consecutive indices
// from *ctr (one atomic per warp and round); -1 for lanes that did not ask.  All 32 lanes call it.
__device__ __forceinline__ int64_t claim(unsigned long long* ctr, bool need) {
    const unsigned full = 0xffffffffu;
    const unsigned m = __ballot_sync(full, need);
    if (m == 0u) return -1;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long b = 0;
    if (lane == leader) b = atomicAdd(ctr, (unsigned long long)__popc(m));
    b = __shfl_sync(full, b, leader);
    return need ? (int64_t)(b + (unsigned long long)__popc(m & ((1u << lane) - 1u))) : -1;
}

constexpr int kTravBlock = 128;
// a warp stops stepping to refill once this many of its lanes wait for a query (closest-hit and
// any-hit kernels)
constexpr int kRefillClosest = 16;
constexpr int kRefillAny = 28;

// Visibility of `target` from o: direction normalize(target - o), t in (t_min, |target - o| - eps).
template <bool TL = false>
__device__ __forceinline__ bool visible(const Trav& T, f3 o, f3 target, int32_t exclude, float t_min, float eps,
                                        uint32_t* flags) {
    float L;
    const f3 u = normalize(sub(target, o), &L);
    const float tmax = L - eps;
    if (!(tmax > t_min)) return true;
    float th;
    return traverse<true, TL>(T, o, u, exclude, t_min, tmax, &th, flags) < 0;
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
