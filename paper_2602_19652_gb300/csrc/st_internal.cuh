// Internal declarations shared by the translation units of libsonotrace (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sonotrace.h"

namespace st {

// ------------------------------------------------------------------ constants
constexpr int kLeafMax = 4;        // triangles per BVH leaf after collapsing small subtrees
constexpr int kStack = 128;        // traversal stack entries per thread
constexpr int32_t kEmptyRef = INT32_MIN;  // unused child slot of a 4-wide BVH node (no valid leaf has this code)
constexpr int kMaxBounces = 8;     // B limit (material chain packed in 8 bytes)
constexpr int kMaxMics = 4096;

// error flag bits written by kernels into Ctx::d_flags
constexpr uint32_t kFlagStackOverflow = 1u;  // (unused: a traversal that would overflow its stack restarts)
constexpr uint32_t kFlagBadIndex = 2u;
constexpr uint32_t kFlagBadVertex = 4u;
constexpr uint32_t kFlagBadTree = 8u;
constexpr uint32_t kFlagCheck = 16u;  // a bounds check of the checked build failed (the access was skipped)

// Bounds-checked build (-DST_CHECKS, `build(checks=True)`): indices read from device data (tree references,
// leaf and triangle ids, materials) are checked before they index an array; a failed check sets kFlagCheck
// in the launch's flags word, skips the access and takes `action`, and the call returns ST_ERR_CUDA.  In
// the normal build the checks compile to nothing.
#ifdef ST_CHECKS
#define ST_CHECK_OR(cond, flags, action)                   \
    do {                                                   \
        if (!(cond)) {                                     \
            if (flags) atomicOr((flags), kFlagCheck);      \
            action;                                        \
        }                                                  \
    } while (0)
#else
#define ST_CHECK_OR(cond, flags, action) \
    do {                                 \
    } while (0)
#endif

// ------------------------------------------------------------------ device buffers
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};
cudaError_t grow(DevBuf& b, size_t bytes);
void release(DevBuf& b);
template <class T>
T* ptr(const DevBuf& b) {
    return static_cast<T*>(b.p);
}

// ------------------------------------------------------------------ scene on the device
struct InstanceDev;

struct SceneDev {
    int64_t n_verts = 0, n_tris = 0;
    DevBuf verts;      // [V][3] f32
    DevBuf tris;       // [T][3] i32
    DevBuf tri_mat;    // [T] i32
    DevBuf tri_obj;    // [T] i32
    DevBuf nrm;        // [T][3] f32 geometric normals (input triangle order)
    // LBVH
    DevBuf nodes;      // 4-wide BVH: [n4][8] float4: lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of the 4 children, refs, pad
    DevBuf tri_v;      // [T][3] float4 in leaf order; tri_v[3i].w = triangle index bits
    int32_t root = 0;  // child-ref encoding of the root
    int64_t n_nodes = 0;  // 4-wide nodes
    // LBVH topology kept for refits: binary children, leaf ranges, parents, leaf order, wide-node flags
    // and numbering
    DevBuf bvh_child, bvh_range, bvh_par_i, bvh_par_l, bvh_perm, bvh_wflag, bvh_widx;
    bool bvh_ready = false;
    float bounds_lo[3] = {0, 0, 0}, bounds_hi[3] = {0, 0, 0};
    // curvature and diffraction CDFs
    DevBuf G;          // [V] f32
    DevBuf C;          // [T] f32
    int32_t n_obj = 0;
    DevBuf mesh_tris;  // [T] i32, triangles grouped by mesh, ascending within a mesh
    DevBuf mesh_off;   // [n_obj+1] i64
    DevBuf cdf;        // [T] u64 per-mesh inclusive prefix, in mesh_tris order
    DevBuf n_samples;  // [n_obj] i64
    DevBuf sample_off; // [n_obj+1] i64
    int64_t total_samples = 0;
    // materials (host copies; device band tables are built per frequency grid)
    int32_t n_mat = 0, n_bands = 0;
    std::vector<float> band_hz, k_band, beta_band, diff_band;
    bool built = false;
    // Two-level structure of an instanced scene (on request): nodes / root / n_nodes then hold the top-level
    // BVH over the instances' world boxes and no world-triangle hierarchy is kept.  Each prototype has a
    // 4-wide BVH over its own triangles in object space, built once (blas_*); inst_rec holds 8 float4 per
    // instance (map rows, inverse rows with |A^-1|_inf, prototype root and first world triangle, world box)
    // and tlas_inst the instance ids in top-level leaf order.
    const InstanceDev* inst = nullptr;  // the instance tables of an instanced scene
    bool two_level = false;
    bool tl_ready = false;    // the two-level structure matches the current transforms
    bool blas_ready = false;  // the prototypes' BVHs are built
    DevBuf blas_nodes, blas_tri, blas_root, proto_box, inst_rec, tlas_inst;
    int64_t blas_n_nodes = 0;
};

struct st_scene_impl;

// ------------------------------------------------------------------ helpers for launches
// Every kernel launch of the library calls note_launch() first; the count is reported in st_stats.
void note_launch();
int64_t launch_count();

inline unsigned grid_for(int64_t n, int block, int64_t cap = 152 * 32) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ------------------------------------------------------------------ primitives (st_sort.cu)
// Stable LSD radix sort of (u64 key, u32 value) pairs over the low `bits` bits of the key.
// Scratch must hold sort_scratch_bytes(n) bytes.
size_t sort_scratch_bytes(int64_t n);
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, void* scratch, cudaStream_t s);
// Exclusive scan of n u32 flags/counts into out (u32), total written to *total (device, may be null).
size_t scan_scratch_bytes(int64_t n);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* scratch,
                               cudaStream_t s);
cudaError_t inclusive_scan_u64(const uint64_t* in, uint64_t* out, int64_t n, void* scratch, cudaStream_t s);

// ------------------------------------------------------------------ scene build (st_scene.cu)
struct CurvParamsDev {
    float eta, area_ref, hc_frac;
    double dither;
    int32_t samples_per_vertex;
    int64_t budget;
    uint64_t seed;
};
// Validates indices and vertices (flags), computes normals, welds, curvature, C, CDFs, sample
// counts and the LBVH.  Synchronises once.  Returns a CUDA error or sets *mesh_error.
// refit: keep the LBVH topology of an earlier build (new vertex positions, same triangles): boxes,
// wide nodes and leaf triangles are recomputed; keep_curvature: also keep curvature, metric, CDFs and
// sample counts (valid for rigid motions of whole meshes)
cudaError_t scene_build(SceneDev& S, const CurvParamsDev& cp, cudaStream_t s, bool* mesh_error, std::string* msg,
                        bool refit = false, bool keep_curvature = false);

// Instanced scene: the prototypes (concatenated) and the instance table, kept on the device so that new
// transforms expand the world vertices again.  Instance i is a copy of prototype iproto[i]; it owns world
// vertices vbase[i] .. vbase[i+1] and triangles tbase[i] .. tbase[i+1].
struct InstanceDev {
    int32_t n_proto = 0, n_inst = 0;
    int64_t nv = 0, nt = 0;  // world vertices and triangles
    DevBuf pverts;           // [pv][3] f32 prototype vertices
    DevBuf ptris;            // [pt][3] i32 prototype-local vertex indices
    DevBuf pmat;             // [pt] i32 materials
    DevBuf pvoff, ptoff;     // [n_proto + 1] i64 prototype vertex / triangle offsets
    DevBuf iproto;           // [n_inst] i32
    DevBuf vbase, tbase;     // [n_inst + 1] i64
    DevBuf xform;            // [n_inst][12] f32 row-major [A | b]
    std::vector<int64_t> pvoff_h, ptoff_h;  // host copies of the prototype offsets
};
// world vertices [nv][3] from the transforms xf [n_inst][12] (device)
cudaError_t expand_instance_verts(const InstanceDev& I, const float* xf, float* out, cudaStream_t s);
// world triangles [nt][3], their materials and objects (object = instance id)
cudaError_t expand_instance_tris(const InstanceDev& I, int32_t* tris, int32_t* mat, int32_t* obj, cudaStream_t s);

// ------------------------------------------------------------------ tracing (st_trace.cu)
struct TraceArgs {
    // scene
    const float4* nodes;
    const float4* tri_v;
    int32_t root;
    int32_t max_iter;
    unsigned long long* visits;
    int32_t stack_limit;  // traversal stack entries per query (1..kStack; a query that needs more restarts stackless)
    unsigned long long* restarts;  // device counter of stackless restarts (or null)
    int32_t refill;  // lane-refill threshold of the persistent traversal kernels (0 = default)
    // two-level scenes (null for flat ones): prototypes' object-space BVH nodes and leaf-order triangles,
    // instance records, instance ids of the top-level leaves (nodes / root are then the top level)
    const float4* bnodes = nullptr;
    const float4* btri = nullptr;
    const float4* inst = nullptr;
    const int32_t* tinst = nullptr;
    // array sizes the checked build compares indices with: wide nodes, leaf-order triangles, prototype nodes,
    // prototype triangles, instances, world triangles
    int64_t chk[6] = {0, 0, 0, 0, 0, 0};
    const float* nrm;
    // rays
    float s[3];
    float q[4];
    const float* R;       // device [3]: receiver reference point for the per-hit visibility ray
    const float* dirs;    // [N][3] local directions
    const uint32_t* perm; // [N] processing order of the first bounce (rays sorted by direction) or null
    int64_t N;
    int32_t B;
    double r_max;
    float t_min, los_eps;
    // state (SoA, indexed by ray id)
    float* ox; float* oy; float* oz;
    float* dx; float* dy; float* dz;
    double* racc;
    int32_t* prev;
    // queues
    uint32_t* q_in; uint32_t* q_out;
    uint32_t* n_in; uint32_t* n_out;
    // closest hits of the current bounce [N], the visibility queue (record ids) and the lane-refill
    // counters (three per bounce)
    int32_t* hit_tri; float* hit_t;
    uint32_t* vis_q; uint32_t* vis_n;
    unsigned long long* ctr;
    // optional: visibility queue sorted by the Morton code of the hit points (scene bounds lo, 1024 / extent)
    // before it is traced, so that neighbouring lanes share nodes; keys [N] and sort scratch, or null
    uint64_t* sort_keys; void* sort_scr;
    float blo[3], bscale[3];
    // per-microphone receiver test (ST_LOS_PER_MIC): M queries per record (query = record id * M + m), the
    // record's bit m of rec_mask set when microphone m is visible; null rec_mask: one query per record
    uint64_t* rec_mask; const float* mics; int32_t M;
    // records [N][B]
    int32_t* rec_tri;
    float* rec_p;    // [N][B][3]
    float* rec_d;    // [N][B][3]
    double* rec_r;
    uint8_t* rec_los;
    uint32_t* flags;
    unsigned long long* queries;  // [0] closest-hit segments, [1] any-hit segments
};
cudaError_t trace_rays(TraceArgs& a, cudaStream_t s, int block);
// perm = indices 0..n-1 sorted by an octahedral Morton key of dirs (keys: n u64 scratch)
cudaError_t direction_order(const float* dirs, int64_t n, uint64_t* keys, uint32_t* perm, void* scratch,
                            cudaStream_t s);

struct DiffArgs {
    const float4* nodes;
    const float4* tri_v;
    int32_t root;
    int32_t max_iter;
    unsigned long long* visits;
    int32_t stack_limit;  // traversal stack entries per query (1..kStack; a query that needs more restarts stackless)
    unsigned long long* restarts;  // device counter of stackless restarts (or null)
    int32_t refill;  // lane-refill threshold of the persistent traversal kernels (0 = default)
    // two-level scenes (null for flat ones): prototypes' object-space BVH nodes and leaf-order triangles,
    // instance records, instance ids of the top-level leaves (nodes / root are then the top level)
    const float4* bnodes = nullptr;
    const float4* btri = nullptr;
    const float4* inst = nullptr;
    const int32_t* tinst = nullptr;
    // array sizes the checked build compares indices with: wide nodes, leaf-order triangles, prototype nodes,
    // prototype triangles, instances, world triangles
    int64_t chk[6] = {0, 0, 0, 0, 0, 0};
    const float* nrm;
    const float* verts;
    const int32_t* tris;
    int32_t n_obj;
    const int32_t* mesh_tris;
    const int64_t* mesh_off;
    const uint64_t* cdf;
    const int64_t* sample_off;
    int64_t K;
    uint64_t seed;
    uint32_t pose;
    float s[3];
    float fwd[3];
    float cos_fov;        // <= -1: off
    float cos_inc;
    float t_min, los_eps;
    int32_t* cand_tri;
    float* cand_p;        // [K][3]
    uint8_t* keep;
    uint32_t* los_q; uint32_t* los_n;  // candidates that passed the filters: their line-of-sight queries
    unsigned long long* ctr;           // lane-refill counter of the line-of-sight kernel
    uint32_t* flags;
    unsigned long long* queries;
    // optional: line-of-sight queue sorted by the Morton code of the candidate points (keys [K], scratch)
    uint64_t* sort_keys; void* sort_scr;
    float blo[3], bscale[3];
};
cudaError_t diffraction_sample(DiffArgs& a, cudaStream_t s);

struct DirectArgs {
    const float4* nodes;
    const float4* tri_v;
    int32_t root;
    int32_t max_iter;
    unsigned long long* visits;
    int32_t stack_limit;  // traversal stack entries per query (1..kStack; a query that needs more restarts stackless)
    unsigned long long* restarts;  // device counter of stackless restarts (or null)
    int32_t refill;  // lane-refill threshold of the persistent traversal kernels (0 = default)
    // two-level scenes (null for flat ones): prototypes' object-space BVH nodes and leaf-order triangles,
    // instance records, instance ids of the top-level leaves (nodes / root are then the top level)
    const float4* bnodes = nullptr;
    const float4* btri = nullptr;
    const float4* inst = nullptr;
    const int32_t* tinst = nullptr;
    // array sizes the checked build compares indices with: wide nodes, leaf-order triangles, prototype nodes,
    // prototype triangles, instances, world triangles
    int64_t chk[6] = {0, 0, 0, 0, 0, 0};
    float s[3];
    const float* mics;
    int32_t M;
    float t_min, los_eps;
    uint8_t* vis;
    uint32_t* flags;
    unsigned long long* queries;
};
cudaError_t direct_visibility(DirectArgs& a, cudaStream_t s);

void mic_centroid_host_order(const float* mics_dev, int32_t M, float* R_dev, cudaStream_t s);

// ------------------------------------------------------------------ accumulation (st_accum.cu)
// Unified contributor list ("paths") feeding the accumulator.
struct PathList {
    int64_t n_max = 0;
    DevBuf px, py, pz, dx, dy, dz, rhi, rlo, chain_lo, chain_hi, meta, dep;
    DevBuf mask;  // u64 per path, per-microphone receiver test only (grown separately)
    // meta: bits 0..3 = chain length (specular) or 0 (diffraction), bits 8..15 = material of the
    // last leg's surface
};

struct AccumTables {
    int32_t F = 0, n_mat = 0, n_bands = 0;
    DevBuf band, kband, bband;  // device copies of the band centres, reflection and lobe-width band values (adjoint)
    DevBuf lk;     // [n_mat][F] log2 k(mat, f)
    DevBuf g2;     // [n_mat][F] lobe exponent 1/(2 beta^2) * log2(e)
    DevBuf lid;    // [n_mat][F] log2 I_d(mat, f)
    DevBuf qhi, qlo;  // [F] f_k / c as float-float
    DevBuf bw;        // [F] float2 (lower band index, upper band weight)
    double f_lo = 0, df = 0, c = 343, a0 = 0, a1 = 0;
};

struct AccumArgs {
    int kind;               // 0 specular, 1 diffraction
    int64_t n_paths;        // upper bound; actual count in *d_count
    const uint32_t* d_count;
    const uint32_t* d_base; // optional: first path of this launch in the path arrays (device), null = 0
    const uint64_t* mask;   // optional (per-microphone receiver test): bit m of mask[path] = microphone m
                            // receives the path; null = every microphone
    int32_t tile_tp, tile_kb;  // optional tile override: mic pairs per CTA, shared-memory KB (0 = default)
    int32_t tile_kt;           // optional: bins per thread of the general accumulator, 8 or 16 (0 = default)
    const float* px; const float* py; const float* pz;
    const float* dx; const float* dy; const float* dz;
    const float* rhi; const float* rlo;
    const uint32_t* chain_lo; const uint32_t* chain_hi;
    const uint32_t* meta;
    const float* dep;       // per path: emitter directivity coordinate theta / dtheta (or -1 = omni)
    const float* mics;      // [M][3]
    int32_t M, F;
    const float* lk; const float* g2; const float* lid;
    int32_t n_mat_tab;      // materials in the per-bin tables
    int32_t n_bands_tab;    // bands of the material (and receiver directivity) tables
    const float* qhi; const float* qlo;
    float dq_hi, dq_lo;     // (f_{k+1} - f_k) / c as float-float
    float atm2_0, atm2_step;  // log2 amplitude decay per metre at bin 0 and per bin step
    const float* etab;      // emitter table [n_theta][F] or null
    int32_t n_theta;
    const float* mic_tab;   // receiver tables [M][n_el][n_az][n_bands] or null (omni)
    const float* mic_q;     // receiver orientations [M][4] or null (identity)
    int32_t n_el, n_az;
    const float2* bw;       // [F] band interpolation per bin: (index of the lower band, weight of the upper)
    int32_t reflection_mode;
    float2* partial;        // [n_chunks][M][F]
    int32_t n_chunks;
    const float* jac;       // adjoint only: per specular path dP/ds (3x3 row-major) and dr/ds, or null
};
cudaError_t build_accum_tables(AccumTables& T, const SceneDev& S, int32_t F, double f_lo, double f_hi, double c,
                               double a0, double a1, cudaStream_t s);
cudaError_t accumulate(const AccumArgs& a, cudaStream_t s);
cudaError_t reduce_partials(const float2* partial, int32_t n_chunks, int64_t MF, float2* out, cudaStream_t s);
int32_t accum_chunks(int64_t n_paths_hint, int32_t M, int32_t F, int32_t n_mat, int32_t dir_nb, int32_t tile_tp = 0,
                     int32_t tile_kb = 0, int32_t tile_kt = 0);
// emitter ray sets (st_rays.cu): kind 0 spherical Fibonacci, 1 zonal equal-area centres
cudaError_t ray_directions(int kind, int64_t n, float* out, DevBuf& scratch, cudaStream_t s);
// impulse responses / received signals from accumulated spectra (st_signal.cu)
cudaError_t signal_response(const float2* S, int n_comp, int M, int F, double f_lo, double f_hi, double fs,
                            int n_samples, const float* window, const float* call, int call_len, int per_comp,
                            float2* E_buf, float2* G_buf, float* out, cudaStream_t s);
// diffraction accumulation on the tensor cores (st_accum_mma.cu): omni emitter and receivers, paths grouped
// by material (material_order sorts the compacted candidate indices and writes the groups' offsets
// mat_off [n_mat + 1] on the device)
bool diffraction_mma_applies(const AccumArgs& a);
int32_t diffraction_mma_chunks(int64_t n_paths_hint, int32_t M, int32_t F, int32_t n_mat);
size_t material_order_scratch(int64_t cap);
cudaError_t material_order(const uint32_t* count, int64_t cap, const int32_t* cand_tri, const int32_t* tri_mat,
                           int n_mat, uint32_t* idx, uint32_t* mat_off, void* scratch, cudaStream_t s);
cudaError_t accumulate_diffraction_mma(const AccumArgs& a, const uint32_t* mat_off, cudaStream_t s);
struct AdjointArgs;
// the diffraction adjoint's position gradients on the tensor cores (same path order and chunking as the
// forward); its CTA grid: n_mb microphone blocks x n_bb bin blocks per chunk
void adjoint_diffraction_mma_shape(int32_t M, int32_t F, int32_t* n_mb, int32_t* n_bb);
cudaError_t adjoint_diffraction_mma(const AccumArgs& a, const AdjointArgs& j, const uint32_t* mat_off,
                                    cudaStream_t s);
// narrow receiver arrays (one microphone pair): a separate accumulator kernel
bool narrow_accum(int32_t M);
int32_t narrow_chunks(int64_t n_paths_hint, int32_t M, int32_t F, int32_t n_mat, int32_t dir_nb);
cudaError_t accumulate_narrow(const AccumArgs& a, cudaStream_t s);

struct GatherArgs {
    // specular
    int64_t N; int32_t B;
    const int32_t* rec_tri; const float* rec_p; const float* rec_d; const double* rec_r; const uint8_t* rec_los;
    const int32_t* tri_mat;
    const float* dirs; float q[4]; float fwd[3]; float inv_dtheta; int has_etab;
    // diffraction
    int64_t K; const int32_t* cand_tri; const float* cand_p; const uint8_t* keep; float s[3];
    // outputs
    const uint32_t* idx;   // compacted source indices
    const uint32_t* count;
    PathList* out;
    const uint64_t* rec_mask;  // optional: per-microphone visibility of the records, copied to out->mask
    int32_t n_mat = 256;       // checked build: materials of the scene
    uint32_t* chk = nullptr;   // checked build: flags word
};
cudaError_t gather_specular(const GatherArgs& g, cudaStream_t s);
// Stable sort of the compacted specular indices idx[0 .. cap) by emitter-table row (entries past *g.count
// last); keys [cap] and scratch (sort_scratch_bytes(cap)) are the caller's.
cudaError_t theta_order(const GatherArgs& g, int64_t cap, uint32_t* idx, uint64_t* keys, void* scratch,
                        cudaStream_t s);
// Stable sort of the compacted specular indices idx[0 .. cap) by the material counts of their reflection chains
// (materials 0..3; last_only: by the last hit's material), entries past *g.count last: the adjoint forms its
// reflection sums once per run of equal counts.  keys [cap] and scratch (sort_scratch_bytes(cap)) are the caller's.
cudaError_t chain_order(const GatherArgs& g, int64_t cap, int last_only, uint32_t* idx, uint64_t* keys, void* scratch,
                        cudaStream_t s);
cudaError_t gather_diffraction(const GatherArgs& g, cudaStream_t s);
cudaError_t flags_visible_records(const int32_t* rec_tri, const uint8_t* rec_los, int64_t n, uint32_t* flags,
                                  cudaStream_t s);
cudaError_t flags_from_u8(const uint8_t* keep, int64_t n, uint32_t* flags, cudaStream_t s);
cudaError_t compact_indices(const uint32_t* flags, const uint32_t* scan, int64_t n, uint32_t* idx, cudaStream_t s);

// ------------------------------------------------------------------ batched form (st_batch.cu)
// One pose of a batch as the device sees it.
struct JobDev {
    // scene
    const float4* nodes;
    const float4* tri_v;
    const float* nrm;
    const int32_t* tri_mat;
    const float* verts;
    const int32_t* tris;
    const int32_t* mesh_tris;
    const int64_t* mesh_off;
    const uint64_t* cdf;
    const int64_t* sample_off;
    int32_t root, max_iter, n_obj;
    int32_t n_mat;          // materials of the scene
    int32_t diff_mma;       // diffraction accumulated on the tensor cores (paths grouped by material)
    int64_t chk_nodes, chk_tris;  // checked build: wide nodes and triangles of the scene (see Trav::chk)
    float cos_fov;          // <= -1: field of view off
    // sensor inputs (the caller's device memory, read at run time)
    const float* s;
    const float* q;
    const float* dirs;
    const float* mics;
    // per-job derived data and tables (batch-owned)
    float* R;               // [3] receiver reference point
    float* fwd;             // [3] emitter forward axis
    const uint32_t* perm;   // [N] first-bounce processing order
    const float* qhi;
    const float* qlo;
    const float2* bw;       // [F] band index and weight of each bin
    // directivity (null: omni): emitter table [n_theta][F] (angle coordinate theta * inv_dtheta), receiver
    // tables [M][n_el][n_az][n_bands] and orientations [M][4]
    const float* etab;
    const float* mic_tab;
    const float* mic_q;
    int32_t n_theta, n_el, n_az, n_bands;
    float inv_dtheta;
    // sizes and offsets into the batch's global arrays
    int64_t N, K, ray_off, rec_off, samp_off, mic_off, mf_off;
    int32_t B, M, F;
    uint32_t pose;
    double f_lo, df;
    float2* out;            // spectra [3][M][F]
};

// entries per job of a batch's material offsets (materials 0 .. 254 and the end)
constexpr int kMatStride = 256;

struct BatchArgs {
    const JobDev* jobs;
    int32_t n_jobs;
    const int64_t* ray_offs;   // [n_jobs+1] each, ascending
    const int64_t* rec_offs;
    const int64_t* samp_offs;
    const int64_t* mic_offs;
    const int64_t* mf_offs;
    int64_t N_total, R_total, K_total, M_total, MF_total;
    double r_max, c, a0, a1;
    float t_min, los_eps, cos_inc, direct_gain;
    uint64_t seed;
    // ray state and queues
    float* ox; float* oy; float* oz; float* dx; float* dy; float* dz;
    double* racc;
    int32_t* prev;
    uint32_t* q_in; uint32_t* q_out; uint32_t* n_in; uint32_t* n_out;
    // records [R_total]
    int32_t* rec_tri; float* rec_p; float* rec_d; double* rec_r; uint8_t* rec_los;
    // candidates [K_total], direct visibility [M_total]
    int32_t* cand_tri; float* cand_p; uint8_t* keep; uint8_t* dvis;
    uint32_t* ranges;          // [n_jobs][4]: specular first path, count, diffraction first path, count
    // lane-refill traversal: closest hits [N_total], visibility queues of record / candidate ids and
    // their lengths, query counters ([0] closest hits, [1] record visibility, [2] candidate visibility)
    int32_t* hit_tri; float* hit_t;
    uint32_t* vis_q; uint32_t* vis_n; uint32_t* los_q; uint32_t* los_n;
    unsigned long long* ctr;
    uint32_t* flags;
    unsigned long long* queries;
    int32_t stack_limit;       // traversal stack entries per query (1..kStack; more: the query restarts stackless)
    int32_t refill;            // lane-refill threshold of the persistent traversal kernels (0 = default)
    // per-microphone receiver test (null otherwise): visible microphones of each record [R_total], and the
    // visibility queue of (record << 6 | microphone) entries, at most Q_total = sum over jobs of N x M a bounce
    uint64_t* rec_mask;
    uint64_t* vis_qm;
    int64_t Q_total;
};

cudaError_t batch_prep(const JobDev* jobs, int n_jobs, cudaStream_t s);
cudaError_t batch_trace(BatchArgs& a, int max_b, int64_t n_total, int block, cudaStream_t s);
cudaError_t batch_diffraction(const BatchArgs& a, cudaStream_t s);
cudaError_t batch_direct(const BatchArgs& a, cudaStream_t s);
cudaError_t batch_ranges(const BatchArgs& a, const uint32_t* scan_rec, const uint32_t* total_rec,
                         const uint32_t* scan_cand, const uint32_t* total_cand, cudaStream_t s);
cudaError_t batch_gather_spec(const BatchArgs& a, const uint32_t* idx, const uint32_t* count, PathList& P,
                              cudaStream_t s);
cudaError_t batch_gather_diff(const BatchArgs& a, const uint32_t* idx, const uint32_t* count, PathList& P,
                              cudaStream_t s);
cudaError_t batch_direct_accum(const BatchArgs& a, cudaStream_t s);

// Adjoint of one accumulation launch (st_adjoint.cu).
struct AdjointArgs {
    const float2* G;        // [M][F] dL/dRe S + j dL/dIm S of this component
    int do_pos;             // accumulate microphone / emitter position gradients
    int do_k;               // accumulate reflection sums V for materials mat_base .. mat_base + 3
    int do_beta;            // with do_k: V holds the lobe sums -gamma^2 Re w of the last hit's material instead
    int mat_base;
    float* v_part;          // [n_chunks * n_mb][4][F]
    float* mic_part;        // [n_chunks * n_bb][M][3]
    float* emit_part;       // [n_chunks * n_mb * n_bb][3]
    float s[3];             // emitter
    float a_0, a_step;      // amplitude decay (nepers per metre) at bin 0 and per bin
    float w_0, w_step;      // 2 pi f / c at bin 0 and per bin (rad per metre)
};

struct DirectAccumArgs {
    float s[3];
    const float* mics; int32_t M, F;
    const uint8_t* vis;
    double f_lo, df, c, a0, a1;
    float gain;
    const float* etab; int32_t n_theta; float fwd[3];
    const float* mic_tab; const float* mic_q; int32_t n_el, n_az, n_bands; const float2* bw;
    float2* out;           // [M][F] (component 2 of the spectra)
};
cudaError_t accumulate_direct(const DirectAccumArgs& a, const float* qhi, const float* qlo, cudaStream_t s);

namespace acc {
struct Geom;
}
acc::Geom adjoint_geom(int M, int F, int n_mat, int mat_direct = 0, int tp_max = 16, int kt = 8);
size_t adjoint_smem(const acc::Geom& g);
cudaError_t adjoint_launch(const AccumArgs& a, const AdjointArgs& j, const acc::Geom& g, cudaStream_t s);
cudaError_t adjoint_direct(const DirectAccumArgs& a, const float* qhi, const float* qlo, const float2* G,
                           float* mic_out, float* emit_out, cudaStream_t s);
cudaError_t adjoint_dk(const float* v_part, int n_slices, int F, int mat_base, int n_mat_launch, int n_bands,
                       const float* band_hz_dev, const float* k_dev, double f_lo, double df, float* dk, int n_mat,
                       cudaStream_t s);
// per compacted specular path: dP_j/ds (3x3 row-major) and dr_j/ds along its frozen chain (12 floats)
cudaError_t chain_jacobians(const uint32_t* idx, const uint32_t* count, int64_t n_max, int32_t B, const int32_t* rec_tri,
                            const float* rec_d, const float* nrm, const float* dirs, const float q[4], float* jac,
                            cudaStream_t s);
cudaError_t adjoint_dbeta(const float* v_part, int n_slices, int F, int mat_base, int n_mat_launch, int n_bands,
                          const float* band_hz_dev, const float* beta_dev, double f_lo, double df, float* dbeta,
                          cudaStream_t s);
cudaError_t adjoint_pos(const float* mic_parts, int n_mic_slices, const float* emit_parts, int n_emit_slices, int M,
                        float* dmic, float* demit, cudaStream_t s);

// last j in [0, n) with off[j] <= g (off ascending, off[0] = 0)
__device__ __forceinline__ int find_job(const int64_t* off, int n, int64_t g) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}


}  // namespace st
