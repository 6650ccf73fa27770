// C ABI of libsonotrace: contexts, scenes, inputs and the simulate pipeline.
//
// One simulate call issues, on the context's stream:
//   receiver reference point -> B bounce launches (Algorithm 1) -> visible-record compaction and
//   gathering -> diffraction sampling + filters + compaction (Sec. III-D) -> direct visibility and
//   spectrum (Sec. III-E) -> specular / diffraction accumulation and fixed-order chunk reduction.
// No host synchronisation happens inside unless statistics are requested.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>
#include <stdarg.h>

#include "st_accum_dev.cuh"
#include "st_internal.cuh"

using namespace st;

namespace st {

namespace {
// allocation-failure injection (st_inject_alloc_failure): allocations left before the injected
// failure, or -1 when off
int64_t g_fail_alloc_after = -1;
}  // namespace

cudaError_t grow(DevBuf& b, size_t bytes) {
    if (bytes <= b.cap && b.p) return cudaSuccess;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = std::max<size_t>(bytes, 256);
    if (g_fail_alloc_after >= 0 && g_fail_alloc_after-- == 0) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.cap = want;
    return cudaSuccess;
}

namespace {
int64_t g_launches = 0;  // host-side count of kernel launches issued by this library (not thread-safe)
}
void note_launch() { ++g_launches; }
int64_t launch_count() { return g_launches; }

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

}  // namespace st

struct BatchState;
struct st_scene;

struct st_ctx {
    int32_t device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // emitter
    bool has_emitter = false;
    float s[3] = {0, 0, 0}, q[4] = {1, 0, 0, 0};
    int64_t N = 0;
    DevBuf dirs, etab, perm, ord_keys, ord_scr;
    DevBuf th_keys, th_scr;          // emitter-table row order of the specular path list
    DevBuf vs_keys, vs_scr;          // hit-point Morton order of the visibility queries
    int32_t n_theta = 0;
    float fov_half = 4.0f;
    // receivers
    bool has_rx = false;
    int32_t M = 0;
    DevBuf mics, mic_q, mic_tab;
    bool has_mic_q = false;
    int32_t mic_nb = 0, n_el = 0, n_az = 0;  // receiver directivity tables (mic_nb = 0: omni)
    // frequencies
    bool has_freq = false;
    int32_t F = 0;
    double f_lo = 0, f_hi = 0;
    // tables cache
    AccumTables tables;
    const void* tables_scene = nullptr;
    uint64_t tables_version = 0;
    double tables_key[5] = {0, 0, 0, 0, 0};
    // work buffers
    DevBuf st_o[3], st_d[3], st_r, st_prev, q0, q1, counts, queries, flags, R, rec_tri, rec_p, rec_d, rec_r, rec_los;
    DevBuf sflags, sscan, sidx, scratch;
    PathList paths, paths_diff;  // gathered specular / diffraction paths of the last simulate
    DevBuf cand_tri, cand_p, keep, dvis, partial;
    DevBuf host_out;
    DevBuf adj_v, adj_mic, adj_emit;  // adjoint partial sums
    const st_scene* last_scene = nullptr;
    uint64_t last_scene_version = 0;
    int64_t last_N = 0, last_K = 0;
    int32_t last_B = 0, last_M = 0, last_F = 0;
    bool has_last = false;
    // last simulate parameters (for the adjoint)
    st_sim_params last_params;
    int32_t last_chunks_spec = 0, last_chunks_diff = 0;
    DevBuf mat_off, mat_scr;  // diffraction paths by material (tensor-core accumulation)
    bool last_diff_mma = false;  // the last simulate's diffraction list is in material order (mat_off valid)
    float last_fwd[3] = {1, 0, 0};
    bool count_visits = false;  // ST_COUNT_VISITS=1 in the environment: node/triangle visit counters
    st_tune tune{0, 0, 0, 0};   // launch shapes (st_autotune); 0 = default
    BatchState* batch = nullptr;
    std::vector<st_scene*> scenes;  // scenes loaded into this context (freed by st_destroy)
    DevBuf sig_e, sig_g;             // impulse responses: call spectrum [F], combined spectra [rows][F]
    DevBuf ray_tab;                  // zone table of the zonal ray set
    DevBuf adj_jac;                  // backward: chain jacobians of the specular paths [paths][12]
    DevBuf hit_tri, hit_t, vis_q, los_q, trav_cnt;
    DevBuf rec_mask;                 // per-microphone receiver test: visible microphones of each record  // lane-refill traversal: closest hits, query queues, counters
    cudaEvent_t ev[10] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // stage overlap: the diffraction stage and the direct path of a simulate run on a side stream while
    // the specular paths are traced (own copies of the buffers both would otherwise share)
    bool overlap = true;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    DevBuf los_keys, los_scr, dflags, dscan, didx, dscratch, dpartial;
    // backward: the specular path list of the last simulate put in chain order (keys and sort scratch)
    bool paths_chain_order = false;
    DevBuf ck_keys, ck_scr;
};

// Buffers and the recorded graph of the last batch structure.
struct BatchState {
    uint64_t key = 0;
    bool valid = false;
    int32_t n_jobs = 0, max_b = 0;
    std::vector<AccumTables> tables;
    std::vector<JobDev> jobs;
    std::vector<int32_t> chunks_spec, chunks_diff;
    DevBuf jobs_dev, offs, derived, perm, ord_keys, ord_scr;
    DevBuf st_o[3], st_d[3], st_r, st_prev, q0, q1, counts, queries, flags;
    DevBuf rec_tri, rec_p, rec_d, rec_r, rec_los, cand_tri, cand_p, keep, dvis, ranges;
    DevBuf sflags, sscan, sidx, scratch;
    DevBuf hit_tri, hit_t, vis_q, los_q;  // lane-refill traversal
    DevBuf rec_mask, vis_qm;              // per-microphone receiver test
    bool per_mic = false;
    int64_t Q_total = 0;                  // per-microphone visibility queries a bounce, at most
    DevBuf narrow_partial;  // chunk partials of the jobs accumulated on their own, one slice per branch
    size_t narrow_slice = 0;  // bytes of one branch's slice
    // persistent accumulation: one task per (job, path kind) -- the specular tasks, then the diffraction ones
    // -- their chunk partials, the work-item counter, item counts and the largest tile's shared memory
    std::vector<int32_t> narrow_jobs;  // jobs accumulated on their own (one microphone pair, or receiver tables)
    DevBuf tasks, part_all, qctr;
    int32_t n_tasks_spec = 0, n_tasks_diff = 0;
    int64_t items_spec = 0, items_diff = 0, n_out = 0;
    // diffraction on the tensor cores (jobs with diff_mma): their tasks follow the diffraction ones in the table;
    // the compacted candidates are sorted by (job, material) and mat_off holds each such job's groups
    int32_t n_tasks_mma = 0;
    int64_t items_mma = 0;
    bool any_mma = false;
    bool any_table_order = false;  // some job's diffraction paths go in emitter-table row order (its table)
    DevBuf mat_off, mat_scr;
    size_t smem_spec = 0, smem_diff = 0;
    PathList spec, diff;
    int64_t N_total = 0, R_total = 0, K_total = 0, M_total = 0, MF_total = 0;
    cudaStream_t main = nullptr;     // the batch runs here (capturable even when the context's stream is
                                     // the legacy default stream), ordered after/before the context's stream
    std::vector<cudaEvent_t> events;    // context -> main, main -> context
    // stage overlap (as in st_simulate): diffraction, its compaction and the direct visibility on a side
    // branch beside the trace; own scan scratch for the candidates
    bool overlap = false;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    DevBuf dscratch;
    // the jobs accumulated on their own run on kSoloBranches graph branches beside the work-queue launches
    cudaStream_t branch[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t br_fork = nullptr, br_join[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct st_scene {
    st_ctx* ctx = nullptr;
    SceneDev S;
    bool has_materials = false;
    uint64_t version = 0;
    st::CurvParamsDev cp{};  // parameters of the last precompute (reused by refits)
    bool precomputed = false;  // a precompute succeeded once (cp holds its parameters)
    bool instanced = false;  // loaded by st_scene_load_instances
    st::InstanceDev inst;
};

// Entry of every call on a context: select its device and drop a stale, non-sticky error left by
// earlier unrelated runtime calls, so that the launch checks below see only this call's errors.
static void enter(const st_ctx* c) {
    cudaSetDevice(c->device);
    (void)cudaGetLastError();
}

static void scene_free(st_scene* sc) {
    SceneDev& S = sc->S;
    for (DevBuf* b : {&S.verts, &S.tris, &S.tri_mat, &S.tri_obj, &S.nrm, &S.nodes, &S.tri_v, &S.G, &S.C, &S.mesh_tris,
                      &S.mesh_off, &S.cdf, &S.n_samples, &S.sample_off, &S.bvh_child, &S.bvh_range, &S.bvh_par_i,
                      &S.bvh_par_l, &S.bvh_perm, &S.bvh_wflag, &S.bvh_widx, &S.blas_nodes, &S.blas_tri, &S.blas_root,
                      &S.proto_box, &S.inst_rec, &S.tlas_inst})
        st::release(*b);
    st::InstanceDev& I = sc->inst;
    for (DevBuf* b : {&I.pverts, &I.ptris, &I.pmat, &I.pvoff, &I.ptoff, &I.iproto, &I.vbase, &I.tbase, &I.xform})
        st::release(*b);
    delete sc;
}


// ---- logging (ST_LOG=1: every error, 2: also one line per simulate, backward, precompute and batch) and
// NVTX ranges around the entry points and the stages of a simulate (seen by profilers that record NVTX)
static int log_level() {
    static const int lv = [] {
        const char* e = getenv("ST_LOG");
        return e ? atoi(e) : 0;
    }();
    return lv;
}

static void st_log(int level, const char* fmt, ...) {
    if (log_level() < level) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    fprintf(stderr, "sonotrace: %s\n", buf);
}

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Scene fields of the traversal arguments: the world-triangle BVH of a flat scene, or the top level and the
// prototypes' BVHs of a two-level one (whose iteration bound also counts instance steps and every instance's
// own nodes and triangles).
template <class A>
static void scene_trav_args(A& a, const SceneDev& S) {
    a.nodes = ptr<float4>(S.nodes);
    a.tri_v = ptr<float4>(S.tri_v);
    a.root = S.root;
    a.max_iter = (int32_t)std::min<int64_t>(2 * S.n_tris + 8, (int64_t)1 << 30);
    a.chk[0] = S.n_nodes > 0 ? S.n_nodes : 1;  // (a scene of one leaf keeps one node allocated)
    a.chk[1] = S.n_tris;
    a.chk[5] = S.n_tris;
    if (S.two_level) {
        a.chk[2] = std::max<int64_t>(S.blas_n_nodes, 1);
        a.chk[3] = S.inst ? S.inst->ptoff_h.back() : 0;
        a.chk[4] = S.inst ? S.inst->n_inst : 0;
        const int64_t n_inst = S.inst ? S.inst->n_inst : 0;
        a.bnodes = ptr<float4>(S.blas_nodes);
        a.btri = ptr<float4>(S.blas_tri);
        a.inst = ptr<float4>(S.inst_rec);
        a.tinst = ptr<int32_t>(S.tlas_inst);
        a.max_iter = (int32_t)std::min<int64_t>(2 * S.n_tris + 3 * n_inst + 8, (int64_t)1 << 30);
    }
}

namespace {

st_status fail(st_ctx* c, st_status code, const std::string& msg) {
    if (c) c->err = msg;
    st_log(1, "error %d: %s", (int)code, msg.c_str());
    return code;
}

st_status cuda_fail(st_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA, m);
}

#define CKC(ctx, x, where)                                   \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

cudaMemcpyKind kind_in(int32_t mem) { return mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int32_t mem) { return mem == ST_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

// a batched job's accumulation takes about 1/kBatchChunkDiv of the chunks that would fill the GPU alone (a job
// of a million paths or more takes them all: it is accumulated on its own)
constexpr int kBatchChunkDiv = 8;

// triangle count from which the visibility queries of a simulate are sorted by hit point (the 4-wide
// hierarchy and the triangles then take well over half of L2)
constexpr int64_t kVisSortTris = 1000000;

uint64_t g_scene_version = 1;

void batch_release(BatchState& B);
void batch_release_public(BatchState& B) { batch_release(B); }

}  // namespace

extern "C" {

void st_curv_params_default(st_curv_params* p) {
    if (!p) return;
    p->eta = 1.0f;
    p->area_ref = 1e-4f;
    p->dither = 1e-3;
    p->hc_frac = 0.25f;
    p->samples_per_vertex = 64;
    p->sample_budget = 4000000;
    p->seed = 0;
}

void st_sim_params_default(st_sim_params* p) {
    if (!p) return;
    p->max_bounces = 3;
    p->max_distance = 1e9;
    p->c = 343.0;
    p->alpha0_db_m = 0.0;
    p->alpha1_db_m_khz = 0.033;
    p->t_min = 1e-5f;
    p->los_eps = 1e-4f;
    p->reflection_mode = 0;
    p->components = ST_COMP_SPECULAR | ST_COMP_DIFFRACTION | ST_COMP_DIRECT;
    p->theta_inc_rad = (float)(80.0 * M_PI / 180.0);
    p->direct_gain = 1.0f;
    p->seed = 0;
    p->pose_index = 0;
    p->los_mode = ST_LOS_REFERENCE;
}

int32_t st_checked_build(void) {
#ifdef ST_CHECKS
    return 1;
#else
    return 0;
#endif
}

const char* st_status_string(st_status s) {
    switch (s) {
        case ST_OK: return "ok";
        case ST_ERR_ARG: return "invalid argument";
        case ST_ERR_CUDA: return "CUDA error";
        case ST_ERR_OOM: return "out of device memory";
        case ST_ERR_MESH: return "invalid mesh";
        case ST_ERR_TIMEOUT: return "device wait timed out";
        case ST_ERR_STATE: return "call out of order";
        case ST_ERR_OVERFLOW: return "device structure overflow";
        default: return "unknown status";
    }
}

const char* st_last_error(const st_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

st_status st_create(st_ctx** out, int32_t device, void* cuda_stream) {
    if (!out) return ST_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return ST_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return ST_ERR_CUDA;
    st_ctx* c = new st_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    const char* cv = getenv("ST_COUNT_VISITS");
    c->count_visits = cv && cv[0] == '1';
    for (auto& e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            delete c;
            return ST_ERR_CUDA;
        }
    *out = c;
    return ST_OK;
}

st_status st_destroy(st_ctx* c) {
    if (!c) return ST_ERR_ARG;
    enter(c);
    cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    for (DevBuf* b : {&c->mic_q, &c->mic_tab, &c->tables.bw}) release(*b);
    for (DevBuf* b : {&c->dirs, &c->etab, &c->perm, &c->ord_keys, &c->ord_scr, &c->th_keys, &c->th_scr, &c->vs_keys, &c->vs_scr, &c->mics, &c->st_o[0], &c->st_o[1], &c->st_o[2], &c->st_d[0], &c->st_d[1],
                      &c->st_d[2], &c->st_r, &c->st_prev, &c->q0, &c->q1, &c->counts, &c->queries, &c->flags, &c->R, &c->rec_tri,
                      &c->rec_p, &c->rec_d, &c->rec_r, &c->rec_los, &c->sflags, &c->sscan, &c->sidx, &c->scratch,
                      &c->cand_tri, &c->cand_p, &c->keep, &c->dvis, &c->partial, &c->host_out, &c->mat_off, &c->mat_scr, &c->tables.lk,
                      &c->tables.g2, &c->tables.lid, &c->tables.qhi, &c->tables.qlo})
        release(*b);
    for (PathList* P : {&c->paths, &c->paths_diff})
        for (DevBuf* b : {&P->px, &P->py, &P->pz, &P->dx, &P->dy, &P->dz, &P->rhi, &P->rlo, &P->chain_lo, &P->chain_hi,
                          &P->meta, &P->dep, &P->mask})
            release(*b);
    for (DevBuf* b : {&c->adj_v, &c->adj_mic, &c->adj_emit, &c->tables.band, &c->tables.kband, &c->tables.bband,
                      &c->sig_e, &c->sig_g,
                      &c->ray_tab, &c->adj_jac, &c->hit_tri, &c->hit_t, &c->vis_q, &c->los_q, &c->trav_cnt,
                      &c->rec_mask})
        release(*b);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    for (DevBuf* b : {&c->los_keys, &c->los_scr, &c->dflags, &c->dscan, &c->didx, &c->dscratch, &c->dpartial,
                      &c->ck_keys, &c->ck_scr})
        release(*b);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->batch) {
        batch_release_public(*c->batch);
        delete c->batch;
    }
    for (st_scene* sc : c->scenes) scene_free(sc);
    delete c;
    return ST_OK;
}

st_status st_set_stage_overlap(st_ctx* c, int32_t on) {
    if (!c) return ST_ERR_ARG;
    c->overlap = on != 0;
    return ST_OK;
}

st_status st_set_stream(st_ctx* c, void* stream) {
    if (!c) return ST_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return ST_OK;
}

// ------------------------------------------------------------------ scene
st_status st_scene_load(st_ctx* c, const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                        const int32_t* tri_material, const int32_t* tri_object, int32_t mem, st_scene** out) {
    if (!c || !out) return ST_ERR_ARG;
    *out = nullptr;
    if (!verts || !tris || !tri_material || !tri_object || n_verts <= 0 || n_tris <= 0 ||
        n_tris >= (1ll << 28) || n_verts >= (1ll << 31) || (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE))
        return fail(c, ST_ERR_ARG, "scene_load: null pointer or size out of range (1..2^28 triangles)");
    enter(c);
    st_scene* sc = new st_scene();
    sc->ctx = c;
    SceneDev& S = sc->S;
    S.n_verts = n_verts;
    S.n_tris = n_tris;
    cudaError_t e;
    if ((e = grow(S.verts, (size_t)n_verts * 12)) != cudaSuccess || (e = grow(S.tris, (size_t)n_tris * 12)) != cudaSuccess ||
        (e = grow(S.tri_mat, (size_t)n_tris * 4)) != cudaSuccess || (e = grow(S.tri_obj, (size_t)n_tris * 4)) != cudaSuccess) {
        scene_free(sc);
        return cuda_fail(c, e, "scene_load alloc");
    }
    cudaMemcpyAsync(S.verts.p, verts, (size_t)n_verts * 12, kind_in(mem), c->stream);
    cudaMemcpyAsync(S.tris.p, tris, (size_t)n_tris * 12, kind_in(mem), c->stream);
    cudaMemcpyAsync(S.tri_mat.p, tri_material, (size_t)n_tris * 4, kind_in(mem), c->stream);
    cudaMemcpyAsync(S.tri_obj.p, tri_object, (size_t)n_tris * 4, kind_in(mem), c->stream);
    // mesh count: max object id + 1 (host side needs it to size per-mesh arrays)
    std::vector<int32_t> obj(n_tris);
    e = cudaMemcpyAsync(obj.data(), S.tri_obj.p, (size_t)n_tris * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        scene_free(sc);
        return cuda_fail(c, e, "scene_load copy");
    }
    int32_t mx = -1;
    for (int32_t o : obj) {
        if (o < 0) {
            scene_free(sc);
            return fail(c, ST_ERR_MESH, "scene_load: negative object id");
        }
        mx = std::max(mx, o);
    }
    if (mx >= (1 << 24)) {
        scene_free(sc);
        return fail(c, ST_ERR_MESH, "scene_load: object ids must be < 2^24");
    }
    S.n_obj = mx + 1;
    sc->version = g_scene_version++;
    c->scenes.push_back(sc);
    *out = sc;
    return ST_OK;
}

st_status st_scene_set_materials(st_scene* sc, int32_t n_mat, int32_t n_bands, const float* band_hz, const float* k,
                                 const float* beta, const float* diffr) {
    if (!sc) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    if (n_mat <= 0 || n_mat > 255 || n_bands <= 0 || n_bands > 64 || !band_hz || !k || !beta || !diffr)
        return fail(c, ST_ERR_ARG, "set_materials: 1..255 materials, 1..64 bands, non-null tables");
    for (int b = 1; b < n_bands; ++b)
        if (!(band_hz[b] > band_hz[b - 1])) return fail(c, ST_ERR_ARG, "set_materials: band centres must ascend");
    for (int i = 0; i < n_mat * n_bands; ++i)
        if (!(beta[i] > 0.0f) || !(k[i] >= 0.0f) || !(diffr[i] >= 0.0f) || !isfinite(k[i]) || !isfinite(beta[i]))
            return fail(c, ST_ERR_ARG, "set_materials: need beta > 0, k >= 0, I_d >= 0, finite");
    SceneDev& S = sc->S;
    S.n_mat = n_mat;
    S.n_bands = n_bands;
    S.band_hz.assign(band_hz, band_hz + n_bands);
    S.k_band.assign(k, k + (size_t)n_mat * n_bands);
    S.beta_band.assign(beta, beta + (size_t)n_mat * n_bands);
    S.diff_band.assign(diffr, diffr + (size_t)n_mat * n_bands);
    sc->has_materials = true;
    sc->version = g_scene_version++;
    return ST_OK;
}

static st_status precompute_impl(st_scene* sc, const st_curv_params* params) {
    if (!sc) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    if (!sc->has_materials) return fail(c, ST_ERR_STATE, "scene_precompute: set materials first");
    st_curv_params p;
    st_curv_params_default(&p);
    if (params) p = *params;
    if (!(p.area_ref > 0.0f) || p.samples_per_vertex < 0 || !(p.dither >= 0.0))
        return fail(c, ST_ERR_ARG, "scene_precompute: area_ref > 0, samples_per_vertex >= 0, dither >= 0");
    enter(c);
    CurvParamsDev cp{p.eta, p.area_ref, p.hc_frac, p.dither, p.samples_per_vertex, p.sample_budget, p.seed};
    bool mesh_err = false;
    std::string msg;
    cudaError_t e = scene_build(sc->S, cp, c->stream, &mesh_err, &msg);
    if (e != cudaSuccess) return cuda_fail(c, e, "scene_precompute");
    if (mesh_err) return fail(c, ST_ERR_MESH, "scene_precompute: " + msg);
    sc->cp = cp;
    sc->precomputed = true;
    sc->version = g_scene_version++;
    return ST_OK;
}

// Refit of a precomputed scene whose vertex buffer holds new positions (same triangles); a scene left
// unbuilt by a failed update is built in full instead, with the parameters of its last precompute.
static st_status refit_scene(st_scene* sc, int32_t flags, const char* what) {
    st_ctx* c = sc->ctx;
    bool mesh_err = false;
    std::string msg;
    const bool refit = sc->S.built;
    cudaError_t e = scene_build(sc->S, sc->cp, c->stream, &mesh_err, &msg, refit,
                                refit && (flags & ST_REFIT_KEEP_CURVATURE) != 0);
    sc->version = g_scene_version++;
    if (e != cudaSuccess || mesh_err) sc->S.built = false;  // precompute again before the next simulate
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    if (mesh_err) return fail(c, ST_ERR_MESH, std::string(what) + ": " + msg);
    return ST_OK;
}

st_status st_scene_update_vertices(st_scene* sc, const float* verts, int32_t mem, int32_t flags) {
    if (!sc) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    if (!verts || (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE))
        return fail(c, ST_ERR_ARG, "scene_update_vertices: null pointer or bad memory kind");
    if (!sc->precomputed) return fail(c, ST_ERR_STATE, "scene_update_vertices: precompute first");
    if (sc->S.two_level)
        return fail(c, ST_ERR_STATE, "scene_update_vertices: a two-level scene moves by st_scene_set_instance_transforms");
    enter(c);
    CKC(c, cudaMemcpyAsync(sc->S.verts.p, verts, (size_t)sc->S.n_verts * 12, kind_in(mem), c->stream),
        "scene_update_vertices copy");
    return refit_scene(sc, flags, "scene_update_vertices");
}

st_status st_scene_load_instances(st_ctx* c, int32_t n_proto, const int64_t* proto_vert_offset,
                                  const float* proto_verts, const int64_t* proto_tri_offset, const int32_t* proto_tris,
                                  const int32_t* proto_tri_material, int32_t n_inst, const int32_t* inst_proto,
                                  const float* inst_xform, st_scene** out) {
    if (!c || !out) return ST_ERR_ARG;
    *out = nullptr;
    if (n_proto < 1 || n_inst < 1 || n_inst >= (1 << 24) || !proto_vert_offset || !proto_verts || !proto_tri_offset ||
        !proto_tris || !proto_tri_material || !inst_proto || !inst_xform)
        return fail(c, ST_ERR_ARG, "scene_load_instances: null pointer, no prototype, or 1..2^24 instances");
    if (proto_vert_offset[0] != 0 || proto_tri_offset[0] != 0)
        return fail(c, ST_ERR_ARG, "scene_load_instances: offsets must start at 0");
    for (int32_t q = 0; q < n_proto; ++q)
        if (proto_vert_offset[q + 1] < proto_vert_offset[q] || proto_tri_offset[q + 1] < proto_tri_offset[q] ||
            proto_vert_offset[q + 1] >= (1ll << 31) || proto_tri_offset[q + 1] >= (1ll << 28))
            return fail(c, ST_ERR_ARG, "scene_load_instances: offsets must ascend (< 2^31 vertices, < 2^28 triangles)");
    const int64_t pv = proto_vert_offset[n_proto], pt = proto_tri_offset[n_proto];
    // prototype meshes: local indices in range, finite vertices
    for (int32_t q = 0; q < n_proto; ++q) {
        const int64_t nvq = proto_vert_offset[q + 1] - proto_vert_offset[q];
        for (int64_t t = proto_tri_offset[q]; t < proto_tri_offset[q + 1]; ++t)
            for (int k = 0; k < 3; ++k)
                if (proto_tris[3 * t + k] < 0 || proto_tris[3 * t + k] >= nvq)
                    return fail(c, ST_ERR_MESH, "scene_load_instances: prototype vertex index out of range");
    }
    for (int64_t e = 0; e < 3 * pv; ++e)
        if (!std::isfinite(proto_verts[e])) return fail(c, ST_ERR_MESH, "scene_load_instances: non-finite vertex");
    // instance table: world bases
    std::vector<int64_t> vbase(n_inst + 1), tbase(n_inst + 1);
    vbase[0] = tbase[0] = 0;
    for (int32_t i = 0; i < n_inst; ++i) {
        const int32_t q = inst_proto[i];
        if (q < 0 || q >= n_proto) return fail(c, ST_ERR_MESH, "scene_load_instances: prototype id out of range");
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(inst_xform[12 * (int64_t)i + k]))
                return fail(c, ST_ERR_MESH, "scene_load_instances: non-finite transform");
        vbase[i + 1] = vbase[i] + (proto_vert_offset[q + 1] - proto_vert_offset[q]);
        tbase[i + 1] = tbase[i] + (proto_tri_offset[q + 1] - proto_tri_offset[q]);
        if (vbase[i + 1] >= (1ll << 31) || tbase[i + 1] >= (1ll << 28))
            return fail(c, ST_ERR_ARG, "scene_load_instances: more than 2^31 vertices or 2^28 triangles in the world");
    }
    const int64_t NV = vbase[n_inst], NT = tbase[n_inst];
    if (NV < 1 || NT < 1) return fail(c, ST_ERR_ARG, "scene_load_instances: the instances hold no triangle");
    enter(c);
    st_scene* sc = new st_scene();
    sc->ctx = c;
    sc->instanced = true;
    st::InstanceDev& I = sc->inst;
    sc->S.inst = &I;
    I.pvoff_h.assign(proto_vert_offset, proto_vert_offset + n_proto + 1);
    I.ptoff_h.assign(proto_tri_offset, proto_tri_offset + n_proto + 1);
    I.n_proto = n_proto;
    I.n_inst = n_inst;
    I.nv = NV;
    I.nt = NT;
    SceneDev& S = sc->S;
    S.n_verts = NV;
    S.n_tris = NT;
    S.n_obj = n_inst;
    cudaError_t e = cudaSuccess;
    const std::pair<DevBuf*, size_t> allocs[] = {
        {&I.pverts, (size_t)std::max<int64_t>(pv, 1) * 12}, {&I.ptris, (size_t)std::max<int64_t>(pt, 1) * 12},
        {&I.pmat, (size_t)std::max<int64_t>(pt, 1) * 4},    {&I.pvoff, (size_t)(n_proto + 1) * 8},
        {&I.ptoff, (size_t)(n_proto + 1) * 8},              {&I.iproto, (size_t)n_inst * 4},
        {&I.vbase, (size_t)(n_inst + 1) * 8},               {&I.tbase, (size_t)(n_inst + 1) * 8},
        {&I.xform, (size_t)n_inst * 48},                    {&S.verts, (size_t)NV * 12},
        {&S.tris, (size_t)NT * 12},                         {&S.tri_mat, (size_t)NT * 4},
        {&S.tri_obj, (size_t)NT * 4}};
    for (const auto& [b, bytes] : allocs)
        if (e == cudaSuccess) e = grow(*b, bytes);
    auto up = [&](DevBuf& b, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes > 0) e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, c->stream);
    };
    up(I.pverts, proto_verts, (size_t)pv * 12);
    up(I.ptris, proto_tris, (size_t)pt * 12);
    up(I.pmat, proto_tri_material, (size_t)pt * 4);
    up(I.pvoff, proto_vert_offset, (size_t)(n_proto + 1) * 8);
    up(I.ptoff, proto_tri_offset, (size_t)(n_proto + 1) * 8);
    up(I.iproto, inst_proto, (size_t)n_inst * 4);
    up(I.vbase, vbase.data(), (size_t)(n_inst + 1) * 8);
    up(I.tbase, tbase.data(), (size_t)(n_inst + 1) * 8);
    up(I.xform, inst_xform, (size_t)n_inst * 48);
    if (e == cudaSuccess) e = st::expand_instance_verts(I, ptr<float>(I.xform), ptr<float>(S.verts), c->stream);
    if (e == cudaSuccess)
        e = st::expand_instance_tris(I, ptr<int32_t>(S.tris), ptr<int32_t>(S.tri_mat), ptr<int32_t>(S.tri_obj), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host tables above are released on return
    if (e != cudaSuccess) {
        scene_free(sc);
        return cuda_fail(c, e, "scene_load_instances");
    }
    sc->version = g_scene_version++;
    c->scenes.push_back(sc);
    *out = sc;
    return ST_OK;
}

st_status st_scene_set_instance_transforms(st_scene* sc, const float* inst_xform, int32_t mem, int32_t flags) {
    if (!sc) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    if (!inst_xform || (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE))
        return fail(c, ST_ERR_ARG, "scene_set_instance_transforms: null pointer or bad memory kind");
    if (!sc->instanced) return fail(c, ST_ERR_STATE, "scene_set_instance_transforms: not an instanced scene");
    if (!sc->precomputed) return fail(c, ST_ERR_STATE, "scene_set_instance_transforms: precompute first");
    enter(c);
    st::InstanceDev& I = sc->inst;
    CKC(c, cudaMemcpyAsync(I.xform.p, inst_xform, (size_t)I.n_inst * 48, kind_in(mem), c->stream),
        "scene_set_instance_transforms copy");
    CKC(c, st::expand_instance_verts(I, ptr<float>(I.xform), ptr<float>(sc->S.verts), c->stream),
        "scene_set_instance_transforms expand");
    return refit_scene(sc, flags, "scene_set_instance_transforms");  // non-finite results: ST_ERR_MESH
}

st_status st_scene_set_structure(st_scene* sc, int32_t structure) {
    if (!sc) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    if (structure != ST_STRUCTURE_FLAT && structure != ST_STRUCTURE_TWO_LEVEL)
        return fail(c, ST_ERR_ARG, "scene_set_structure: ST_STRUCTURE_FLAT or ST_STRUCTURE_TWO_LEVEL");
    if (structure == ST_STRUCTURE_TWO_LEVEL && !sc->instanced)
        return fail(c, ST_ERR_STATE, "scene_set_structure: two levels need a scene loaded by st_scene_load_instances");
    const bool tl = structure == ST_STRUCTURE_TWO_LEVEL;
    if (tl == sc->S.two_level) return ST_OK;
    enter(c);
    CKC(c, cudaStreamSynchronize(c->stream), "scene_set_structure sync");  // earlier simulates may read the scene
    sc->S.two_level = tl;
    sc->S.tl_ready = false;
    sc->S.bvh_ready = false;
    if (c->batch) c->batch->valid = false;
    if (!sc->precomputed) return ST_OK;
    // rebuild with the parameters of the last precompute
    bool mesh_err = false;
    std::string msg;
    cudaError_t e = scene_build(sc->S, sc->cp, c->stream, &mesh_err, &msg);
    sc->version = g_scene_version++;
    if (e != cudaSuccess || mesh_err) sc->S.built = false;
    if (e != cudaSuccess) return cuda_fail(c, e, "scene_set_structure");
    if (mesh_err) return fail(c, ST_ERR_MESH, "scene_set_structure: " + msg);
    return ST_OK;
}

st_status st_scene_get_geometry(st_scene* sc, int64_t* n_verts, int64_t* n_tris, float* verts, int32_t* tris,
                                int32_t* tri_material, int32_t* tri_object, int32_t mem) {
    if (!sc) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    if (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE) return fail(c, ST_ERR_ARG, "scene_get_geometry: bad memory kind");
    if (n_verts) *n_verts = sc->S.n_verts;
    if (n_tris) *n_tris = sc->S.n_tris;
    enter(c);
    const SceneDev& S = sc->S;
    if (verts) CKC(c, cudaMemcpyAsync(verts, S.verts.p, (size_t)S.n_verts * 12, kind_out(mem), c->stream), "get verts");
    if (tris) CKC(c, cudaMemcpyAsync(tris, S.tris.p, (size_t)S.n_tris * 12, kind_out(mem), c->stream), "get tris");
    if (tri_material)
        CKC(c, cudaMemcpyAsync(tri_material, S.tri_mat.p, (size_t)S.n_tris * 4, kind_out(mem), c->stream), "get mat");
    if (tri_object)
        CKC(c, cudaMemcpyAsync(tri_object, S.tri_obj.p, (size_t)S.n_tris * 4, kind_out(mem), c->stream), "get obj");
    CKC(c, cudaStreamSynchronize(c->stream), "get geometry sync");
    return ST_OK;
}

st_status st_scene_get_curvature(st_scene* sc, float* G, float* C, int64_t* n_samples, int32_t mem) {
    if (!sc) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    if (!sc->S.built) return fail(c, ST_ERR_STATE, "scene_get_curvature: precompute first");
    enter(c);
    if (G) CKC(c, cudaMemcpyAsync(G, sc->S.G.p, (size_t)sc->S.n_verts * 4, kind_out(mem), c->stream), "get G");
    if (C) CKC(c, cudaMemcpyAsync(C, sc->S.C.p, (size_t)sc->S.n_tris * 4, kind_out(mem), c->stream), "get C");
    if (n_samples)
        CKC(c, cudaMemcpyAsync(n_samples, sc->S.n_samples.p, (size_t)sc->S.n_obj * 8, kind_out(mem), c->stream),
            "get n_samples");
    CKC(c, cudaStreamSynchronize(c->stream), "get curvature sync");
    return ST_OK;
}

st_status st_scene_destroy(st_scene* sc) {
    if (!sc) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    enter(c);
    cudaStreamSynchronize(c->stream);
    if (c->batch) c->batch->valid = false;  // a recorded batch may reference the scene
    if (c->tables_scene == sc) c->tables_scene = nullptr;
    c->scenes.erase(std::remove(c->scenes.begin(), c->scenes.end(), sc), c->scenes.end());
    scene_free(sc);
    return ST_OK;
}

// ------------------------------------------------------------------ sensor inputs
st_status st_set_emitter(st_ctx* c, const float pos[3], const float quat[4], int64_t n_rays, const float* dirs,
                         const float* dir_table, int32_t n_theta, float fov_half_rad, int32_t mem) {
    if (!c) return ST_ERR_ARG;
    if (!pos || !quat || n_rays < 0 || n_rays > (1ll << 31) - 1 || (n_rays > 0 && !dirs) ||
        (dir_table && n_theta < 2) || (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE))
        return fail(c, ST_ERR_ARG, "set_emitter: bad argument");
    enter(c);
    float hp[3], hq[4];
    if (mem == ST_MEM_DEVICE) {
        CKC(c, cudaMemcpyAsync(hp, pos, 12, cudaMemcpyDeviceToHost, c->stream), "set_emitter pos");
        CKC(c, cudaMemcpyAsync(hq, quat, 16, cudaMemcpyDeviceToHost, c->stream), "set_emitter quat");
        CKC(c, cudaStreamSynchronize(c->stream), "set_emitter sync");
    } else {
        memcpy(hp, pos, 12);
        memcpy(hq, quat, 16);
    }
    memcpy(c->s, hp, 12);
    memcpy(c->q, hq, 16);
    c->N = n_rays;
    if (n_rays > 0) {
        CKC(c, grow(c->dirs, (size_t)n_rays * 12), "set_emitter alloc");
        CKC(c, cudaMemcpyAsync(c->dirs.p, dirs, (size_t)n_rays * 12, kind_in(mem), c->stream), "set_emitter dirs");
        // first-bounce processing order: rays sorted by direction (coherent warps)
        CKC(c, grow(c->perm, (size_t)n_rays * 4), "set_emitter alloc");
        CKC(c, grow(c->ord_keys, (size_t)n_rays * 8), "set_emitter alloc");
        CKC(c, grow(c->ord_scr, sort_scratch_bytes(n_rays)), "set_emitter alloc");
        CKC(c, direction_order(ptr<float>(c->dirs), n_rays, ptr<uint64_t>(c->ord_keys), ptr<uint32_t>(c->perm),
                               c->ord_scr.p, c->stream),
            "set_emitter order");
    }
    c->n_theta = dir_table ? n_theta : 0;
    c->fov_half = fov_half_rad;
    c->has_emitter = true;
    if (dir_table) {
        // the bin count is known at simulate time; keep the raw table and check its size there
        if (!c->has_freq) return fail(c, ST_ERR_STATE, "set_emitter: set the frequency grid before a directivity table");
        const size_t bytes = (size_t)n_theta * c->F * 4;
        CKC(c, grow(c->etab, bytes), "set_emitter table alloc");
        CKC(c, cudaMemcpyAsync(c->etab.p, dir_table, bytes, kind_in(mem), c->stream), "set_emitter table");
    }
    return ST_OK;
}

st_status st_set_receivers(st_ctx* c, int32_t n_mics, const float* pos, const float* quats, const float* tables,
                           int32_t n_el, int32_t n_az, int32_t n_bands, int32_t mem) {
    if (!c) return ST_ERR_ARG;
    if (n_mics <= 0 || n_mics > kMaxMics || !pos || (mem != ST_MEM_HOST && mem != ST_MEM_DEVICE))
        return fail(c, ST_ERR_ARG, "set_receivers: 1..4096 microphones, non-null positions");
    if (tables && (n_el < 2 || n_az < 1 || n_bands < 1 || n_bands > 64))
        return fail(c, ST_ERR_ARG, "set_receivers: tables need n_el >= 2, n_az >= 1, 1..64 bands");
    enter(c);
    CKC(c, grow(c->mics, (size_t)n_mics * 12), "set_receivers alloc");
    CKC(c, cudaMemcpyAsync(c->mics.p, pos, (size_t)n_mics * 12, kind_in(mem), c->stream), "set_receivers copy");
    c->has_mic_q = quats != nullptr;
    if (quats) {
        CKC(c, grow(c->mic_q, (size_t)n_mics * 16), "set_receivers alloc");
        CKC(c, cudaMemcpyAsync(c->mic_q.p, quats, (size_t)n_mics * 16, kind_in(mem), c->stream), "set_receivers copy");
    }
    c->mic_nb = 0;
    if (tables) {
        const size_t bytes = (size_t)n_mics * n_el * n_az * n_bands * 4;
        CKC(c, grow(c->mic_tab, bytes), "set_receivers alloc");
        CKC(c, cudaMemcpyAsync(c->mic_tab.p, tables, bytes, kind_in(mem), c->stream), "set_receivers copy");
        c->mic_nb = n_bands;
        c->n_el = n_el;
        c->n_az = n_az;
    }
    c->M = n_mics;
    c->has_rx = true;
    return ST_OK;
}

void st_inject_alloc_failure(int64_t after) { st::g_fail_alloc_after = after < 0 ? -1 : after; }

st_status st_set_frequency_grid(st_ctx* c, int32_t n_bins, const float* f_hz) {
    if (!c) return ST_ERR_ARG;
    if (!f_hz || n_bins <= 0 || n_bins > (1 << 20)) return fail(c, ST_ERR_ARG, "set_frequency_grid: 1..2^20 bins");
    const double f_lo = f_hz[0], f_hi = f_hz[n_bins - 1];
    if (!(f_lo > 0.0) || !std::isfinite(f_hi)) return fail(c, ST_ERR_ARG, "set_frequency_grid: 0 < f_0, finite bins");
    const double df = n_bins > 1 ? (f_hi - f_lo) / (double)(n_bins - 1) : 0.0;
    for (int32_t k = 1; k < n_bins; ++k)
        if (!((double)f_hz[k] > (double)f_hz[k - 1]))
            return fail(c, ST_ERR_ARG, "set_frequency_grid: bins must be strictly ascending");
    // the accumulators advance every path's phasor by one constant bin spacing (one complex step per
    // bin), so the bins must lie on f_0 + k df: each within the float32 rounding of that grid point
    for (int32_t k = 1; k + 1 < n_bins; ++k) {
        const double want = f_lo + (double)k * df;
        if (std::fabs((double)f_hz[k] - want) > 4.0 * 1.2e-7 * std::fabs(want))
            return fail(c, ST_ERR_ARG, "set_frequency_grid: bins must be uniformly spaced");
    }
    return st_set_frequencies(c, n_bins, f_lo, f_hi);
}

st_status st_set_frequencies(st_ctx* c, int32_t n_bins, double f_lo, double f_hi) {
    if (!c) return ST_ERR_ARG;
    if (n_bins <= 0 || n_bins > (1 << 20) || !(f_lo > 0.0) || !(f_hi >= f_lo) || (n_bins > 1 && !(f_hi > f_lo)))
        return fail(c, ST_ERR_ARG, "set_frequencies: 1..2^20 bins, 0 < f_lo < f_hi");
    c->F = n_bins;
    c->f_lo = f_lo;
    c->f_hi = f_hi;
    c->has_freq = true;
    return ST_OK;
}

// ------------------------------------------------------------------ simulate
static st_status ensure_paths(st_ctx* c, PathList& P, int64_t n) {
    if (P.n_max >= n) return ST_OK;
    for (DevBuf* b : {&P.px, &P.py, &P.pz, &P.dx, &P.dy, &P.dz, &P.rhi, &P.rlo, &P.chain_lo, &P.chain_hi, &P.meta, &P.dep})
        CKC(c, grow(*b, (size_t)std::max<int64_t>(n, 1) * 4), "path list alloc");
    P.n_max = n;
    return ST_OK;
}

static st_status simulate_impl(st_ctx* c, st_scene* sc, const st_sim_params* params, void* spectra_out,
                               st_stats* stats) {
    if (!c || !sc || !spectra_out) return fail(c, ST_ERR_ARG, "simulate: null argument");
    if (!c->has_emitter || !c->has_rx || !c->has_freq)
        return fail(c, ST_ERR_STATE, "simulate: set emitter, receivers and frequencies first");
    if (!sc->S.built || !sc->has_materials) return fail(c, ST_ERR_STATE, "simulate: scene not precomputed");
    st_sim_params p;
    st_sim_params_default(&p);
    if (params) p = *params;
    if (p.max_bounces < 1 || p.max_bounces > kMaxBounces || !(p.c > 0.0) || !(p.t_min >= 0.0f) ||
        !(p.los_eps >= 0.0f) || p.reflection_mode < 0 || p.reflection_mode > 1)
        return fail(c, ST_ERR_ARG, "simulate: 1..8 bounces, c > 0, t_min >= 0, los_eps >= 0");
    if (p.los_mode != ST_LOS_REFERENCE && p.los_mode != ST_LOS_PER_MIC)
        return fail(c, ST_ERR_ARG, "simulate: los_mode must be ST_LOS_REFERENCE or ST_LOS_PER_MIC");
    if (p.los_mode == ST_LOS_PER_MIC &&
        (c->M > 64 || (uint64_t)c->N * (uint64_t)p.max_bounces * (uint64_t)c->M >= ((uint64_t)1 << 32)))
        return fail(c, ST_ERR_ARG, "simulate: the per-microphone receiver test needs M <= 64 and N * B * M < 2^32");
    if (c->n_theta > 0 && c->etab.cap < (size_t)c->n_theta * c->F * 4)
        return fail(c, ST_ERR_ARG, "simulate: emitter table was set for a different bin count");
    if (c->mic_nb > 0 && c->mic_nb != sc->S.n_bands)
        return fail(c, ST_ERR_ARG, "simulate: receiver tables must use the materials' bands");
    enter(c);
    cudaStream_t s = c->stream;
    SceneDev& S = sc->S;
    const int64_t N = c->N;
    const int32_t B = p.max_bounces, M = c->M, F = c->F;
    const int64_t NB = N * B;
    if (stats) CKC(c, cudaEventRecord(c->ev[0], s), "event");
    const int64_t launches0 = launch_count();

    // ---- per-bin tables (cached per scene materials, grid and constants)
    const double key[5] = {(double)F, c->f_lo, c->f_hi, p.c, 0.0};
    if (c->tables_scene != sc || c->tables_version != sc->version || memcmp(key, c->tables_key, sizeof(key)) != 0) {
        CKC(c, build_accum_tables(c->tables, S, F, c->f_lo, c->f_hi, p.c, p.alpha0_db_m, p.alpha1_db_m_khz, s),
            "tables");
        c->tables_scene = sc;
        c->tables_version = sc->version;
        memcpy(c->tables_key, key, sizeof(key));
    }
    AccumTables& T = c->tables;

    // ---- buffers
    const int64_t K = (p.components & ST_COMP_DIFFRACTION) ? S.total_samples : 0;
    const int64_t nflag = std::max<int64_t>(std::max<int64_t>(NB, K), 1);
    for (int k = 0; k < 3; ++k) {
        CKC(c, grow(c->st_o[k], (size_t)std::max<int64_t>(N, 1) * 4), "alloc");
        CKC(c, grow(c->st_d[k], (size_t)std::max<int64_t>(N, 1) * 4), "alloc");
    }
    CKC(c, grow(c->st_r, (size_t)std::max<int64_t>(N, 1) * 8), "alloc");
    CKC(c, grow(c->st_prev, (size_t)std::max<int64_t>(N, 1) * 4), "alloc");
    CKC(c, grow(c->q0, (size_t)std::max<int64_t>(N, 1) * 4), "alloc");
    CKC(c, grow(c->q1, (size_t)std::max<int64_t>(N, 1) * 4), "alloc");
    CKC(c, grow(c->counts, 64), "alloc");
    CKC(c, grow(c->queries, 64), "alloc");
    CKC(c, grow(c->flags, 16), "alloc");
    CKC(c, grow(c->R, 16), "alloc");
    CKC(c, grow(c->hit_tri, (size_t)std::max<int64_t>(N, 1) * 4), "alloc");
    CKC(c, grow(c->hit_t, (size_t)std::max<int64_t>(N, 1) * 4), "alloc");
    const bool per_mic = p.los_mode == ST_LOS_PER_MIC;
    CKC(c, grow(c->vis_q, (size_t)std::max<int64_t>(N, 1) * (per_mic ? (size_t)M : 1) * 4), "alloc");
    if (per_mic) {
        CKC(c, grow(c->rec_mask, (size_t)std::max<int64_t>(NB, 1) * 8), "alloc");
        CKC(c, grow(c->paths.mask, (size_t)std::max<int64_t>(NB, 1) * 8), "alloc");
    }
    CKC(c, grow(c->trav_cnt, 64), "alloc");
    CKC(c, grow(c->rec_tri, (size_t)std::max<int64_t>(NB, 1) * 4), "alloc");
    CKC(c, grow(c->rec_p, (size_t)std::max<int64_t>(NB, 1) * 12), "alloc");
    CKC(c, grow(c->rec_d, (size_t)std::max<int64_t>(NB, 1) * 12), "alloc");
    CKC(c, grow(c->rec_r, (size_t)std::max<int64_t>(NB, 1) * 8), "alloc");
    CKC(c, grow(c->rec_los, (size_t)std::max<int64_t>(NB, 1)), "alloc");
    CKC(c, grow(c->sflags, (size_t)nflag * 4), "alloc");
    CKC(c, grow(c->sscan, (size_t)nflag * 4), "alloc");
    CKC(c, grow(c->sidx, (size_t)nflag * 4), "alloc");
    CKC(c, grow(c->scratch, scan_scratch_bytes(nflag)), "alloc");
    // Scenes whose hierarchy and triangles are well beyond L2 trace their visibility queries in the Morton
    // order of the hit points (all go to one point, so neighbours in that order share most nodes)
    const bool vsort = S.n_tris >= kVisSortTris && N > 1 && !per_mic;
    if (vsort) {
        CKC(c, grow(c->vs_keys, (size_t)N * 8), "alloc");
        CKC(c, grow(c->vs_scr, sort_scratch_bytes(N)), "alloc");
    }
    if (K > 1) {  // the line-of-sight queue of the diffraction candidates is sorted likewise (own buffers)
        CKC(c, grow(c->los_keys, (size_t)K * 8), "alloc");
        CKC(c, grow(c->los_scr, sort_scratch_bytes(K)), "alloc");
    }
    if (c->n_theta > 0 && NB > 1) {  // emitter-table row order of the specular path list
        CKC(c, grow(c->th_keys, (size_t)NB * 8), "alloc");
        CKC(c, grow(c->th_scr, sort_scratch_bytes(NB)), "alloc");
    }
    CKC(c, grow(c->dvis, (size_t)M), "alloc");
    st_status ps = ensure_paths(c, c->paths, std::max<int64_t>(NB, 1));
    if (ps != ST_OK) return ps;
    ps = ensure_paths(c, c->paths_diff, std::max<int64_t>(K, 1));
    if (ps != ST_OK) return ps;
    if (K > 0) {
        CKC(c, grow(c->cand_tri, (size_t)K * 4), "alloc");
        CKC(c, grow(c->cand_p, (size_t)K * 12), "alloc");
        CKC(c, grow(c->keep, (size_t)K), "alloc");
        CKC(c, grow(c->los_q, (size_t)K * 4), "alloc");
    }
    const int32_t chunks_spec =
        accum_chunks(NB, M, F, S.n_mat, c->mic_nb, c->tune.mic_pairs_per_cta, c->tune.smem_kb, c->tune.bins_per_thread);
    // diffraction on the tensor cores when the per-bin factor depends on material and bin only
    bool diff_mma = false;
    {
        AccumArgs probe{};
        probe.kind = 1;
        probe.etab = c->n_theta > 0 ? ptr<float>(c->etab) : nullptr;
        probe.mic_tab = c->mic_nb > 0 ? ptr<float>(c->mic_tab) : nullptr;
        probe.M = M;
        probe.F = F;
        probe.n_mat_tab = S.n_mat;
        diff_mma = K > 0 && diffraction_mma_applies(probe);
    }
    const int32_t chunks_diff =
        diff_mma ? diffraction_mma_chunks(K, M, F, S.n_mat)
                 : accum_chunks(K, M, F, S.n_mat, c->mic_nb, c->tune.mic_pairs_per_cta, c->tune.smem_kb,
                                c->tune.bins_per_thread);
    if (diff_mma) {
        CKC(c, grow(c->mat_off, (size_t)(S.n_mat + 1) * 4), "alloc");
        CKC(c, grow(c->mat_scr, material_order_scratch(K)), "alloc");
    }
    CKC(c, grow(c->partial, (size_t)chunks_spec * M * F * 8), "alloc");
    if (K > 0) {  // the diffraction stage's compaction and partial spectra (it may run beside the specular one)
        CKC(c, grow(c->dflags, (size_t)K * 4), "alloc");
        CKC(c, grow(c->dscan, (size_t)K * 4), "alloc");
        CKC(c, grow(c->didx, (size_t)K * 4), "alloc");
        CKC(c, grow(c->dscratch, scan_scratch_bytes(K)), "alloc");
        CKC(c, grow(c->dpartial, (size_t)chunks_diff * M * F * 8), "alloc");
    }

    float2* out = static_cast<float2*>(spectra_out);
    const int64_t MF = (int64_t)M * F;
    CKC(c, cudaMemsetAsync(out, 0, (size_t)3 * MF * 8, s), "memset out");
    CKC(c, cudaMemsetAsync(c->flags.p, 0, 16, s), "memset");
    CKC(c, cudaMemsetAsync(c->counts.p, 0, 64, s), "memset");
    CKC(c, cudaMemsetAsync(c->queries.p, 0, 64, s), "memset");
    unsigned long long* qctr = ptr<unsigned long long>(c->queries);
    CKC(c, cudaMemsetAsync(c->rec_tri.p, 0xff, (size_t)std::max<int64_t>(NB, 1) * 4, s), "memset");
    CKC(c, cudaMemsetAsync(c->rec_los.p, 0, (size_t)std::max<int64_t>(NB, 1), s), "memset");
    if (per_mic) CKC(c, cudaMemsetAsync(c->rec_mask.p, 0, (size_t)std::max<int64_t>(NB, 1) * 8, s), "memset");
    CKC(c, cudaMemsetAsync(c->rec_r.p, 0, (size_t)std::max<int64_t>(NB, 1) * 8, s), "memset");
    CKC(c, cudaMemsetAsync(c->rec_p.p, 0, (size_t)std::max<int64_t>(NB, 1) * 12, s), "memset");
    CKC(c, cudaMemsetAsync(c->rec_d.p, 0, (size_t)std::max<int64_t>(NB, 1) * 12, s), "memset");
    uint32_t* cnt = ptr<uint32_t>(c->counts);  // [0],[1] queue counts, [2] visible records, [3] kept candidates
    mic_centroid_host_order(ptr<float>(c->mics), M, ptr<float>(c->R), s);
    CKC(c, cudaGetLastError(), "centroid");

    float fwd[3];
    {
        // forward axis = q applied to +x (host float32, the same steps as the device rotation)
        const float* q = c->q;
        const float vx = 1.0f, vy = 0.0f, vz = 0.0f;
        const float cx = q[2] * vz - q[3] * vy, cy = q[3] * vx - q[1] * vz, cz = q[1] * vy - q[2] * vx;
        const float tx = 2.0f * cx, ty = 2.0f * cy, tz = 2.0f * cz;
        const float c2x = q[2] * tz - q[3] * ty, c2y = q[3] * tx - q[1] * tz, c2z = q[1] * ty - q[2] * tx;
        fwd[0] = (vx + q[0] * tx) + c2x;
        fwd[1] = (vy + q[0] * ty) + c2y;
        fwd[2] = (vz + q[0] * tz) + c2z;
    }

    // ---- stage overlap: the diffraction stage (sampling and line of sight, Sec. III-D; its accumulation)
    // and the direct path run on the context's side stream while the specular paths are traced on the
    // context's stream, filling the traversal launches' tails; the specular accumulation waits for both
    // and runs alone.  The stages share no buffer (the diffraction stage has its own sort, compaction and
    // partial-spectra buffers) and no result depends on the order (fixed-order sums, compaction by scan).
    const bool overlap = c->overlap && (p.components & ST_COMP_SPECULAR) && N > 0 &&
                         (K > 0 || (p.components & ST_COMP_DIRECT));
    cudaStream_t s2 = s;
    bool joined = false;
    if (overlap) {
        if (!c->side) {
            CKC(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "side stream");
            CKC(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event");
            CKC(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event");
        }
        CKC(c, cudaEventRecord(c->ev_fork, s), "fork");
        CKC(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork");
        s2 = c->side;
    }
    // a call that fails between the fork and the join still orders the side stream's work before the
    // context stream's next work
    struct JoinGuard {
        st_ctx* c;
        cudaStream_t s;
        const bool& active;
        const bool& done;
        ~JoinGuard() {
            if (active && !done) {
                cudaEventRecord(c->ev_join, c->side);
                cudaStreamWaitEvent(s, c->ev_join, 0);
            }
        }
    } join_guard{c, s, overlap, joined};

    auto stage_trace = [&]() -> st_status {
        // ---- Algorithm 1
        if (p.components & ST_COMP_SPECULAR && N > 0) {
            NvtxRange range("st_simulate: trace");
            TraceArgs ta{};
            scene_trav_args(ta, S);
            ta.visits = c->count_visits ? qctr + 2 : nullptr;
            ta.stack_limit = c->tune.stack_depth > 0 ? std::min(c->tune.stack_depth, kStack) : kStack;
            ta.restarts = qctr + 6;
            ta.refill = c->tune.refill_lanes;
            ta.nrm = ptr<float>(S.nrm);
            memcpy(ta.s, c->s, 12);
            memcpy(ta.q, c->q, 16);
            ta.R = ptr<float>(c->R);
            ta.dirs = ptr<float>(c->dirs);
            ta.perm = ptr<uint32_t>(c->perm);
            ta.N = N;
            ta.B = B;
            ta.r_max = p.max_distance;
            ta.t_min = p.t_min;
            ta.los_eps = p.los_eps;
            ta.ox = ptr<float>(c->st_o[0]);
            ta.oy = ptr<float>(c->st_o[1]);
            ta.oz = ptr<float>(c->st_o[2]);
            ta.dx = ptr<float>(c->st_d[0]);
            ta.dy = ptr<float>(c->st_d[1]);
            ta.dz = ptr<float>(c->st_d[2]);
            ta.racc = ptr<double>(c->st_r);
            ta.prev = ptr<int32_t>(c->st_prev);
            ta.q_in = ptr<uint32_t>(c->q0);
            ta.q_out = ptr<uint32_t>(c->q1);
            ta.n_in = cnt + 0;
            ta.n_out = cnt + 1;
            ta.rec_tri = ptr<int32_t>(c->rec_tri);
            ta.rec_p = ptr<float>(c->rec_p);
            ta.rec_d = ptr<float>(c->rec_d);
            ta.rec_r = ptr<double>(c->rec_r);
            ta.rec_los = ptr<uint8_t>(c->rec_los);
            ta.flags = ptr<uint32_t>(c->flags);
            ta.queries = qctr;
            ta.hit_tri = ptr<int32_t>(c->hit_tri);
            ta.hit_t = ptr<float>(c->hit_t);
            ta.vis_q = ptr<uint32_t>(c->vis_q);
            ta.vis_n = ptr<uint32_t>(c->trav_cnt);
            ta.ctr = reinterpret_cast<unsigned long long*>(ptr<char>(c->trav_cnt) + 16);
            ta.rec_mask = per_mic ? ptr<uint64_t>(c->rec_mask) : nullptr;
            ta.mics = ptr<float>(c->mics);
            ta.M = M;
            ta.sort_keys = vsort ? ptr<uint64_t>(c->vs_keys) : nullptr;
            ta.sort_scr = vsort ? c->vs_scr.p : nullptr;
            for (int k = 0; k < 3; ++k) {
                const float ext = S.bounds_hi[k] - S.bounds_lo[k];
                ta.blo[k] = S.bounds_lo[k];
                ta.bscale[k] = ext > 0.0f ? 1024.0f / ext : 0.0f;
            }
            CKC(c, trace_rays(ta, s, c->tune.rays_per_block > 0 ? c->tune.rays_per_block : 128), "trace");
        }
        return ST_OK;
    };
    auto stage_diffraction = [&]() -> st_status {
        // ---- diffraction (Sec. III-D)
        if (K > 0) {
            NvtxRange range("st_simulate: diffraction sampling");
            DiffArgs da{};
            scene_trav_args(da, S);
            da.visits = c->count_visits ? qctr + 2 : nullptr;
            da.stack_limit = c->tune.stack_depth > 0 ? std::min(c->tune.stack_depth, kStack) : kStack;
            da.restarts = qctr + 6;
            da.refill = c->tune.refill_lanes;
            da.nrm = ptr<float>(S.nrm);
            da.verts = ptr<float>(S.verts);
            da.tris = ptr<int32_t>(S.tris);
            da.n_obj = S.n_obj;
            da.mesh_tris = ptr<int32_t>(S.mesh_tris);
            da.mesh_off = ptr<int64_t>(S.mesh_off);
            da.cdf = ptr<uint64_t>(S.cdf);
            da.sample_off = ptr<int64_t>(S.sample_off);
            da.K = K;
            da.seed = p.seed;
            da.pose = p.pose_index;
            memcpy(da.s, c->s, 12);
            memcpy(da.fwd, fwd, 12);
            da.cos_fov = c->fov_half >= (float)M_PI ? -2.0f : (float)cos((double)c->fov_half);
            da.cos_inc = (float)cos((double)p.theta_inc_rad);
            da.t_min = p.t_min;
            da.los_eps = p.los_eps;
            da.cand_tri = ptr<int32_t>(c->cand_tri);
            da.cand_p = ptr<float>(c->cand_p);
            da.keep = ptr<uint8_t>(c->keep);
            da.flags = ptr<uint32_t>(c->flags);
            da.queries = qctr;
            da.los_q = ptr<uint32_t>(c->los_q);
            da.los_n = ptr<uint32_t>(c->trav_cnt) + 1;
            da.ctr = reinterpret_cast<unsigned long long*>(ptr<char>(c->trav_cnt) + 32);
            da.sort_keys = K > 1 ? ptr<uint64_t>(c->los_keys) : nullptr;
            da.sort_scr = K > 1 ? c->los_scr.p : nullptr;
            for (int k = 0; k < 3; ++k) {
                const float ext = S.bounds_hi[k] - S.bounds_lo[k];
                da.blo[k] = S.bounds_lo[k];
                da.bscale[k] = ext > 0.0f ? 1024.0f / ext : 0.0f;
            }
            if (stats) CKC(c, cudaEventRecord(c->ev[8], s2), "event");
            CKC(c, diffraction_sample(da, s2), "diffraction");
            if (stats) CKC(c, cudaEventRecord(c->ev[9], s2), "event");
        }
        return ST_OK;
    };

    const float inv_dtheta = c->n_theta > 1 ? (float)((c->n_theta - 1) / M_PI) : 0.0f;
    const double l2_10_over_20 = log2(10.0) / 20.0;
    AccumArgs aa{};
    aa.mics = ptr<float>(c->mics);
    aa.M = M;
    aa.F = F;
    aa.lk = ptr<float>(T.lk);
    aa.g2 = ptr<float>(T.g2);
    aa.lid = ptr<float>(T.lid);
    aa.n_mat_tab = T.n_mat;
    aa.n_bands_tab = S.n_bands;
    aa.bw = ptr<float2>(T.bw);
    aa.qhi = ptr<float>(T.qhi);
    aa.qlo = ptr<float>(T.qlo);
    {
        const double dq = T.df / p.c;
        aa.dq_hi = (float)dq;
        aa.dq_lo = (float)(dq - (double)aa.dq_hi);
        aa.atm2_0 = (float)(-(p.alpha0_db_m + p.alpha1_db_m_khz * c->f_lo / 1000.0) * l2_10_over_20);
        aa.atm2_step = (float)(-(p.alpha1_db_m_khz * T.df / 1000.0) * l2_10_over_20);
    }
    aa.etab = c->n_theta > 0 ? ptr<float>(c->etab) : nullptr;
    aa.n_theta = c->n_theta;
    aa.n_bands_tab = S.n_bands;
    aa.mic_tab = c->mic_nb > 0 ? ptr<float>(c->mic_tab) : nullptr;
    aa.mic_q = (c->mic_nb > 0 && c->has_mic_q) ? ptr<float>(c->mic_q) : nullptr;
    aa.n_el = c->n_el;
    aa.n_az = c->n_az;
    aa.bw = ptr<float2>(T.bw);
    aa.reflection_mode = p.reflection_mode;
    aa.partial = ptr<float2>(c->partial);
    aa.tile_tp = c->tune.mic_pairs_per_cta;
    aa.tile_kb = c->tune.smem_kb;
    aa.tile_kt = c->tune.bins_per_thread;

    GatherArgs ga{};
    ga.N = N;
    ga.B = B;
    ga.rec_tri = ptr<int32_t>(c->rec_tri);
    ga.rec_p = ptr<float>(c->rec_p);
    ga.rec_d = ptr<float>(c->rec_d);
    ga.rec_r = ptr<double>(c->rec_r);
    ga.rec_los = ptr<uint8_t>(c->rec_los);
    ga.tri_mat = ptr<int32_t>(S.tri_mat);
    ga.dirs = ptr<float>(c->dirs);
    memcpy(ga.q, c->q, 16);
    memcpy(ga.fwd, fwd, 12);
    ga.inv_dtheta = inv_dtheta;
    ga.has_etab = c->n_theta > 0;
    ga.K = K;
    ga.cand_tri = ptr<int32_t>(c->cand_tri);
    ga.cand_p = ptr<float>(c->cand_p);
    ga.keep = ptr<uint8_t>(c->keep);
    memcpy(ga.s, c->s, 12);
    ga.idx = ptr<uint32_t>(c->sidx);
    ga.rec_mask = per_mic ? ptr<uint64_t>(c->rec_mask) : nullptr;
    ga.n_mat = S.n_mat;
    ga.chk = ptr<uint32_t>(c->flags);
    auto set_paths = [&](AccumArgs& x, PathList& PL) {
        x.px = ptr<float>(PL.px);
        x.py = ptr<float>(PL.py);
        x.pz = ptr<float>(PL.pz);
        x.dx = ptr<float>(PL.dx);
        x.dy = ptr<float>(PL.dy);
        x.dz = ptr<float>(PL.dz);
        x.rhi = ptr<float>(PL.rhi);
        x.rlo = ptr<float>(PL.rlo);
        x.chain_lo = ptr<uint32_t>(PL.chain_lo);
        x.chain_hi = ptr<uint32_t>(PL.chain_hi);
        x.meta = ptr<uint32_t>(PL.meta);
        x.dep = ptr<float>(PL.dep);
    };

    int n_accum = 0;  // bit 0: specular launch issued, bit 1: diffraction launch issued
    auto stage_specular = [&]() -> st_status {
        // ---- specular accumulation (Eq. 2-4)
        if (p.components & ST_COMP_SPECULAR && NB > 0) {
            NvtxRange range("st_simulate: specular accumulation");
            CKC(c, flags_visible_records(ptr<int32_t>(c->rec_tri), ptr<uint8_t>(c->rec_los), NB, ptr<uint32_t>(c->sflags), s),
                "flags");
            CKC(c, exclusive_scan_u32(ptr<uint32_t>(c->sflags), ptr<uint32_t>(c->sscan), NB, cnt + 2, c->scratch.p, s),
                "scan");
            CKC(c, compact_indices(ptr<uint32_t>(c->sflags), ptr<uint32_t>(c->sscan), NB, ptr<uint32_t>(c->sidx), s),
                "compact");
            ga.count = cnt + 2;
            ga.out = &c->paths;
            if (ga.has_etab && NB > 1) {  // paths in emitter-table row order: a tile's paths share table rows
                CKC(c, theta_order(ga, NB, ptr<uint32_t>(c->sidx), ptr<uint64_t>(c->th_keys), c->th_scr.p, s), "order");
            }
            CKC(c, gather_specular(ga, s), "gather");
            AccumArgs x = aa;
            x.kind = 0;
            x.n_paths = NB;
            x.d_count = cnt + 2;
            set_paths(x, c->paths);
            x.mask = per_mic ? ptr<uint64_t>(c->paths.mask) : nullptr;
            x.n_chunks = chunks_spec;
            // the side stream's stages end before the accumulation starts, so that it runs alone
            if (overlap) {
                CKC(c, cudaEventRecord(c->ev_join, s2), "join");
                CKC(c, cudaStreamWaitEvent(s, c->ev_join, 0), "join");
                joined = true;
            }
            if (stats) CKC(c, cudaEventRecord(c->ev[4], s), "event");
            CKC(c, accumulate(x, s), "accumulate specular");
            if (stats) CKC(c, cudaEventRecord(c->ev[5], s), "event");
            n_accum++;
            CKC(c, reduce_partials(ptr<float2>(c->partial), chunks_spec, MF, out, s), "reduce");
        }
        return ST_OK;
    };
    auto stage_diffraction_accumulation = [&]() -> st_status {
        // ---- diffraction accumulation (Eq. 7-8)
        if (K > 0) {
            NvtxRange range("st_simulate: diffraction accumulation");
            CKC(c, flags_from_u8(ptr<uint8_t>(c->keep), K, ptr<uint32_t>(c->dflags), s2), "flags");
            CKC(c, exclusive_scan_u32(ptr<uint32_t>(c->dflags), ptr<uint32_t>(c->dscan), K, cnt + 3, c->dscratch.p, s2),
                "scan");
            CKC(c, compact_indices(ptr<uint32_t>(c->dflags), ptr<uint32_t>(c->dscan), K, ptr<uint32_t>(c->didx), s2),
                "compact");
            GatherArgs gd = ga;
            gd.idx = ptr<uint32_t>(c->didx);
            gd.count = cnt + 3;
            gd.out = &c->paths_diff;
            if (diff_mma)  // path list grouped by material (stable: within a material the compaction order)
                CKC(c, material_order(cnt + 3, K, ptr<int32_t>(c->cand_tri), ptr<int32_t>(S.tri_mat), S.n_mat,
                                      ptr<uint32_t>(c->didx), ptr<uint32_t>(c->mat_off), c->mat_scr.p, s2),
                    "material order");
            CKC(c, gather_diffraction(gd, s2), "gather");
            AccumArgs x = aa;
            x.kind = 1;
            x.n_paths = K;
            x.d_count = cnt + 3;
            set_paths(x, c->paths_diff);
            x.n_chunks = chunks_diff;
            x.partial = ptr<float2>(c->dpartial);
            if (stats) CKC(c, cudaEventRecord(c->ev[6], s2), "event");
            if (diff_mma)
                CKC(c, accumulate_diffraction_mma(x, ptr<uint32_t>(c->mat_off), s2), "accumulate diffraction");
            else
                CKC(c, accumulate(x, s2), "accumulate diffraction");
            if (stats) CKC(c, cudaEventRecord(c->ev[7], s2), "event");
            n_accum += 2;
            CKC(c, reduce_partials(ptr<float2>(c->dpartial), chunks_diff, MF, out + MF, s2), "reduce");
        }
        return ST_OK;
    };
    auto stage_direct = [&]() -> st_status {
        // ---- direct path (Eq. 11-12)
        if (p.components & ST_COMP_DIRECT) {
            NvtxRange range("st_simulate: direct path");
            DirectArgs dv{};
            scene_trav_args(dv, S);
            dv.visits = c->count_visits ? qctr + 2 : nullptr;
            dv.stack_limit = c->tune.stack_depth > 0 ? std::min(c->tune.stack_depth, kStack) : kStack;
            dv.restarts = qctr + 6;
            dv.refill = c->tune.refill_lanes;
            memcpy(dv.s, c->s, 12);
            dv.mics = ptr<float>(c->mics);
            dv.M = M;
            dv.t_min = p.t_min;
            dv.los_eps = p.los_eps;
            dv.vis = ptr<uint8_t>(c->dvis);
            dv.flags = ptr<uint32_t>(c->flags);
            dv.queries = qctr;
            CKC(c, direct_visibility(dv, s2), "direct visibility");
            DirectAccumArgs da{};
            memcpy(da.s, c->s, 12);
            da.mics = ptr<float>(c->mics);
            da.M = M;
            da.F = F;
            da.vis = ptr<uint8_t>(c->dvis);
            da.f_lo = c->f_lo;
            da.df = T.df;
            da.c = p.c;
            da.a0 = p.alpha0_db_m;
            da.a1 = p.alpha1_db_m_khz;
            da.gain = p.direct_gain;
            da.etab = c->n_theta > 0 ? ptr<float>(c->etab) : nullptr;
            da.n_theta = c->n_theta;
            memcpy(da.fwd, fwd, 12);
            da.mic_tab = c->mic_nb > 0 ? ptr<float>(c->mic_tab) : nullptr;
            da.mic_q = (c->mic_nb > 0 && c->has_mic_q) ? ptr<float>(c->mic_q) : nullptr;
            da.n_el = c->n_el;
            da.n_az = c->n_az;
            da.n_bands = S.n_bands;
            da.bw = ptr<float2>(T.bw);
            da.out = out + 2 * MF;
            CKC(c, accumulate_direct(da, ptr<float>(T.qhi), ptr<float>(T.qlo), s2), "direct");
        } else {
            CKC(c, cudaMemsetAsync(c->dvis.p, 0, (size_t)M, s2), "memset");
        }
        return ST_OK;
    };

    if (overlap) {  // side stream: diffraction, its accumulation, the direct path; context stream: the trace
        st_status r = stage_diffraction();
        if (r == ST_OK) r = stage_diffraction_accumulation();
        if (r == ST_OK) r = stage_direct();
        if (r == ST_OK) r = stage_trace();
        if (r == ST_OK && stats) r = cudaEventRecord(c->ev[1], s) == cudaSuccess ? ST_OK : fail(c, ST_ERR_CUDA, "event");
        if (r == ST_OK) r = stage_specular();
        if (r == ST_OK && !joined) {
            CKC(c, cudaEventRecord(c->ev_join, s2), "join");
            CKC(c, cudaStreamWaitEvent(s, c->ev_join, 0), "join");
            joined = true;
        }
        if (r != ST_OK) return r;
    } else {
        st_status r = stage_trace();
        if (r == ST_OK && stats) r = cudaEventRecord(c->ev[1], s) == cudaSuccess ? ST_OK : fail(c, ST_ERR_CUDA, "event");
        if (r == ST_OK) r = stage_diffraction();
        if (r == ST_OK) r = stage_specular();
        if (r == ST_OK) r = stage_diffraction_accumulation();
        if (r == ST_OK) r = stage_direct();
        if (r != ST_OK) return r;
    }
    if (stats) CKC(c, cudaEventRecord(c->ev[3], s), "event");

    c->last_N = N;
    c->last_B = B;
    c->last_K = K;
    c->last_M = M;
    c->last_F = F;
    c->last_params = p;
    c->last_scene = sc;
    c->last_scene_version = sc->version;
    c->last_chunks_spec = chunks_spec;
    c->last_fwd[0] = fwd[0];
    c->last_fwd[1] = fwd[1];
    c->last_fwd[2] = fwd[2];
    c->last_chunks_diff = chunks_diff;
    c->last_diff_mma = diff_mma;
    c->has_last = true;
    c->paths_chain_order = false;

    // device-side error flags are checked whenever the caller synchronises through stats
    if (stats) {
        uint32_t h[4] = {0, 0, 0, 0}, fl = 0;
        unsigned long long hq[7] = {0, 0, 0, 0, 0, 0, 0};
        CKC(c, cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, s), "stats");
        CKC(c, cudaMemcpyAsync(hq, qctr, 56, cudaMemcpyDeviceToHost, s), "stats");
        CKC(c, cudaMemcpyAsync(&fl, c->flags.p, 4, cudaMemcpyDeviceToHost, s), "stats");
        CKC(c, cudaStreamSynchronize(s), "stats sync");
        memset(stats, 0, sizeof(*stats));
        stats->rays = N;
        stats->closest_queries = (int64_t)hq[0];
        stats->shadow_queries = (int64_t)hq[1];
        for (int k = 0; k < 4; ++k) stats->visits[k] = (int64_t)hq[2 + k];
        stats->stack_restarts = (int64_t)hq[6];
        stats->records = 0;
        stats->visible_records = h[2];
        stats->candidates = K;
        stats->candidates_kept = h[3];
        float ms;
        // with the stage overlap the diffraction stage runs beside the trace, and the accumulation stage (from
        // the end of the trace) includes the wait for the side stream
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        stats->ms_trace = ms;
        stats->ms_diffraction = 0.0f;
        if (K > 0) {
            cudaEventElapsedTime(&ms, c->ev[8], c->ev[9]);
            stats->ms_diffraction = ms;
        }
        cudaEventElapsedTime(&ms, (K > 0 && !overlap) ? c->ev[9] : c->ev[1], c->ev[3]);
        stats->ms_accumulate = ms;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[3]);
        stats->ms_total = ms;
        stats->kernel_launches = launch_count() - launches0;
        stats->ms_accum_kernel = 0.0f;
        stats->accum_launches = 0;
        if (n_accum & 1) {
            cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]);
            stats->ms_accum_kernel += ms;
            stats->ms_accum_specular = ms;
            stats->accum_launches++;
        }
        if (n_accum & 2) {
            cudaEventElapsedTime(&ms, c->ev[6], c->ev[7]);
            stats->ms_accum_kernel += ms;
            stats->ms_accum_diffraction = ms;
            stats->accum_launches++;
        }
        stats->terms_specular = (int64_t)((n_accum & 1) ? h[2] : 0) * M * F;
        stats->terms_diffraction = (int64_t)((n_accum & 2) ? h[3] : 0) * M * F;
        stats->terms = stats->terms_specular + stats->terms_diffraction;
        stats->diffraction_tensor = diff_mma ? 1 : 0;
        if (fl & kFlagBadTree) return fail(c, ST_ERR_CUDA, "malformed BVH: traversal exceeded the node count");
        if (fl & kFlagCheck) return fail(c, ST_ERR_CUDA, "a bounds check of the checked build failed");
    }
#ifdef ST_CHECKS
    {  // the checked build reads the flags after every simulate
        uint32_t fl = 0;
        CKC(c, cudaMemcpyAsync(&fl, c->flags.p, 4, cudaMemcpyDeviceToHost, s), "checks");
        CKC(c, cudaStreamSynchronize(s), "checks sync");
        if (fl & kFlagCheck) return fail(c, ST_ERR_CUDA, "a bounds check of the checked build failed");
    }
#endif
    return ST_OK;
}

st_status st_simulate_host(st_ctx* c, st_scene* sc, const st_sim_params* params, void* spectra_out, st_stats* stats) {
    if (!c || !spectra_out) return fail(c, ST_ERR_ARG, "simulate_host: null argument");
    enter(c);
    const size_t bytes = (size_t)3 * c->M * c->F * 8;
    CKC(c, grow(c->host_out, bytes), "alloc");
    st_status r = st_simulate(c, sc, params, c->host_out.p, stats);
    if (r != ST_OK) return r;
    CKC(c, cudaMemcpyAsync(spectra_out, c->host_out.p, bytes, cudaMemcpyDeviceToHost, c->stream), "copy out");
    CKC(c, cudaStreamSynchronize(c->stream), "sync");
    return ST_OK;
}

st_status st_get_paths(st_ctx* c, int32_t* tri, float* point, float* dir, double* r, uint8_t* los, int32_t mem) {
    if (!c) return ST_ERR_ARG;
    if (!c->has_last) return fail(c, ST_ERR_STATE, "get_paths: no simulate yet");
    enter(c);
    const size_t nb = (size_t)c->last_N * c->last_B;
    if (nb == 0) return ST_OK;  // no emitter rays: nothing to copy
    if (tri) CKC(c, cudaMemcpyAsync(tri, c->rec_tri.p, nb * 4, kind_out(mem), c->stream), "get_paths");
    if (point) CKC(c, cudaMemcpyAsync(point, c->rec_p.p, nb * 12, kind_out(mem), c->stream), "get_paths");
    if (dir) CKC(c, cudaMemcpyAsync(dir, c->rec_d.p, nb * 12, kind_out(mem), c->stream), "get_paths");
    if (r) CKC(c, cudaMemcpyAsync(r, c->rec_r.p, nb * 8, kind_out(mem), c->stream), "get_paths");
    if (los) CKC(c, cudaMemcpyAsync(los, c->rec_los.p, nb, kind_out(mem), c->stream), "get_paths");
    CKC(c, cudaStreamSynchronize(c->stream), "get_paths sync");
    return ST_OK;
}

st_status st_get_receiver_masks(st_ctx* c, uint64_t* mask, int32_t mem) {
    if (!c || !mask) return ST_ERR_ARG;
    if (!c->has_last || c->last_params.los_mode != ST_LOS_PER_MIC)
        return fail(c, ST_ERR_STATE, "get_receiver_masks: the last simulate made no per-microphone receiver test");
    enter(c);
    const size_t nb = (size_t)c->last_N * c->last_B;
    if (nb == 0) return ST_OK;
    CKC(c, cudaMemcpyAsync(mask, c->rec_mask.p, nb * 8, kind_out(mem), c->stream), "get_receiver_masks");
    CKC(c, cudaStreamSynchronize(c->stream), "get_receiver_masks sync");
    return ST_OK;
}

st_status st_get_diffraction(st_ctx* c, int64_t* n_out, int32_t* tri, float* point, uint8_t* keep, int64_t capacity,
                             int32_t mem) {
    if (!c || !n_out) return ST_ERR_ARG;
    if (!c->has_last) return fail(c, ST_ERR_STATE, "get_diffraction: no simulate yet");
    *n_out = c->last_K;
    const int64_t n = std::min(capacity, c->last_K);
    enter(c);
    if (n > 0) {
        if (tri) CKC(c, cudaMemcpyAsync(tri, c->cand_tri.p, (size_t)n * 4, kind_out(mem), c->stream), "get_diffraction");
        if (point) CKC(c, cudaMemcpyAsync(point, c->cand_p.p, (size_t)n * 12, kind_out(mem), c->stream), "get_diffraction");
        if (keep) CKC(c, cudaMemcpyAsync(keep, c->keep.p, (size_t)n, kind_out(mem), c->stream), "get_diffraction");
    }
    CKC(c, cudaStreamSynchronize(c->stream), "get_diffraction sync");
    return ST_OK;
}

st_status st_get_direct_visibility(st_ctx* c, uint8_t* vis, int32_t mem) {
    if (!c || !vis) return ST_ERR_ARG;
    if (!c->has_last) return fail(c, ST_ERR_STATE, "get_direct_visibility: no simulate yet");
    enter(c);
    CKC(c, cudaMemcpyAsync(vis, c->dvis.p, (size_t)c->last_M, kind_out(mem), c->stream), "get_direct_visibility");
    CKC(c, cudaStreamSynchronize(c->stream), "sync");
    return ST_OK;
}

static st_status backward_impl(st_ctx* c, st_scene* sc, const void* grad_spectra, float* grad_k, float* grad_mic,
                               float* grad_emitter, float* grad_beta) {
    if (!c || !sc || !grad_spectra) return fail(c, ST_ERR_ARG, "backward: null argument");
    if (!c->has_last || c->last_scene != sc || c->last_scene_version != sc->version)
        return fail(c, ST_ERR_STATE, "backward: needs the last simulate of this scene, unchanged since");
    if ((grad_mic || grad_emitter) && c->n_theta > 0)
        return fail(c, ST_ERR_ARG, "backward: position gradients need an omni emitter");
    if (c->mic_nb > 0) return fail(c, ST_ERR_ARG, "backward: needs omni receivers");
    enter(c);
    cudaStream_t s = c->stream;
    const st_sim_params& p = c->last_params;
    SceneDev& S = sc->S;
    AccumTables& T = c->tables;
    const int32_t M = c->last_M, F = c->last_F;
    const int64_t MF = (int64_t)M * F;
    const float2* G = static_cast<const float2*>(grad_spectra);
    const bool want_pos = grad_mic || grad_emitter;
    uint32_t* cnt = ptr<uint32_t>(c->counts);
    // per-microphone receiver test: the specular path list carries each path's microphone mask (the
    // producers give a microphone that does not see the path a zero anchor, so its terms add nothing)
    const uint64_t* spec_mask = p.los_mode == ST_LOS_PER_MIC ? ptr<uint64_t>(c->paths.mask) : nullptr;

    const double l10 = log(10.0) / 20.0;
    AccumArgs aa{};
    aa.mics = ptr<float>(c->mics);
    aa.M = M;
    aa.F = F;
    aa.lk = ptr<float>(T.lk);
    aa.g2 = ptr<float>(T.g2);
    aa.lid = ptr<float>(T.lid);
    aa.n_mat_tab = T.n_mat;
    aa.n_bands_tab = S.n_bands;
    aa.bw = ptr<float2>(T.bw);
    aa.qhi = ptr<float>(T.qhi);
    aa.qlo = ptr<float>(T.qlo);
    {
        const double dq = T.df / p.c;
        aa.dq_hi = (float)dq;
        aa.dq_lo = (float)(dq - (double)aa.dq_hi);
        const double l2 = log2(10.0) / 20.0;
        aa.atm2_0 = (float)(-(p.alpha0_db_m + p.alpha1_db_m_khz * c->f_lo / 1000.0) * l2);
        aa.atm2_step = (float)(-(p.alpha1_db_m_khz * T.df / 1000.0) * l2);
    }
    aa.etab = c->n_theta > 0 ? ptr<float>(c->etab) : nullptr;
    aa.n_theta = c->n_theta;
    aa.reflection_mode = p.reflection_mode;
    AdjointArgs ja{};
    memcpy(ja.s, c->s, 12);
    ja.a_0 = (float)((p.alpha0_db_m + p.alpha1_db_m_khz * c->f_lo / 1000.0) * l10);
    ja.a_step = (float)(p.alpha1_db_m_khz * T.df / 1000.0 * l10);
    ja.w_0 = (float)(2.0 * M_PI * c->f_lo / p.c);
    ja.w_step = (float)(2.0 * M_PI * T.df / p.c);

    // microphone pairs per CTA of the specular and diffraction adjoints (ST_ADJ_TP="spec,diff" overrides); the
    // diffraction adjoint takes 16 bins per thread and 8 pairs, so that a CTA covers 512 bins and forms each
    // (path, microphone) anchor once on such grids
    int adj_tp[2] = {16, 8};
    if (const char* e = getenv("ST_ADJ_TP")) {
        int u = 0, v = 0;
        if (sscanf(e, "%d,%d", &u, &v) == 2 && u >= 1 && u <= 16 && v >= 1 && v <= 16) {
            adj_tp[0] = u;
            adj_tp[1] = v;
        }
    }
    const acc::Geom g = adjoint_geom(M, F, T.n_mat, 0, adj_tp[0]);
    // same tile shape for the diffraction paths; without an emitter table their per-(material, bin) factor is
    // read from the material table, so tiles hold more paths
    const acc::Geom gd = adjoint_geom(M, F, T.n_mat, aa.etab ? 0 : 1, adj_tp[1], 16);
    // chunking from the path lists' capacities (the counts stay on the device: no synchronisation), per path
    // kind: two CTAs per SM over the kind's own tile grid
    auto chunks_for = [](const acc::Geom& gg, int64_t n_paths) {
        const int ctas_ = std::max(gg.n_mb * gg.n_bb, 1);
        const int64_t tiles = std::max<int64_t>(1, (n_paths + gg.PT - 1) / gg.PT);
        return (int32_t)std::max<int64_t>(1, std::min<int64_t>(std::max(152 * 2 / ctas_, 1), (tiles + 7) / 8));
    };
    const int32_t chunks = chunks_for(g, c->last_N * c->last_B);
    // diffraction on the tensor cores when the forward put its paths in material order
    const bool diff_mma = c->last_diff_mma && c->last_K > 0;
    int32_t dm_mb = 0, dm_bb = 0;
    adjoint_diffraction_mma_shape(M, F, &dm_mb, &dm_bb);
    const int32_t chunks_d = diff_mma ? diffraction_mma_chunks(c->last_K, M, F, T.n_mat) : chunks_for(gd, c->last_K);
    const int ctas = g.n_mb * g.n_bb;
    const int spec_mic_slices = chunks * g.n_bb, spec_emit_slices = chunks * ctas;
    const int diff_mic_slices = chunks_d * (diff_mma ? dm_bb : gd.n_bb);
    const int diff_emit_slices = chunks_d * (diff_mma ? dm_mb * dm_bb : gd.n_mb * gd.n_bb);
    const int mic_slices = spec_mic_slices + diff_mic_slices + 1;     // specular, diffraction, direct
    const int emit_slices = spec_emit_slices + diff_emit_slices + M;  // direct: one slice per microphone
    CKC(c, grow(c->adj_v, (size_t)chunks * g.n_mb * 4 * F * 4), "alloc");
    CKC(c, grow(c->adj_mic, (size_t)mic_slices * M * 3 * 4), "alloc");
    CKC(c, grow(c->adj_emit, (size_t)emit_slices * 3 * 4), "alloc");
    CKC(c, cudaMemsetAsync(c->adj_mic.p, 0, (size_t)mic_slices * M * 3 * 4, s), "memset");
    CKC(c, cudaMemsetAsync(c->adj_emit.p, 0, (size_t)emit_slices * 3 * 4, s), "memset");
    float* micp = ptr<float>(c->adj_mic);
    float* emitp = ptr<float>(c->adj_emit);
    if (grad_k) CKC(c, cudaMemsetAsync(grad_k, 0, (size_t)S.n_mat * S.n_bands * 4, s), "memset");
    if (grad_beta) CKC(c, cudaMemsetAsync(grad_beta, 0, (size_t)S.n_mat * S.n_bands * 4, s), "memset");

    auto set_paths = [&](AccumArgs& x, PathList& PL) {
        x.px = ptr<float>(PL.px);
        x.py = ptr<float>(PL.py);
        x.pz = ptr<float>(PL.pz);
        x.dx = ptr<float>(PL.dx);
        x.dy = ptr<float>(PL.dy);
        x.dz = ptr<float>(PL.dz);
        x.rhi = ptr<float>(PL.rhi);
        x.rlo = ptr<float>(PL.rlo);
        x.chain_lo = ptr<uint32_t>(PL.chain_lo);
        x.chain_hi = ptr<uint32_t>(PL.chain_hi);
        x.meta = ptr<uint32_t>(PL.meta);
        x.dep = ptr<float>(PL.dep);
    };
    // The diffraction and direct-path adjoints (positions) share nothing with the specular part but G and the
    // zeroed gradient slices, each writing its own: with the stage overlap they run on the context's side
    // stream beside the specular part's preparation and adjoint, joined before the position sums.
    const bool side_pos = c->overlap && c->side && want_pos &&
                          (c->last_K > 0 || (p.components & ST_COMP_DIRECT)) &&
                          (p.components & ST_COMP_SPECULAR) && c->last_N > 0;
    cudaStream_t s2 = s;
    bool joined = false;
    if (side_pos) {
        CKC(c, cudaEventRecord(c->ev_fork, s), "fork");
        CKC(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork");
        s2 = c->side;
    }
    struct JoinGuard {
        st_ctx* c;
        cudaStream_t s;
        const bool& active;
        const bool& done;
        ~JoinGuard() {
            if (active && !done) {
                cudaEventRecord(c->ev_join, c->side);
                cudaStreamWaitEvent(s, c->ev_join, 0);
            }
        }
    } join_guard{c, s, side_pos, joined};
    auto positions_beside = [&]() -> st_status {
        // ---- diffraction: positions
        if (want_pos && c->last_K > 0) {
            AccumArgs x = aa;
            x.kind = 1;
            x.d_count = cnt + 3;
            x.n_chunks = chunks_d;
            set_paths(x, c->paths_diff);
            AdjointArgs jj = ja;
            jj.G = G + MF;
            jj.do_pos = 1;
            jj.do_k = 0;
            jj.v_part = ptr<float>(c->adj_v);
            jj.mic_part = micp + (size_t)spec_mic_slices * M * 3;
            jj.emit_part = emitp + (size_t)spec_emit_slices * 3;
            if (diff_mma)
                CKC(c, adjoint_diffraction_mma(x, jj, ptr<uint32_t>(c->mat_off), s2), "adjoint diffraction");
            else
                CKC(c, adjoint_launch(x, jj, gd, s2), "adjoint diffraction");
        }
        // ---- direct path
        if (want_pos && (p.components & ST_COMP_DIRECT)) {
            DirectAccumArgs da{};
            memcpy(da.s, c->s, 12);
            da.mics = ptr<float>(c->mics);
            da.M = M;
            da.F = F;
            da.vis = ptr<uint8_t>(c->dvis);
            da.f_lo = c->f_lo;
            da.df = T.df;
            da.c = p.c;
            da.a0 = p.alpha0_db_m;
            da.a1 = p.alpha1_db_m_khz;
            da.gain = p.direct_gain;
            CKC(c, adjoint_direct(da, ptr<float>(T.qhi), ptr<float>(T.qlo), G + 2 * MF,
                                  micp + (size_t)(spec_mic_slices + diff_mic_slices) * M * 3,
                                  emitp + (size_t)(spec_emit_slices + diff_emit_slices) * 3, s2),
                "adjoint direct");
        }
        return ST_OK;
    };
    if (side_pos) {
        const st_status r = positions_beside();
        if (r != ST_OK) return r;
    }
    // ---- specular: reflection sums in batches of four materials, positions with the first batch
    if ((p.components & ST_COMP_SPECULAR) && c->last_N > 0 && (grad_k || want_pos)) {
        AccumArgs x = aa;
        x.kind = 0;
        x.d_count = cnt + 2;
        x.n_chunks = chunks;
        set_paths(x, c->paths);
        x.mask = spec_mask;
        const int64_t NB = c->last_N * c->last_B;
        if (!c->paths_chain_order || grad_emitter) {
            // the compaction of the last simulate, repeated: the visible records in the order of its path list
            CKC(c, flags_visible_records(ptr<int32_t>(c->rec_tri), ptr<uint8_t>(c->rec_los), NB,
                                         ptr<uint32_t>(c->sflags), s),
                "flags");
            CKC(c, exclusive_scan_u32(ptr<uint32_t>(c->sflags), ptr<uint32_t>(c->sscan), NB, cnt + 2, c->scratch.p, s),
                "scan");
            CKC(c, compact_indices(ptr<uint32_t>(c->sflags), ptr<uint32_t>(c->sscan), NB, ptr<uint32_t>(c->sidx), s),
                "compact");
        }
        if (c->n_theta == 0 && NB > 1) {
            // chain order (omni emitter; with an emitter table the list keeps its table-row order): paths with
            // equal material counts next to each other, so that the adjoint reduces their reflection sums once
            // per run; the path list is gathered again in that order (once per simulate) and the chain
            // jacobians follow it
            GatherArgs ga{};
            ga.N = c->last_N;
            ga.B = c->last_B;
            ga.rec_tri = ptr<int32_t>(c->rec_tri);
            ga.rec_p = ptr<float>(c->rec_p);
            ga.rec_d = ptr<float>(c->rec_d);
            ga.rec_r = ptr<double>(c->rec_r);
            ga.rec_los = ptr<uint8_t>(c->rec_los);
            ga.tri_mat = ptr<int32_t>(S.tri_mat);
            ga.dirs = ptr<float>(c->dirs);
            memcpy(ga.q, c->q, 16);
            memcpy(ga.fwd, c->last_fwd, 12);
            ga.has_etab = false;
            ga.idx = ptr<uint32_t>(c->sidx);
            ga.count = cnt + 2;
            ga.out = &c->paths;
            ga.rec_mask = spec_mask ? ptr<uint64_t>(c->rec_mask) : nullptr;
            ga.n_mat = S.n_mat;
            ga.chk = ptr<uint32_t>(c->flags);
            if (!c->paths_chain_order || grad_emitter) {  // (the sort is stable: the same order every time)
                CKC(c, grow(c->ck_keys, (size_t)NB * 8), "alloc");
                CKC(c, grow(c->ck_scr, sort_scratch_bytes(NB)), "alloc");
                CKC(c, chain_order(ga, NB, p.reflection_mode == 1 ? 1 : 0, ptr<uint32_t>(c->sidx),
                                   ptr<uint64_t>(c->ck_keys), c->ck_scr.p, s),
                    "chain order");
            }
            if (!c->paths_chain_order) CKC(c, gather_specular(ga, s), "gather");
            c->paths_chain_order = true;
        }
        if (grad_emitter) {
            // the emitter moves the hit points: chain jacobians of the visible records, in the order of
            // the path list
            CKC(c, grow(c->adj_jac, (size_t)NB * 48), "alloc");
            CKC(c, chain_jacobians(ptr<uint32_t>(c->sidx), cnt + 2, NB, c->last_B, ptr<int32_t>(c->rec_tri),
                                   ptr<float>(c->rec_d), ptr<float>(S.nrm), ptr<float>(c->dirs), c->q,
                                   ptr<float>(c->adj_jac), s),
                "chain jacobians");
            x.jac = ptr<float>(c->adj_jac);
        }
        const int n_batches = grad_k ? (S.n_mat + 3) / 4 : 1;
        for (int bt = 0; bt < n_batches; ++bt) {
            AdjointArgs jj = ja;
            jj.G = G;
            jj.do_pos = (bt == 0 && want_pos) ? 1 : 0;
            jj.do_k = grad_k ? 1 : 0;
            jj.mat_base = 4 * bt;
            jj.v_part = ptr<float>(c->adj_v);
            jj.mic_part = micp;
            jj.emit_part = emitp;
            CKC(c, adjoint_launch(x, jj, g, s), "adjoint specular");
            if (grad_k)
                CKC(c, adjoint_dk(ptr<float>(c->adj_v), chunks * g.n_mb, F, 4 * bt, std::min(4, S.n_mat - 4 * bt),
                                  S.n_bands, ptr<float>(T.band), ptr<float>(T.kband), c->f_lo, T.df, grad_k, S.n_mat,
                                  s),
                    "adjoint dk");
        }
    }
    // ---- specular: lobe-width sums (the last hit's material), in batches of four materials
    if ((p.components & ST_COMP_SPECULAR) && c->last_N > 0 && grad_beta) {
        AccumArgs x = aa;
        x.kind = 0;
        x.d_count = cnt + 2;
        x.n_chunks = chunks;
        set_paths(x, c->paths);
        x.mask = spec_mask;
        for (int bt = 0; bt < (S.n_mat + 3) / 4; ++bt) {
            AdjointArgs jj = ja;
            jj.G = G;
            jj.do_pos = 0;
            jj.do_k = 1;
            jj.do_beta = 1;
            jj.mat_base = 4 * bt;
            jj.v_part = ptr<float>(c->adj_v);
            jj.mic_part = micp;
            jj.emit_part = emitp;
            CKC(c, adjoint_launch(x, jj, g, s), "adjoint lobe widths");
            CKC(c, adjoint_dbeta(ptr<float>(c->adj_v), chunks * g.n_mb, F, 4 * bt, std::min(4, S.n_mat - 4 * bt),
                                 S.n_bands, ptr<float>(T.band), ptr<float>(T.bband), c->f_lo, T.df, grad_beta, s),
                "adjoint dbeta");
        }
    }
    if (!side_pos) {
        const st_status r = positions_beside();
        if (r != ST_OK) return r;
    } else {
        CKC(c, cudaEventRecord(c->ev_join, s2), "join");
        CKC(c, cudaStreamWaitEvent(s, c->ev_join, 0), "join");
        joined = true;
    }
    if (want_pos)
        CKC(c, adjoint_pos(micp, mic_slices, emitp, emit_slices, M, grad_mic, grad_emitter, s), "adjoint reduce");
    return ST_OK;
}

st_status st_ray_directions(st_ctx* c, int32_t kind, int64_t n, float* out) {
    if (!c || !out || n < 1 || (kind != ST_RAYS_FIBONACCI && kind != ST_RAYS_ZONAL) || n >= ((int64_t)1 << 40))
        return fail(c, ST_ERR_ARG, "ray_directions: null output, n < 1 or unknown kind");
    enter(c);
    CKC(c, ray_directions(kind, n, out, c->ray_tab, c->stream), "ray directions");
    return ST_OK;
}

st_status st_impulse_response(st_ctx* c, const void* spectra, int32_t n_comp, int32_t n_mics, int32_t n_bins,
                              double f_lo, double f_hi, double fs, int32_t n_samples, const float* window,
                              const float* call, int32_t call_len, int32_t flags, float* out) {
    if (!c || !spectra || !out) return fail(c, ST_ERR_ARG, "impulse_response: null pointer");
    if (n_comp < 1 || n_comp > 3 || n_mics < 1 || n_bins < 1 || n_samples < 1 || !(fs > 0.0) || !(f_hi >= f_lo) ||
        call_len < 0 || (call_len > 0 && !call) || (n_bins > 1 && !(f_hi > f_lo)))
        return fail(c, ST_ERR_ARG, "impulse_response: bad sizes or grid");
    enter(c);
    const int per_comp = (flags & ST_IR_PER_COMPONENT) ? 1 : 0;
    const int64_t rows = per_comp ? (int64_t)n_comp * n_mics : n_mics;
    if (rows > 65535) return fail(c, ST_ERR_ARG, "impulse_response: more than 65535 output rows");
    CKC(c, grow(c->sig_e, (size_t)n_bins * 8), "alloc");
    CKC(c, grow(c->sig_g, (size_t)rows * n_bins * 8), "alloc");
    CKC(c, signal_response(static_cast<const float2*>(spectra), n_comp, n_mics, n_bins, f_lo, f_hi, fs, n_samples,
                           window, call_len > 0 ? call : nullptr, call_len, per_comp, ptr<float2>(c->sig_e),
                           ptr<float2>(c->sig_g), out, c->stream),
        "impulse response");
    return ST_OK;
}

st_status st_backward(st_ctx* c, st_scene* sc, const void* grad_spectra, float* grad_k, float* grad_mic,
                      float* grad_emitter) {
    NvtxRange range("st_backward");
    const st_status r = backward_impl(c, sc, grad_spectra, grad_k, grad_mic, grad_emitter, nullptr);
    if (r == ST_OK)
        st_log(2, "backward: %s%s%s", grad_k ? "reflection " : "", grad_mic ? "microphones " : "",
               grad_emitter ? "emitter" : "");
    return r;
}

st_status st_backward_beta(st_ctx* c, st_scene* sc, const void* grad_spectra, float* grad_beta) {
    if (!grad_beta) return fail(c, ST_ERR_ARG, "backward_beta: null output");
    NvtxRange range("st_backward_beta");
    return backward_impl(c, sc, grad_spectra, nullptr, nullptr, nullptr, grad_beta);
}

}  // extern "C"

// ------------------------------------------------------------------ batched form
namespace {

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

bool tune_ok(const st_tune& t) {
    return (t.rays_per_block == 0 || t.rays_per_block == 64 || t.rays_per_block == 128 || t.rays_per_block == 256) &&
           (t.mic_pairs_per_cta == 0 || (t.mic_pairs_per_cta >= 1 && t.mic_pairs_per_cta <= 16)) &&
           (t.smem_kb == 0 || (t.smem_kb >= 32 && t.smem_kb <= 160)) && t.stack_depth >= 0 && t.stack_depth <= kStack &&
           t.refill_lanes >= 0 && t.refill_lanes <= 32 &&
           (t.bins_per_thread == 0 || t.bins_per_thread == 8 || t.bins_per_thread == 16);
}

void batch_free_graph(BatchState& B) {
    if (B.exec) cudaGraphExecDestroy(B.exec);
    if (B.graph) cudaGraphDestroy(B.graph);
    B.exec = nullptr;
    B.graph = nullptr;
}

void batch_release(BatchState& B) {
    batch_free_graph(B);
    for (DevBuf* b : {&B.jobs_dev, &B.offs, &B.derived, &B.perm, &B.ord_keys, &B.ord_scr, &B.st_o[0], &B.st_o[1],
                      &B.st_o[2], &B.st_d[0], &B.st_d[1], &B.st_d[2], &B.st_r, &B.st_prev, &B.q0, &B.q1, &B.counts,
                      &B.queries, &B.flags, &B.rec_tri, &B.rec_p, &B.rec_d, &B.rec_r, &B.rec_los, &B.cand_tri,
                      &B.cand_p, &B.keep, &B.dvis, &B.ranges, &B.sflags, &B.sscan, &B.sidx, &B.scratch, &B.hit_tri,
                      &B.hit_t, &B.vis_q, &B.los_q, &B.rec_mask, &B.vis_qm})
        release(*b);
    release(B.narrow_partial);
    for (DevBuf* d : {&B.tasks, &B.part_all, &B.qctr, &B.mat_off, &B.mat_scr}) release(*d);
    for (auto& T : B.tables)
        for (DevBuf* b : {&T.lk, &T.g2, &T.lid, &T.qhi, &T.qlo, &T.bw, &T.band, &T.kband, &T.bband}) release(*b);
    for (PathList* P : {&B.spec, &B.diff})
        for (DevBuf* b : {&P->px, &P->py, &P->pz, &P->dx, &P->dy, &P->dz, &P->rhi, &P->rlo, &P->chain_lo, &P->chain_hi,
                          &P->meta, &P->dep, &P->mask})
            release(*b);
    for (auto ev : B.events) cudaEventDestroy(ev);
    if (B.main) cudaStreamDestroy(B.main);
    B.main = nullptr;
    B.events.clear();
    release(B.dscratch);
    for (int k = 0; k < 4; ++k) {
        if (B.branch[k]) cudaStreamDestroy(B.branch[k]);
        if (B.br_join[k]) cudaEventDestroy(B.br_join[k]);
        B.branch[k] = nullptr;
        B.br_join[k] = nullptr;
    }
    if (B.br_fork) cudaEventDestroy(B.br_fork);
    B.br_fork = nullptr;
    if (B.ev_fork) cudaEventDestroy(B.ev_fork);
    if (B.ev_join) cudaEventDestroy(B.ev_join);
    if (B.side) cudaStreamDestroy(B.side);
    B.ev_fork = B.ev_join = nullptr;
    B.side = nullptr;
}

// Jobs accumulated one after the other by the single-pose path's launch (not through the work queue): one
// microphone pair (the narrow accumulator is several times faster for them), receiver directivity tables
// (the tile's per-microphone band tables), and jobs of a million paths or more, which fill the GPU alone
// with their full chunk count (in the queue they would take a fraction of it).
static bool big_job(const JobDev& d) { return d.N * (int64_t)d.B >= (1 << 20) || d.K >= (1 << 20); }
static bool solo_accum(const JobDev& d) { return narrow_accum(d.M) || d.mic_tab != nullptr || big_job(d); }

// All stages of one batch on stream s.
// Accumulation arguments of job j's path kind (0 specular, 1 diffraction) in the batch's path lists.
AccumArgs batch_accum_args(BatchState& B, const st_job* jobs, int j, int kind, const st_sim_params& p,
                           const st_tune& tn) {
    const JobDev& jd = B.jobs[j];
    AccumTables& T = B.tables[j];
    SceneDev& S = jobs[j].scene->S;
    const double l2 = log2(10.0) / 20.0;
    AccumArgs x{};
    x.mics = jobs[j].mics;
    x.M = jd.M;
    x.F = jd.F;
    x.lk = ptr<float>(T.lk);
    x.g2 = ptr<float>(T.g2);
    x.lid = ptr<float>(T.lid);
    x.n_mat_tab = T.n_mat;
    x.n_bands_tab = S.n_bands;
    x.bw = ptr<float2>(T.bw);
    x.qhi = ptr<float>(T.qhi);
    x.qlo = ptr<float>(T.qlo);
    const double dq = T.df / p.c;
    x.dq_hi = (float)dq;
    x.dq_lo = (float)(dq - (double)x.dq_hi);
    x.atm2_0 = (float)(-(p.alpha0_db_m + p.alpha1_db_m_khz * jobs[j].f_lo / 1000.0) * l2);
    x.atm2_step = (float)(-(p.alpha1_db_m_khz * T.df / 1000.0) * l2);
    x.reflection_mode = p.reflection_mode;
    x.tile_tp = tn.mic_pairs_per_cta;
    x.tile_kb = tn.smem_kb;
    x.kind = kind;
    x.etab = jd.etab;
    x.n_theta = jd.n_theta;
    x.mic_tab = jd.mic_tab;
    x.mic_q = jd.mic_q;
    x.n_el = jd.n_el;
    x.n_az = jd.n_az;
    uint32_t* rg = ptr<uint32_t>(B.ranges) + 4 * j;
    PathList& L = kind == 0 ? B.spec : B.diff;
    x.n_paths = kind == 0 ? jd.N * jd.B : jd.K;
    x.d_base = rg + (kind == 0 ? 0 : 2);
    x.d_count = rg + (kind == 0 ? 1 : 3);
    x.px = ptr<float>(L.px);
    x.py = ptr<float>(L.py);
    x.pz = ptr<float>(L.pz);
    x.dx = ptr<float>(L.dx);
    x.dy = ptr<float>(L.dy);
    x.dz = ptr<float>(L.dz);
    x.rhi = ptr<float>(L.rhi);
    x.rlo = ptr<float>(L.rlo);
    x.chain_lo = ptr<uint32_t>(L.chain_lo);
    x.chain_hi = ptr<uint32_t>(L.chain_hi);
    x.meta = ptr<uint32_t>(L.meta);
    x.dep = ptr<float>(L.dep);
    x.mask = (kind == 0 && B.per_mic) ? ptr<uint64_t>(B.spec.mask) : nullptr;  // indexed from x.d_base
    x.n_chunks = kind == 0 ? B.chunks_spec[j] : B.chunks_diff[j];
    return x;
}

// The persistent accumulation's task table: per job its specular task (rays) and its diffraction task
// (samples), each with its chunk partials in one buffer; items and outputs numbered in table order.
cudaError_t batch_tasks(st_ctx* c, BatchState& B, const st_job* jobs, const st_sim_params& p, const st_tune& tn,
                        cudaStream_t s) {
    (void)c;
    std::vector<AccumTask> spec, diff, mma;
    B.narrow_jobs.clear();
    for (int j = 0; j < B.n_jobs; ++j) {
        const JobDev& jd = B.jobs[j];
        if (solo_accum(jd)) {  // the single-pose path's accumulator for this shape (same sums)
            B.narrow_jobs.push_back(j);
            continue;
        }
        float2* out = static_cast<float2*>(jobs[j].spectra_out);
        const int64_t MF = (int64_t)jd.M * jd.F;
        if (jd.N > 0) {
            AccumTask t{};
            accum_task(batch_accum_args(B, jobs, j, 0, p, tn), out, &t);
            spec.push_back(t);
        }
        if (jd.K > 0 && jd.diff_mma) {
            AccumTask t{};
            diffraction_mma_task(batch_accum_args(B, jobs, j, 1, p, tn), ptr<uint32_t>(B.mat_off) + (size_t)j * kMatStride,
                                 out + MF, &t);
            mma.push_back(t);
        } else if (jd.K > 0) {
            AccumTask t{};
            accum_task(batch_accum_args(B, jobs, j, 1, p, tn), out + MF, &t);
            diff.push_back(t);
        }
    }
    B.n_tasks_spec = (int32_t)spec.size();
    B.n_tasks_diff = (int32_t)diff.size();
    B.n_tasks_mma = (int32_t)mma.size();
    std::vector<AccumTask> all(spec);
    all.insert(all.end(), diff.begin(), diff.end());
    all.insert(all.end(), mma.begin(), mma.end());
    size_t part = 0;
    int64_t out0 = 0;
    B.items_spec = B.items_diff = B.items_mma = 0;
    B.smem_spec = B.smem_diff = 0;
    size_t smem_mma = 0;
    for (size_t i = 0; i < all.size(); ++i) {
        AccumTask& t = all[i];
        const int cls = i < spec.size() ? 0 : (i < spec.size() + diff.size() ? 1 : 2);
        int64_t& items = cls == 0 ? B.items_spec : (cls == 1 ? B.items_diff : B.items_mma);
        size_t& sm = cls == 0 ? B.smem_spec : (cls == 1 ? B.smem_diff : smem_mma);
        t.item0 = items;
        items += (int64_t)t.g.n_mb * t.g.n_bb * t.a.n_chunks;
        sm = std::max(sm, t.g.smem);
        t.out0 = out0;
        out0 += (int64_t)t.a.M * t.a.F;
        t.a.partial = reinterpret_cast<float2*>((size_t)part);  // offset for now
        part += (size_t)t.a.n_chunks * t.a.M * t.a.F * 8;
    }
    B.n_out = out0;
    cudaError_t e;
    if ((e = grow(B.part_all, std::max<size_t>(part, 256))) != cudaSuccess) return e;
    for (auto& t : all) t.a.partial = reinterpret_cast<float2*>(static_cast<char*>(B.part_all.p) + (size_t)t.a.partial);
    if ((e = grow(B.tasks, std::max<size_t>(all.size(), 1) * sizeof(AccumTask))) != cudaSuccess) return e;
    if ((e = grow(B.qctr, 16)) != cudaSuccess) return e;
    if (!all.empty() &&
        (e = cudaMemcpyAsync(B.tasks.p, all.data(), all.size() * sizeof(AccumTask), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);  // the host table is freed on return
}

cudaError_t batch_issue(st_ctx* c, BatchState& B, const st_job* jobs, const st_sim_params& p, const st_tune& tn,
                        cudaStream_t s) {
    cudaError_t e;
#define CB(x)                          \
    do {                               \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    const int n = B.n_jobs;
    const int64_t* offs = ptr<int64_t>(B.offs);
    BatchArgs a{};
    a.jobs = ptr<JobDev>(B.jobs_dev);
    a.n_jobs = n;
    a.ray_offs = offs;
    a.rec_offs = offs + (n + 1);
    a.samp_offs = offs + 2 * (n + 1);
    a.mic_offs = offs + 3 * (n + 1);
    a.mf_offs = offs + 4 * (n + 1);
    a.N_total = B.N_total;
    a.R_total = B.R_total;
    a.K_total = B.K_total;
    a.M_total = B.M_total;
    a.MF_total = B.MF_total;
    a.r_max = p.max_distance;
    a.c = p.c;
    a.a0 = p.alpha0_db_m;
    a.a1 = p.alpha1_db_m_khz;
    a.t_min = p.t_min;
    a.los_eps = p.los_eps;
    a.cos_inc = (float)cos((double)p.theta_inc_rad);
    a.direct_gain = p.direct_gain;
    a.seed = p.seed;
    a.ox = ptr<float>(B.st_o[0]);
    a.oy = ptr<float>(B.st_o[1]);
    a.oz = ptr<float>(B.st_o[2]);
    a.dx = ptr<float>(B.st_d[0]);
    a.dy = ptr<float>(B.st_d[1]);
    a.dz = ptr<float>(B.st_d[2]);
    a.racc = ptr<double>(B.st_r);
    a.prev = ptr<int32_t>(B.st_prev);
    uint32_t* cnt = ptr<uint32_t>(B.counts);
    a.q_in = ptr<uint32_t>(B.q0);
    a.q_out = ptr<uint32_t>(B.q1);
    a.n_in = cnt + 0;
    a.n_out = cnt + 1;
    a.rec_tri = ptr<int32_t>(B.rec_tri);
    a.rec_p = ptr<float>(B.rec_p);
    a.rec_d = ptr<float>(B.rec_d);
    a.rec_r = ptr<double>(B.rec_r);
    a.rec_los = ptr<uint8_t>(B.rec_los);
    a.cand_tri = ptr<int32_t>(B.cand_tri);
    a.cand_p = ptr<float>(B.cand_p);
    a.keep = ptr<uint8_t>(B.keep);
    a.dvis = ptr<uint8_t>(B.dvis);
    a.ranges = ptr<uint32_t>(B.ranges);
    a.flags = ptr<uint32_t>(B.flags);
    a.stack_limit = tn.stack_depth > 0 ? std::min(tn.stack_depth, kStack) : kStack;
    a.refill = tn.refill_lanes;
    a.queries = ptr<unsigned long long>(B.queries);
    a.hit_tri = ptr<int32_t>(B.hit_tri);
    a.hit_t = ptr<float>(B.hit_t);
    a.vis_q = ptr<uint32_t>(B.vis_q);
    a.los_q = ptr<uint32_t>(B.los_q);
    a.rec_mask = B.per_mic ? ptr<uint64_t>(B.rec_mask) : nullptr;
    a.vis_qm = B.per_mic ? ptr<uint64_t>(B.vis_qm) : nullptr;
    a.Q_total = B.Q_total;
    a.vis_n = cnt + 4;  // counts: [0] [1] live queues, [2] [3] compaction totals, [4] [5] visibility queues,
    a.los_n = cnt + 5;  // bytes 32..55 the three query counters
    a.ctr = reinterpret_cast<unsigned long long*>(cnt + 8);
    const int64_t Rn = std::max<int64_t>(B.R_total, 1);
    CB(cudaMemsetAsync(B.flags.p, 0, 16, s));
    CB(cudaMemsetAsync(B.counts.p, 0, 64, s));
    CB(cudaMemsetAsync(B.queries.p, 0, 64, s));
    CB(cudaMemsetAsync(B.rec_tri.p, 0xff, (size_t)Rn * 4, s));
    CB(cudaMemsetAsync(B.rec_los.p, 0, (size_t)Rn, s));
    for (int j = 0; j < n; ++j) CB(cudaMemsetAsync(jobs[j].spectra_out, 0, (size_t)3 * jobs[j].n_mics * jobs[j].n_bins * 8, s));
    CB(batch_prep(a.jobs, n, s));
    const bool spec = (p.components & ST_COMP_SPECULAR) && B.N_total > 0;
    const bool direct = (p.components & ST_COMP_DIRECT) != 0;
    const int64_t Koff = std::max<int64_t>(B.R_total, 1);  // candidate scan follows the record scan
    // the trace and the compaction of its visible records
    auto issue_trace = [&](cudaStream_t st_) -> cudaError_t {
        cudaError_t e;
        if (spec) {
            CB(batch_trace(a, B.max_b, B.N_total, tn.rays_per_block > 0 ? tn.rays_per_block : 128, st_));
            CB(flags_visible_records(a.rec_tri, a.rec_los, B.R_total, ptr<uint32_t>(B.sflags), st_));
            CB(exclusive_scan_u32(ptr<uint32_t>(B.sflags), ptr<uint32_t>(B.sscan), B.R_total, cnt + 2, B.scratch.p,
                                  st_));
            CB(compact_indices(ptr<uint32_t>(B.sflags), ptr<uint32_t>(B.sscan), B.R_total, ptr<uint32_t>(B.sidx), st_));
            CB(batch_gather_spec(a, ptr<uint32_t>(B.sidx), cnt + 2, B.spec, st_));
        }
        return cudaSuccess;
    };
    // diffraction sampling and filters, the compaction of kept candidates, the direct visibility
    auto issue_diffraction = [&](cudaStream_t st_) -> cudaError_t {
        cudaError_t e;
        if (B.K_total > 0) {
            CB(batch_diffraction(a, st_));
            uint32_t* fl = ptr<uint32_t>(B.sflags) + Koff;
            uint32_t* sc = ptr<uint32_t>(B.sscan) + Koff;
            uint32_t* ix = ptr<uint32_t>(B.sidx) + Koff;
            CB(flags_from_u8(a.keep, B.K_total, fl, st_));
            CB(exclusive_scan_u32(fl, sc, B.K_total, cnt + 3, B.dscratch.p, st_));
            CB(compact_indices(fl, sc, B.K_total, ix, st_));
            if (B.any_mma || B.any_table_order)  // tensor-core jobs' paths grouped by material, jobs with an
                                                 // emitter table's by table row (stable; jobs stay in place)
                CB(batch_material_order(a, cnt + 3, B.K_total, ix, ptr<uint32_t>(B.mat_off), B.mat_scr.p, st_));
            CB(batch_gather_diff(a, ix, cnt + 3, B.diff, st_));
        }
        if (direct) CB(batch_direct(a, st_));
        return cudaSuccess;
    };
    if (B.overlap && spec && (B.K_total > 0 || direct)) {  // a side branch beside the trace, joined before the ranges
        CB(cudaEventRecord(B.ev_fork, s));
        CB(cudaStreamWaitEvent(B.side, B.ev_fork, 0));
        const cudaError_t e1 = issue_diffraction(B.side);
        const cudaError_t e2 = e1 == cudaSuccess ? issue_trace(s) : cudaSuccess;
        CB(cudaEventRecord(B.ev_join, B.side));
        CB(cudaStreamWaitEvent(s, B.ev_join, 0));
        CB(e1);
        CB(e2);
    } else {
        CB(issue_trace(s));
        CB(issue_diffraction(s));
    }
    if (spec || B.K_total > 0)
        CB(batch_ranges(a, ptr<uint32_t>(B.sscan), cnt + 2, ptr<uint32_t>(B.sscan) + Koff, cnt + 3, s));
    if (direct) CB(batch_direct_accum(a, s));
    {  // every job's accumulation: two persistent launches over (job, tile) items, one reduction; the jobs
       // accumulated on their own on branches beside them (job i on branch i mod the branch count, each
       // branch with its own slice of partial spectra), joined at the end
        const int nbr = B.overlap && B.narrow_jobs.size() > 1 ? (int)std::min<size_t>(4, B.narrow_jobs.size()) : 0;
        if (nbr > 0) {
            CB(cudaEventRecord(B.br_fork, s));
            for (int k = 0; k < nbr; ++k) CB(cudaStreamWaitEvent(B.branch[k], B.br_fork, 0));
        }
        auto solo = [&]() -> cudaError_t {
            cudaError_t e;
            for (size_t i = 0; i < B.narrow_jobs.size(); ++i) {
                const int j = B.narrow_jobs[i];
                const int br = nbr > 0 ? (int)(i % nbr) : 0;
                cudaStream_t sj = nbr > 0 ? B.branch[br] : s;
                const JobDev& jd = B.jobs[j];
                const int64_t MF = (int64_t)jd.M * jd.F;
                float2* out = static_cast<float2*>(jobs[j].spectra_out);
                for (int kind = 0; kind < 2; ++kind) {
                    if (kind == 0 ? !(spec && jd.N > 0) : jd.K <= 0) continue;
                    AccumArgs y = batch_accum_args(B, jobs, j, kind, p, tn);
                    y.partial = reinterpret_cast<float2*>(static_cast<char*>(B.narrow_partial.p) + (size_t)br * B.narrow_slice);
                    if (kind == 1 && jd.diff_mma)
                        CB(accumulate_diffraction_mma(y, ptr<uint32_t>(B.mat_off) + (size_t)j * kMatStride, sj));
                    else
                        CB(accumulate(y, sj));
                    CB(reduce_partials(y.partial, y.n_chunks, MF, out + kind * MF, sj));
                }
            }
            return cudaSuccess;
        };
        const AccumTask* tk = ptr<AccumTask>(B.tasks);
        unsigned long long* qc = ptr<unsigned long long>(B.qctr);
        cudaError_t eq = cudaSuccess;
        auto queue = [&]() -> cudaError_t {
            cudaError_t e;
            if (spec) CB(accumulate_queue(0, tk, B.n_tasks_spec, B.items_spec, B.smem_spec, qc, s));
            if (B.K_total > 0)
                CB(accumulate_queue(1, tk + B.n_tasks_spec, B.n_tasks_diff, B.items_diff, B.smem_diff, qc + 1, s));
            if (B.K_total > 0)
                CB(accumulate_diffraction_mma_queue(tk + B.n_tasks_spec + B.n_tasks_diff, B.n_tasks_mma, B.items_mma, s));
            if (spec || B.K_total > 0)
                CB(reduce_tasks(tk, B.n_tasks_spec + B.n_tasks_diff + B.n_tasks_mma, B.n_out, s));
            return cudaSuccess;
        };
        const cudaError_t es = solo();  // (issued first: the branches start beside the queue launches)
        if (es == cudaSuccess) eq = queue();
        for (int k = 0; k < nbr; ++k) {  // joined whatever happened, so that nothing is left unordered
            cudaEventRecord(B.br_join[k], B.branch[k]);
            cudaStreamWaitEvent(s, B.br_join[k], 0);
        }
        CB(es);
        CB(eq);
    }
#undef CB
    return cudaSuccess;
}

}  // namespace

extern "C" {

static st_status simulate_batch_impl(st_ctx* c, int32_t n_jobs, const st_job* jobs, const st_sim_params* params,
                                     const st_tune* tune) {
    if (!c || n_jobs <= 0 || !jobs) return fail(c, ST_ERR_ARG, "simulate_batch: need jobs");
    st_sim_params p;
    st_sim_params_default(&p);
    if (params) p = *params;
    if (p.los_mode != ST_LOS_REFERENCE && p.los_mode != ST_LOS_PER_MIC)
        return fail(c, ST_ERR_ARG, "simulate_batch: los_mode must be ST_LOS_REFERENCE or ST_LOS_PER_MIC");
    const bool per_mic = p.los_mode == ST_LOS_PER_MIC;
    st_tune tn = tune ? *tune : c->tune;
    if (!tune_ok(tn)) return fail(c, ST_ERR_ARG, "simulate_batch: tune out of range");
    for (int j = 0; j < n_jobs; ++j) {
        const st_job& J = jobs[j];
        if (!J.scene || !J.scene->S.built || !J.scene->has_materials || J.scene->ctx != c)
            return fail(c, ST_ERR_STATE, "simulate_batch: every job needs a precomputed scene of this context");
        if (J.scene->S.two_level)
            return fail(c, ST_ERR_ARG, "simulate_batch: two-level scenes are traced by st_simulate");
        if (!J.emitter || !J.emitter_quat || !J.mics || !J.spectra_out || (J.n_rays > 0 && !J.dirs) || J.n_rays < 0 ||
            J.n_mics < 1 || J.n_mics > kMaxMics || J.n_bins < 1 || J.max_bounces < 1 || J.max_bounces > kMaxBounces ||
            !(J.f_lo > 0.0) || !(J.f_hi >= J.f_lo) || (J.n_bins > 1 && !(J.f_hi > J.f_lo)))
            return fail(c, ST_ERR_ARG, "simulate_batch: bad job");
        if ((J.dir_table && J.n_theta < 2) || (J.mic_tables && (J.n_el < 2 || J.n_az < 1 || J.scene->S.n_bands > 64)))
            return fail(c, ST_ERR_ARG, "simulate_batch: directivity tables need n_theta >= 2, n_el >= 2, n_az >= 1, "
                                       "<= 64 bands");
    }
    if (per_mic) {  // queue entries (record << 6 | m) and a 32-bit queue length
        int64_t q = 0;
        for (int j = 0; j < n_jobs; ++j) {
            if (jobs[j].n_mics > 64)
                return fail(c, ST_ERR_ARG, "simulate_batch: the per-microphone receiver test needs M <= 64 per job");
            q += jobs[j].n_rays * jobs[j].n_mics;
        }
        if (q >= (1ll << 32))
            return fail(c, ST_ERR_ARG, "simulate_batch: the per-microphone receiver test needs sum(N M) < 2^32");
    }
    enter(c);
    cudaStream_t s = c->stream;
    if (!c->batch) c->batch = new BatchState();
    BatchState& B = *c->batch;
    // structure key: everything the recorded work depends on except the poses' values
    uint64_t key = 1469598103934665603ull;
    key = fnv(key, &n_jobs, sizeof(n_jobs));
    for (int j = 0; j < n_jobs; ++j) {
        const st_job& J = jobs[j];
        const void* ptrs[9] = {J.scene, J.emitter, J.emitter_quat, J.dirs, J.mics, J.spectra_out, J.dir_table,
                               J.mic_quats, J.mic_tables};
        key = fnv(key, ptrs, sizeof(ptrs));
        const int32_t dv[3] = {J.dir_table ? J.n_theta : 0, J.mic_tables ? J.n_el : 0, J.mic_tables ? J.n_az : 0};
        key = fnv(key, dv, sizeof(dv));
        key = fnv(key, &J.scene->version, sizeof(uint64_t));
        key = fnv(key, &J.n_rays, sizeof(J.n_rays));
        const int32_t iv[3] = {J.n_mics, J.n_bins, J.max_bounces};
        key = fnv(key, iv, sizeof(iv));
        const double fv[2] = {J.f_lo, J.f_hi};
        key = fnv(key, fv, sizeof(fv));
        key = fnv(key, &J.pose_index, sizeof(J.pose_index));
        key = fnv(key, &J.fov_half_rad, sizeof(J.fov_half_rad));
    }
    const double pd[7] = {p.max_distance, p.c, p.alpha0_db_m, p.alpha1_db_m_khz, p.t_min, p.los_eps,
                          (double)p.theta_inc_rad};
    key = fnv(key, pd, sizeof(pd));
    const double pg = p.direct_gain;
    key = fnv(key, &pg, sizeof(pg));
    const int64_t pi[4] = {(int64_t)p.components, (int64_t)p.reflection_mode, (int64_t)p.seed, (int64_t)p.los_mode};
    key = fnv(key, pi, sizeof(pi));
    const int32_t ti[6] = {tn.rays_per_block, tn.mic_pairs_per_cta, tn.smem_kb, tn.stack_depth, tn.refill_lanes,
                           tn.bins_per_thread};
    key = fnv(key, ti, sizeof(ti));
    const int32_t ov = c->overlap ? 1 : 0;
    key = fnv(key, &ov, sizeof(ov));
    if (B.valid && B.key == key && B.exec) {
        const int ne = (int)B.events.size();
        CKC(c, cudaEventRecord(B.events[ne - 2], s), "batch order");
        CKC(c, cudaStreamWaitEvent(B.main, B.events[ne - 2], 0), "batch order");
        CKC(c, cudaGraphLaunch(B.exec, B.main), "batch graph launch");
        CKC(c, cudaEventRecord(B.events[ne - 1], B.main), "batch order");
        CKC(c, cudaStreamWaitEvent(s, B.events[ne - 1], 0), "batch order");
        return ST_OK;
    }
    // ---- (re)build the batch's buffers, tables and job table
    batch_release(B);
    B = BatchState();
    B.n_jobs = n_jobs;
    B.any_mma = false;
    B.any_table_order = false;
    B.tables.resize(n_jobs);
    B.jobs.resize(n_jobs);
    B.chunks_spec.resize(n_jobs);
    B.chunks_diff.resize(n_jobs);
    std::vector<int64_t> ho(5 * (size_t)(n_jobs + 1), 0);
    int64_t* ray_o = ho.data();
    int64_t* rec_o = ray_o + (n_jobs + 1);
    int64_t* smp_o = rec_o + (n_jobs + 1);
    int64_t* mic_o = smp_o + (n_jobs + 1);
    int64_t* mf_o = mic_o + (n_jobs + 1);
    for (int j = 0; j < n_jobs; ++j) {
        const st_job& J = jobs[j];
        const int64_t K = (p.components & ST_COMP_DIFFRACTION) ? J.scene->S.total_samples : 0;
        ray_o[j + 1] = ray_o[j] + J.n_rays;
        rec_o[j + 1] = rec_o[j] + J.n_rays * J.max_bounces;
        smp_o[j + 1] = smp_o[j] + K;
        mic_o[j + 1] = mic_o[j] + J.n_mics;
        mf_o[j + 1] = mf_o[j] + (int64_t)J.n_mics * J.n_bins;
        B.max_b = std::max(B.max_b, (int)J.max_bounces);
    }
    B.per_mic = per_mic;
    B.Q_total = 0;
    for (int j = 0; j < n_jobs; ++j) B.Q_total += per_mic ? jobs[j].n_rays * jobs[j].n_mics : 0;
    B.N_total = ray_o[n_jobs];
    B.R_total = rec_o[n_jobs];
    B.K_total = smp_o[n_jobs];
    B.M_total = mic_o[n_jobs];
    B.MF_total = mf_o[n_jobs];
    const int64_t N1 = std::max<int64_t>(B.N_total, 1), R1 = std::max<int64_t>(B.R_total, 1),
                  K1 = std::max<int64_t>(B.K_total, 1);
    CKC(c, grow(B.offs, ho.size() * 8), "batch alloc");
    CKC(c, cudaMemcpyAsync(B.offs.p, ho.data(), ho.size() * 8, cudaMemcpyHostToDevice, s), "batch copy");
    CKC(c, grow(B.derived, (size_t)n_jobs * 6 * 4), "batch alloc");
    CKC(c, grow(B.perm, (size_t)N1 * 4), "batch alloc");
    int64_t max_n = 1;
    for (int j = 0; j < n_jobs; ++j) max_n = std::max(max_n, jobs[j].n_rays);
    CKC(c, grow(B.ord_keys, (size_t)max_n * 8), "batch alloc");
    CKC(c, grow(B.ord_scr, sort_scratch_bytes(max_n)), "batch alloc");
    for (int k = 0; k < 3; ++k) {
        CKC(c, grow(B.st_o[k], (size_t)N1 * 4), "batch alloc");
        CKC(c, grow(B.st_d[k], (size_t)N1 * 4), "batch alloc");
    }
    CKC(c, grow(B.st_r, (size_t)N1 * 8), "batch alloc");
    CKC(c, grow(B.st_prev, (size_t)N1 * 4), "batch alloc");
    CKC(c, grow(B.q0, (size_t)N1 * 4), "batch alloc");
    CKC(c, grow(B.q1, (size_t)N1 * 4), "batch alloc");
    CKC(c, grow(B.hit_tri, (size_t)N1 * 4), "batch alloc");
    CKC(c, grow(B.hit_t, (size_t)N1 * 4), "batch alloc");
    CKC(c, grow(B.vis_q, (size_t)N1 * 4), "batch alloc");
    if (per_mic) {
        CKC(c, grow(B.rec_mask, (size_t)R1 * 8), "batch alloc");
        CKC(c, grow(B.vis_qm, (size_t)std::max<int64_t>(B.Q_total, 1) * 8), "batch alloc");
    }
    CKC(c, grow(B.counts, 64), "batch alloc");
    CKC(c, grow(B.queries, 64), "batch alloc");
    CKC(c, grow(B.flags, 16), "batch alloc");
    CKC(c, grow(B.rec_tri, (size_t)R1 * 4), "batch alloc");
    CKC(c, grow(B.rec_p, (size_t)R1 * 12), "batch alloc");
    CKC(c, grow(B.rec_d, (size_t)R1 * 12), "batch alloc");
    CKC(c, grow(B.rec_r, (size_t)R1 * 8), "batch alloc");
    CKC(c, grow(B.rec_los, (size_t)R1), "batch alloc");
    CKC(c, grow(B.cand_tri, (size_t)K1 * 4), "batch alloc");
    CKC(c, grow(B.cand_p, (size_t)K1 * 12), "batch alloc");
    CKC(c, grow(B.keep, (size_t)K1), "batch alloc");
    CKC(c, grow(B.los_q, (size_t)K1 * 4), "batch alloc");
    CKC(c, grow(B.dvis, (size_t)std::max<int64_t>(B.M_total, 1)), "batch alloc");
    CKC(c, grow(B.ranges, (size_t)n_jobs * 16), "batch alloc");
    CKC(c, grow(B.sflags, (size_t)(R1 + K1) * 4), "batch alloc");
    CKC(c, grow(B.sscan, (size_t)(R1 + K1) * 4), "batch alloc");
    CKC(c, grow(B.sidx, (size_t)(R1 + K1) * 4), "batch alloc");
    CKC(c, grow(B.scratch, scan_scratch_bytes(R1)), "batch alloc");
    CKC(c, grow(B.dscratch, scan_scratch_bytes(K1)), "batch alloc");
    for (PathList* P : {&B.spec, &B.diff}) {
        const int64_t nP = P == &B.spec ? R1 : K1;
        for (DevBuf* b : {&P->px, &P->py, &P->pz, &P->dx, &P->dy, &P->dz, &P->rhi, &P->rlo, &P->chain_lo, &P->chain_hi,
                          &P->meta, &P->dep})
            CKC(c, grow(*b, (size_t)nP * 4), "batch alloc");
        if (per_mic && P == &B.spec) CKC(c, grow(P->mask, (size_t)nP * 8), "batch alloc");  // u64 per path
        P->n_max = nP;
    }
    size_t narrow_part = 256;  // chunk partials of the largest one-pair job (launched on its own)
    float* derived = ptr<float>(B.derived);
    for (int j = 0; j < n_jobs; ++j) {
        const st_job& J = jobs[j];
        SceneDev& S = J.scene->S;
        CKC(c, build_accum_tables(B.tables[j], S, J.n_bins, J.f_lo, J.f_hi, p.c, p.alpha0_db_m, p.alpha1_db_m_khz, s),
            "batch tables");
        if (J.n_rays > 0)
            CKC(c, direction_order(J.dirs, J.n_rays, ptr<uint64_t>(B.ord_keys), ptr<uint32_t>(B.perm) + ray_o[j],
                                   B.ord_scr.p, s),
                "batch order");
        JobDev& d = B.jobs[j];
        d = JobDev{};
        d.nodes = ptr<float4>(S.nodes);
        d.tri_v = ptr<float4>(S.tri_v);
        d.nrm = ptr<float>(S.nrm);
        d.tri_mat = ptr<int32_t>(S.tri_mat);
        d.verts = ptr<float>(S.verts);
        d.tris = ptr<int32_t>(S.tris);
        d.mesh_tris = ptr<int32_t>(S.mesh_tris);
        d.mesh_off = ptr<int64_t>(S.mesh_off);
        d.cdf = ptr<uint64_t>(S.cdf);
        d.sample_off = ptr<int64_t>(S.sample_off);
        d.root = S.root;
        d.max_iter = (int32_t)std::min<int64_t>(2 * S.n_tris + 8, (int64_t)1 << 30);
        d.n_obj = S.n_obj;
        d.n_mat = S.n_mat;
        d.chk_nodes = S.n_nodes > 0 ? S.n_nodes : 1;
        d.chk_tris = S.n_tris;
        d.cos_fov = J.fov_half_rad >= (float)M_PI ? -2.0f : (float)cos((double)J.fov_half_rad);
        d.s = J.emitter;
        d.q = J.emitter_quat;
        d.dirs = J.dirs;
        d.mics = J.mics;
        d.R = derived + 6 * j;
        d.fwd = derived + 6 * j + 3;
        d.perm = J.n_rays > 0 ? ptr<uint32_t>(B.perm) + ray_o[j] : nullptr;
        d.qhi = ptr<float>(B.tables[j].qhi);
        d.qlo = ptr<float>(B.tables[j].qlo);
        d.bw = ptr<float2>(B.tables[j].bw);
        d.etab = J.dir_table;
        d.n_theta = J.dir_table ? J.n_theta : 0;
        d.inv_dtheta = J.dir_table ? (float)((J.n_theta - 1) / M_PI) : 0.0f;
        d.mic_tab = J.mic_tables;
        d.mic_q = J.mic_tables ? J.mic_quats : nullptr;
        d.n_el = J.mic_tables ? J.n_el : 0;
        d.n_az = J.mic_tables ? J.n_az : 0;
        d.n_bands = S.n_bands;
        d.N = J.n_rays;
        d.K = smp_o[j + 1] - smp_o[j];
        d.ray_off = ray_o[j];
        d.rec_off = rec_o[j];
        d.samp_off = smp_o[j];
        d.mic_off = mic_o[j];
        d.mf_off = mf_o[j];
        d.B = J.max_bounces;
        d.M = J.n_mics;
        d.F = J.n_bins;
        d.pose = J.pose_index;
        d.f_lo = J.f_lo;
        d.df = B.tables[j].df;
        d.out = static_cast<float2*>(J.spectra_out);
        // chunks: the jobs of the work queue share the GPU, so each one's accumulation is split into about an
        // eighth of the chunks that would fill it alone (fewer partial spectra to sum); a job accumulated on its
        // own (one microphone pair, receiver tables, a million paths or more) runs alone and takes them all
        const int nb = solo_accum(d) ? 1 : kBatchChunkDiv;
        const int dir_nb = J.mic_tables ? S.n_bands : 0;
        {
            AccumArgs probe{};
            probe.kind = 1;
            probe.M = d.M;
            probe.F = d.F;
            probe.n_mat_tab = S.n_mat;
            probe.etab = d.etab;
            probe.mic_tab = d.mic_tab;
            d.diff_mma = d.K > 0 && diffraction_mma_applies(probe) ? 1 : 0;
        }
        B.any_mma = B.any_mma || d.diff_mma;
        B.any_table_order = B.any_table_order || (d.etab != nullptr && d.K > 0 && !d.diff_mma);
        B.chunks_spec[j] =
            std::max(1, accum_chunks(d.N * d.B, d.M, d.F, S.n_mat, dir_nb, tn.mic_pairs_per_cta, tn.smem_kb) / nb);
        B.chunks_diff[j] =
            d.diff_mma ? std::max(1, diffraction_mma_chunks(d.K, d.M, d.F, S.n_mat) / nb)
                       : std::max(1, accum_chunks(d.K, d.M, d.F, S.n_mat, dir_nb, tn.mic_pairs_per_cta, tn.smem_kb) / nb);
        if (solo_accum(d))
            narrow_part = std::max(narrow_part, (size_t)std::max(B.chunks_spec[j], B.chunks_diff[j]) * d.M * d.F * 8);
    }
    B.narrow_slice = (narrow_part + 255) & ~(size_t)255;
    CKC(c, grow(B.narrow_partial, 4 * B.narrow_slice), "batch alloc");
    if (B.any_mma || B.any_table_order) {
        CKC(c, grow(B.mat_off, (size_t)n_jobs * kMatStride * 4), "batch alloc");
        CKC(c, grow(B.mat_scr, material_order_scratch(B.K_total)), "batch alloc");
    }
    CKC(c, batch_tasks(c, B, jobs, p, tn, s), "batch tasks");
    CKC(c, grow(B.jobs_dev, sizeof(JobDev) * (size_t)n_jobs), "batch alloc");
    CKC(c, cudaMemcpyAsync(B.jobs_dev.p, B.jobs.data(), sizeof(JobDev) * (size_t)n_jobs, cudaMemcpyHostToDevice, s),
        "batch copy");
    B.events.resize(2);  // context -> batch stream, batch stream -> context
    for (auto& ev : B.events) CKC(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch events");
    CKC(c, cudaStreamCreateWithFlags(&B.main, cudaStreamNonBlocking), "batch streams");
    CKC(c, cudaStreamCreateWithFlags(&B.side, cudaStreamNonBlocking), "batch streams");
    CKC(c, cudaEventCreateWithFlags(&B.ev_fork, cudaEventDisableTiming), "batch events");
    CKC(c, cudaEventCreateWithFlags(&B.ev_join, cudaEventDisableTiming), "batch events");
    CKC(c, cudaEventCreateWithFlags(&B.br_fork, cudaEventDisableTiming), "batch events");
    for (int k = 0; k < 4; ++k) {
        CKC(c, cudaStreamCreateWithFlags(&B.branch[k], cudaStreamNonBlocking), "batch streams");
        CKC(c, cudaEventCreateWithFlags(&B.br_join[k], cudaEventDisableTiming), "batch events");
    }
    B.overlap = c->overlap;
    CKC(c, cudaStreamSynchronize(s), "batch setup");
    // ---- eager run (also sets kernel attributes), then record the graph for later calls
    cudaStream_t ms = B.main;
    CKC(c, batch_issue(c, B, jobs, p, tn, ms), "batch run");
    CKC(c, cudaStreamSynchronize(ms), "batch run");
    uint32_t fl = 0;
    CKC(c, cudaMemcpy(&fl, B.flags.p, 4, cudaMemcpyDeviceToHost), "batch flags");
    if (fl & kFlagBadTree) return fail(c, ST_ERR_CUDA, "malformed BVH: traversal exceeded the node count");
    if (fl & kFlagCheck) return fail(c, ST_ERR_CUDA, "a bounds check of the checked build failed");
    CKC(c, cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal), "batch capture");
    cudaError_t ie = batch_issue(c, B, jobs, p, tn, ms);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(ms, &g);
    if (ie != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, ie, "batch capture");
    }
    CKC(c, ce, "batch capture end");
    B.graph = g;
    CKC(c, cudaGraphInstantiate(&B.exec, g, 0), "batch instantiate");
    B.key = key;
    B.valid = true;
    return ST_OK;
}

st_status st_set_tune(st_ctx* c, const st_tune* tune) {
    if (!c || !tune) return fail(c, ST_ERR_ARG, "set_tune: null argument");
    if (!tune_ok(*tune)) return fail(c, ST_ERR_ARG, "set_tune: value out of range");
    c->tune = *tune;
    return ST_OK;
}

st_status st_autotune(st_ctx* c, const st_job* J, const st_sim_params* params, st_tune* out) {
    if (!c || !J || !out) return fail(c, ST_ERR_ARG, "autotune: null argument");
    if (!J->scene || !J->scene->S.built) return fail(c, ST_ERR_STATE, "autotune: precomputed scene needed");
    enter(c);
    st_status r;
    if ((r = st_set_frequencies(c, J->n_bins, J->f_lo, J->f_hi)) != ST_OK) return r;
    if ((r = st_set_emitter(c, J->emitter, J->emitter_quat, J->n_rays, J->dirs, nullptr, 0, J->fov_half_rad,
                            ST_MEM_DEVICE)) != ST_OK)
        return r;
    if ((r = st_set_receivers(c, J->n_mics, J->mics, nullptr, nullptr, 0, 0, 0, ST_MEM_DEVICE)) != ST_OK) return r;
    st_sim_params p;
    st_sim_params_default(&p);
    if (params) p = *params;
    p.max_bounces = J->max_bounces;
    p.pose_index = J->pose_index;
    p.los_mode = ST_LOS_REFERENCE;  // the tuned shapes serve the batched form
    DevBuf out_buf;
    CKC(c, grow(out_buf, (size_t)3 * J->n_mics * J->n_bins * 8), "autotune alloc");
    const st_tune saved = c->tune;
    const bool saved_overlap = c->overlap;
    c->overlap = false;  // each stage timed on its own
    const int rpb[3] = {64, 128, 256};
    const int tiles[5][2] = {{16, 96}, {8, 96}, {16, 64}, {4, 96}, {16, 128}};
    const int kts[2] = {16, 8};
    const int depths[3] = {0, 48, 24};
    const int refills[4] = {0, 12, 20, 32};
    st_tune best = {128, 16, 96, 0, 0, 0};
    // one parameter at a time, each with the best of the earlier ones: the tracing block size, the accumulator
    // tile (microphone pairs and shared memory), its bins per thread (frequency tile), the traversal stack depth
    // and the lane-refill threshold (rays per warp refill); tracing phases are timed on tracing and diffraction,
    // the others on the accumulator kernels
    const int n_phase[5] = {3, 5, 2, 3, 4};
    for (int phase = 0; phase < 5; ++phase) {
        const int n_cand = n_phase[phase];
        st_tune winner = best;
        float winner_ms = 1e30f;
        for (int i = 0; i < n_cand; ++i) {
            st_tune t = best;
            if (phase == 0) t.rays_per_block = rpb[i];
            else if (phase == 1) {
                t.mic_pairs_per_cta = tiles[i][0];
                t.smem_kb = tiles[i][1];
            } else if (phase == 2) {
                t.bins_per_thread = kts[i];
            } else if (phase == 3) {
                t.stack_depth = depths[i];
            } else {
                t.refill_lanes = refills[i];
            }
            c->tune = t;
            st_stats st;
            float acc = 0.0f;
            for (int rep = 0; rep < 3; ++rep) {
                r = st_simulate(c, J->scene, &p, out_buf.p, &st);
                if (r != ST_OK) {
                    c->tune = saved;
                    c->overlap = saved_overlap;
                    release(out_buf);
                    return r;
                }
                const bool tracing = phase == 0 || phase >= 3;
                if (rep > 0) acc += tracing ? st.ms_trace + st.ms_diffraction : st.ms_accum_kernel;
            }
            if (acc < winner_ms) {
                winner_ms = acc;
                winner = t;
            }
        }
        best = winner;
    }
    release(out_buf);
    c->overlap = saved_overlap;
    c->tune = best;
    *out = best;
    return ST_OK;
}

// ---- checkpoint / resume of a precomputed flat scene
// Blob: "STSC", format version, a header of sizes and parameters, the material tables, then every device
// array of the scene as (u64 byte count, bytes, zero padding to 8 bytes), in a fixed order.
namespace {
constexpr uint32_t kBlobMagic = 0x43535453u;  // "STSC"
constexpr uint32_t kBlobVersion = 1;
struct BlobHeader {
    uint32_t magic, version;
    int64_t n_verts, n_tris, n_nodes, total_samples;
    int32_t n_obj, root, n_mat, n_bands;
    float bounds_lo[3], bounds_hi[3];
    float eta, area_ref, hc_frac;
    int32_t samples_per_vertex;
    double dither;
    int64_t budget;
    uint64_t seed;
    uint64_t checksum;  // FNV-1a over everything after the header
};

// the scene's device arrays with their sizes in bytes, from the counts (a flat precomputed scene has all of
// them; the binary topology only above one leaf)
std::vector<std::pair<DevBuf*, size_t>> scene_arrays(SceneDev& S) {
    const size_t nv = (size_t)S.n_verts, nt = (size_t)S.n_tris, no = (size_t)S.n_obj;
    const bool tree = nt > (size_t)kLeafMax;
    return {{&S.verts, nv * 12},
            {&S.tris, nt * 12},
            {&S.tri_mat, nt * 4},
            {&S.tri_obj, nt * 4},
            {&S.nrm, nt * 12},
            {&S.nodes, (size_t)std::max<int64_t>(S.n_nodes, 1) * 128},
            {&S.tri_v, nt * 48},
            {&S.G, nv * 4},
            {&S.C, nt * 4},
            {&S.mesh_tris, nt * 4},
            {&S.mesh_off, (no + 1) * 8},
            {&S.cdf, nt * 8},
            {&S.n_samples, (no + 1) * 8},
            {&S.sample_off, (no + 1) * 8},
            {&S.bvh_child, tree ? (nt - 1) * 8 : 0},
            {&S.bvh_range, tree ? (nt - 1) * 8 : 0},
            {&S.bvh_par_i, tree ? nt * 4 : 0},
            {&S.bvh_par_l, tree ? nt * 4 : 0},
            {&S.bvh_perm, nt * 4},
            {&S.bvh_wflag, tree ? (nt - 1) * 4 : 0},
            {&S.bvh_widx, tree ? (nt - 1) * 4 : 0}};
}

size_t pad8(size_t n) { return (n + 7) & ~size_t(7); }

uint64_t fnv1a(const char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= (uint8_t)p[i];
        h *= 1099511628211ull;
    }
    return h;
}
}  // namespace

st_status st_scene_serialize(st_scene* sc, void* buf, size_t* bytes) {
    if (!sc || !bytes) return ST_ERR_ARG;
    st_ctx* c = sc->ctx;
    if (!sc->precomputed || !sc->S.built || !sc->S.bvh_ready)
        return fail(c, ST_ERR_STATE, "scene_serialize: a precomputed scene is needed");
    if (sc->instanced) return fail(c, ST_ERR_STATE, "scene_serialize: instanced scenes are not serialised");
    SceneDev& S = sc->S;
    const auto arrays = scene_arrays(S);
    const size_t nb = (size_t)S.n_mat * S.n_bands;
    size_t total = pad8(sizeof(BlobHeader)) + pad8((size_t)S.n_bands * 4) + 3 * pad8(nb * 4);
    for (const auto& a : arrays) total += 8 + pad8(a.second);
    if (!buf) {
        *bytes = total;
        return ST_OK;
    }
    if (*bytes < total) {
        *bytes = total;
        return fail(c, ST_ERR_ARG, "scene_serialize: buffer too small (*bytes holds the size needed)");
    }
    enter(c);
    char* o = static_cast<char*>(buf);
    memset(o, 0, total);
    BlobHeader h{};
    h.magic = kBlobMagic;
    h.version = kBlobVersion;
    h.n_verts = S.n_verts;
    h.n_tris = S.n_tris;
    h.n_nodes = S.n_nodes;
    h.total_samples = S.total_samples;
    h.n_obj = S.n_obj;
    h.root = S.root;
    h.n_mat = S.n_mat;
    h.n_bands = S.n_bands;
    memcpy(h.bounds_lo, S.bounds_lo, 12);
    memcpy(h.bounds_hi, S.bounds_hi, 12);
    h.eta = sc->cp.eta;
    h.area_ref = sc->cp.area_ref;
    h.hc_frac = sc->cp.hc_frac;
    h.samples_per_vertex = sc->cp.samples_per_vertex;
    h.dither = sc->cp.dither;
    h.budget = sc->cp.budget;
    h.seed = sc->cp.seed;
    memcpy(o, &h, sizeof(h));
    size_t at = pad8(sizeof(BlobHeader));
    memcpy(o + at, S.band_hz.data(), (size_t)S.n_bands * 4);
    at += pad8((size_t)S.n_bands * 4);
    for (const std::vector<float>* v : {&S.k_band, &S.beta_band, &S.diff_band}) {
        memcpy(o + at, v->data(), nb * 4);
        at += pad8(nb * 4);
    }
    CKC(c, cudaStreamSynchronize(c->stream), "scene_serialize sync");  // earlier work may still write the scene
    for (const auto& a : arrays) {
        const uint64_t n = a.second;
        memcpy(o + at, &n, 8);
        at += 8;
        if (n) CKC(c, cudaMemcpy(o + at, a.first->p, n, cudaMemcpyDeviceToHost), "scene_serialize copy");
        at += pad8(n);
    }
    h.checksum = fnv1a(o + pad8(sizeof(BlobHeader)), total - pad8(sizeof(BlobHeader)));
    memcpy(o, &h, sizeof(h));
    *bytes = total;
    return ST_OK;
}

st_status st_scene_deserialize(st_ctx* c, const void* buf, size_t bytes, st_scene** out) {
    if (!c || !buf || !out) return ST_ERR_ARG;
    *out = nullptr;
    const char* in = static_cast<const char*>(buf);
    BlobHeader h;
    if (bytes < sizeof(h)) return fail(c, ST_ERR_ARG, "scene_deserialize: blob too short");
    memcpy(&h, in, sizeof(h));
    if (h.magic != kBlobMagic || h.version != kBlobVersion)
        return fail(c, ST_ERR_ARG, "scene_deserialize: not a scene blob of this format version");
    if (h.n_verts <= 0 || h.n_tris <= 0 || h.n_tris >= (1ll << 28) || h.n_verts >= (1ll << 31) || h.n_obj < 1 ||
        h.n_obj > (1 << 24) || h.n_mat < 1 || h.n_mat > 255 || h.n_bands < 1 || h.n_bands > 64 || h.n_nodes < 0 ||
        h.n_nodes >= h.n_tris + 1 || h.total_samples < 0)
        return fail(c, ST_ERR_ARG, "scene_deserialize: sizes out of range");
    // the whole blob is checked before anything reaches the device: its contents index device arrays
    if (bytes < pad8(sizeof(BlobHeader)) || fnv1a(in + pad8(sizeof(BlobHeader)), bytes - pad8(sizeof(BlobHeader))) !=
                                                 h.checksum)
        return fail(c, ST_ERR_ARG, "scene_deserialize: checksum mismatch (truncated or modified blob)");
    enter(c);
    st_scene* sc = new st_scene();
    sc->ctx = c;
    SceneDev& S = sc->S;
    S.n_verts = h.n_verts;
    S.n_tris = h.n_tris;
    S.n_nodes = h.n_nodes;
    S.total_samples = h.total_samples;
    S.n_obj = h.n_obj;
    S.root = h.root;
    S.n_mat = h.n_mat;
    S.n_bands = h.n_bands;
    memcpy(S.bounds_lo, h.bounds_lo, 12);
    memcpy(S.bounds_hi, h.bounds_hi, 12);
    const size_t nb = (size_t)h.n_mat * h.n_bands;
    size_t at = pad8(sizeof(BlobHeader));
    auto fail_free = [&](st_status code, const char* msg) {
        scene_free(sc);
        return fail(c, code, msg);
    };
    if (at + pad8((size_t)h.n_bands * 4) + 3 * pad8(nb * 4) > bytes)
        return fail_free(ST_ERR_ARG, "scene_deserialize: blob too short");
    S.band_hz.assign(reinterpret_cast<const float*>(in + at), reinterpret_cast<const float*>(in + at) + h.n_bands);
    at += pad8((size_t)h.n_bands * 4);
    for (std::vector<float>* v : {&S.k_band, &S.beta_band, &S.diff_band}) {
        v->assign(reinterpret_cast<const float*>(in + at), reinterpret_cast<const float*>(in + at) + nb);
        at += pad8(nb * 4);
    }
    for (const auto& a : scene_arrays(S)) {
        uint64_t n = 0;
        if (at + 8 > bytes) return fail_free(ST_ERR_ARG, "scene_deserialize: blob too short");
        memcpy(&n, in + at, 8);
        at += 8;
        // every array has exactly the size the header's counts give it
        if (n != a.second || n > bytes - at) return fail_free(ST_ERR_ARG, "scene_deserialize: array size mismatch");
        if (n) {
            cudaError_t e = grow(*a.first, n);
            if (e == cudaSuccess) e = cudaMemcpy(a.first->p, in + at, n, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                scene_free(sc);
                return cuda_fail(c, e, "scene_deserialize copy");
            }
        }
        at += pad8(n);
    }
    S.built = true;
    S.bvh_ready = true;
    sc->cp = CurvParamsDev{h.eta, h.area_ref, h.hc_frac, h.dither, h.samples_per_vertex, h.budget, h.seed};
    sc->has_materials = true;
    sc->precomputed = true;
    sc->version = g_scene_version++;
    c->scenes.push_back(sc);
    *out = sc;
    return ST_OK;
}

// ---- entry points with NVTX ranges and ST_LOG lines around the implementations above
st_status st_simulate(st_ctx* c, st_scene* sc, const st_sim_params* params, void* spectra_out, st_stats* stats) {
    NvtxRange range("st_simulate");
    const st_status r = simulate_impl(c, sc, params, spectra_out, stats);
    if (r == ST_OK)
        st_log(2, "simulate: %lld rays x %d bounces, %lld diffraction samples, %d mics x %d bins",
               (long long)c->last_N, (int)c->last_B, (long long)c->last_K, (int)c->last_M, (int)c->last_F);
    return r;
}

st_status st_scene_precompute(st_scene* sc, const st_curv_params* params) {
    NvtxRange range("st_scene_precompute");
    const st_status r = precompute_impl(sc, params);
    if (r == ST_OK)
        st_log(2, "precompute: %lld triangles, %lld diffraction samples%s", (long long)sc->S.n_tris,
               (long long)sc->S.total_samples, sc->S.two_level ? ", two-level" : "");
    return r;
}

st_status st_simulate_batch(st_ctx* c, int32_t n_jobs, const st_job* jobs, const st_sim_params* params,
                            const st_tune* tune) {
    NvtxRange range("st_simulate_batch");
    const st_status r = simulate_batch_impl(c, n_jobs, jobs, params, tune);
    if (r == ST_OK) st_log(2, "simulate_batch: %d jobs", (int)n_jobs);
    return r;
}

}  // extern "C"
