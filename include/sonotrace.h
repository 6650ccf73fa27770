/*
 * sonotrace.h -- C ABI of the GB300 acoustic path-tracing library.
 *
 * The library computes, on one GPU, the specular, diffraction and direct spectra of an
 * in-air ultrasonic scene as described for SonoTraceUE (Jansen & Steckel, arXiv 2602.19652):
 *   - Sec. III-B  geometric pre-processing: Meyer mean curvature G_v, triangle metric C_i (Eq. 1)
 *   - Sec. III-C  Algorithm 1: multi-bounce specular tracing of emitter rays with a visibility ray
 *                 per hit; magnitudes with 1/r^2 spreading, atmospheric decay and the BRDF lobe
 *                 (Eq. 2, 3) synthesised into complex spectra H(f) (Eq. 4), summed over paths
 *   - Sec. III-D  curvature-importance-sampled diffraction candidates, field-of-view, incidence
 *                 and visibility filters, magnitudes M_d (Eq. 7), spectra G(f) (Eq. 8)
 *   - Sec. III-E  the direct emitter-to-receiver path, M_p (Eq. 11), P(f) (Eq. 12)
 * The inverse transforms (Eq. 5-6, 9-10, 13) are linear and act on the summed spectra.
 *
 * Conventions
 *   - Every call returns st_status (0 = ST_OK, < 0 = error) and never throws.  The message of
 *     the last error of a context is available from st_last_error().
 *   - All arrays are row-major, little-endian; float = IEEE binary32, double = binary64.
 *     Complex spectra are interleaved (re, im) float32 pairs.
 *   - A `mem` argument says where a pointer lives: ST_MEM_HOST (pageable or pinned host memory)
 *     or ST_MEM_DEVICE (device memory of the context's GPU).  Inputs are copied; the caller
 *     keeps ownership of everything it passes.
 *   - Work is issued on the context's CUDA stream and is stream-ordered: device outputs are
 *     complete when that stream reaches the point after the call.  Calls that return host
 *     data or statistics synchronise the stream.
 *   - Not thread-safe per context; different contexts may be used from different threads.
 */
#ifndef SONOTRACE_H
#define SONOTRACE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t st_status;
#define ST_OK 0
#define ST_ERR_ARG (-1)      /* invalid argument (null pointer, size out of range, ...) */
#define ST_ERR_CUDA (-2)     /* a CUDA call failed; see st_last_error() */
#define ST_ERR_OOM (-3)      /* device allocation failed */
#define ST_ERR_MESH (-4)     /* index out of range or non-finite vertex in the mesh */
#define ST_ERR_TIMEOUT (-5)  /* a bounded device-side wait gave up */
#define ST_ERR_STATE (-6)    /* call out of order (e.g. simulate before set_receivers) */
#define ST_ERR_OVERFLOW (-7) /* a fixed-size device structure overflowed (reserved: the traversal stack restarts instead) */

#define ST_MEM_HOST 0
#define ST_MEM_DEVICE 1

/* bits of st_sim_params.components and indices of the spectra's first dimension */
#define ST_COMP_SPECULAR 1   /* index 0: H(f), Eq. 4 */
#define ST_COMP_DIFFRACTION 2 /* index 1: G(f), Eq. 8 */
#define ST_COMP_DIRECT 4     /* index 2: P(f), Eq. 12 */

/* Receiver test of a specular hit (st_sim_params.los_mode).  The paper leaves the test unstated: the
   default casts one visibility ray per hit towards the receiver reference point (the microphones'
   centroid) and lets the hit reach every microphone when it is visible; the per-microphone variant casts
   one ray per microphone and lets the hit reach only the microphones it sees (M <= 64). */
#define ST_LOS_REFERENCE 0
#define ST_LOS_PER_MIC 1

typedef struct st_ctx st_ctx;
typedef struct st_scene st_scene;

/* Pre-processing parameters (Sec. III-B and III-D). */
typedef struct st_curv_params {
    float eta;                  /* global scale of Eq. 1 (default 1) */
    float area_ref;             /* w(A) = clamp(A / area_ref, 0, 1), m^2 (default 1e-4) */
    double dither;              /* CDF dither amplitude relative to the mesh-mean weight (default 1e-3) */
    float hc_frac;              /* a triangle is high-curvature if C_i >= hc_frac * max_mesh C (default 0.25) */
    int32_t samples_per_vertex; /* diffraction samples per high-curvature vertex (default 64) */
    int64_t sample_budget;      /* cap on the total sample count, < 0 = none (default 4,000,000) */
    uint64_t seed;              /* Philox key of the CDF dither (default 0) */
} st_curv_params;

/* Simulation parameters (Algorithm 1, Eq. 2-4, 7-8, 11-12). */
typedef struct st_sim_params {
    int32_t max_bounces;        /* B: hit points per ray (default 3), 1..8 */
    double max_distance;        /* a ray ends after the hit whose path length reaches this, m (default 1e9) */
    double c;                   /* speed of sound, m/s (default 343) */
    double alpha0_db_m;         /* air absorption alpha(f) = alpha0 + alpha1 * f[kHz], dB/m (amplitude) */
    double alpha1_db_m_khz;     /* (defaults 0 and 0.033) */
    float t_min;                /* minimum hit distance along a ray, m (default 1e-5) */
    float los_eps;              /* visibility rays stop this short of their target, m (default 1e-4) */
    int32_t reflection_mode;    /* 0: product of k over all hits so far; 1: k of the last hit only */
    int32_t components;         /* ST_COMP_* mask (default all) */
    float theta_inc_rad;        /* diffraction incidence constraint, |n . v_s| >= cos(theta) (default 80 deg) */
    float direct_gain;          /* I_p of Eq. 11 (default 1) */
    uint64_t seed;              /* Philox key of the diffraction samples (default 0) */
    uint32_t pose_index;        /* Philox counter word distinguishing poses (default 0) */
    int32_t los_mode;           /* ST_LOS_* (default ST_LOS_REFERENCE); ST_LOS_PER_MIC needs M <= 64 and
                                   N * B * M < 2^32 (st_backward then follows the masks); in
                                   st_simulate_batch M <= 64 per job and sum(N M) < 2^32;
                                   st_accumulate_specular_noalloc takes the caller's records and ignores it */
} st_sim_params;

/* Optional statistics of one simulate call (filled after the stream is synchronised). */
typedef struct st_stats {
    int64_t rays;               /* emitter rays */
    int64_t closest_queries;    /* closest-hit ray segments traced */
    int64_t shadow_queries;     /* any-hit visibility segments traced */
    int64_t records;            /* specular hit records */
    int64_t visible_records;    /* records whose receiver point is visible */
    int64_t candidates;         /* diffraction samples drawn */
    int64_t candidates_kept;    /* diffraction samples passing the filters */
    int64_t terms;              /* (path, microphone, bin) terms accumulated */
    float ms_trace;             /* device time of ray generation + bounces, ms */
    float ms_diffraction;       /* device time of sampling + filters, ms (with the stage overlap of
                                   st_set_stage_overlap on, this runs beside the trace, so the stage times
                                   overlap) */
    float ms_accumulate;        /* device time of spectrum accumulation, ms (from the end of the trace; with
                                   the overlap on it includes the wait for the diffraction stage) */
    float ms_total;             /* device time of the whole call, ms */
    float ms_accum_kernel;      /* device time of the accumulator kernel launches alone, ms */
    int32_t accum_launches;     /* number of accumulator kernel launches */
    int64_t kernel_launches;    /* kernels launched by this call */
    int64_t visits[4];          /* with ST_COUNT_VISITS=1: BVH nodes and triangles visited by closest-hit
                                   queries, then by any-hit queries (0 otherwise) */
    int64_t stack_restarts;     /* traversal queries that outgrew their stack and restarted from the root */
    float ms_accum_specular;    /* device time of the specular accumulator launch, ms */
    float ms_accum_diffraction; /* device time of the diffraction accumulator launch, ms */
    int64_t terms_specular;     /* (path, microphone, bin) terms of the specular launch */
    int64_t terms_diffraction;  /* ... of the diffraction launch */
    int32_t diffraction_tensor; /* 1: the diffraction launch ran on the tensor cores (k_accum_diff_mma) */
} st_stats;

/* Fill a parameter block with the library defaults (every field; the caller owns the block). */
void st_curv_params_default(st_curv_params* p);
void st_sim_params_default(st_sim_params* p);
/* Static name of a status code ("unknown status" for a value outside the list above). */
const char* st_status_string(st_status s);
/* 1 in the bounds-checked build (compiled with ST_CHECKS: indices read from device data -- tree references,
 * leaf, triangle and material ids -- are checked before they index an array; a failed check skips the access
 * and the call returns ST_ERR_CUDA), 0 otherwise. */
int32_t st_checked_build(void);
/* Message of the last failing call on ctx (owned by ctx, valid until the next call). */
const char* st_last_error(const st_ctx* ctx);

/* Create a context on `device` issuing work on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream).  The library allocates its working memory lazily and owns it until destroy. */
st_status st_create(st_ctx** out, int32_t device, void* cuda_stream);
/* Frees the context, its working memory and every scene still loaded into it (their handles become
 * invalid: do not pass them to st_scene_destroy afterwards). */
st_status st_destroy(st_ctx* ctx);
/* Issue later work on another stream of the same device (a cudaStream_t; NULL = legacy default).  Work
 * already issued stays on the old stream: synchronise it first if later calls read its results. */
st_status st_set_stream(st_ctx* ctx, void* cuda_stream);

/* Scene (Sec. III-B: the registered objects' meshes).  verts [n_verts][3], tris [n_tris][3]
 * (indices into verts), tri_material [n_tris] (index into the material table), tri_object
 * [n_tris] (mesh id >= 0; diffraction CDFs are built per mesh).  Indices out of range or
 * non-finite vertices give ST_ERR_MESH.  The scene belongs to ctx and must be destroyed before it. */
st_status st_scene_load(st_ctx* ctx, const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                        const int32_t* tri_material, const int32_t* tri_object, int32_t mem, st_scene** out);
/* Materials (Sec. III-B): per-band reflection magnitude k [n_mat][n_bands], lobe opening angle
 * beta [n_mat][n_bands] (rad, > 0) and diffraction coefficient I_d [n_mat][n_bands] at band
 * centres band_hz [n_bands] (ascending).  Host pointers.  Values are linear in frequency between
 * centres (beta through the lobe exponent 1/(2 beta^2)) and constant beyond the end bands. */
st_status st_scene_set_materials(st_scene* scene, int32_t n_mat, int32_t n_bands, const float* band_hz,
                                 const float* k, const float* beta, const float* diffr);
/* Build the device LBVH, triangle normals, curvature (G_v, C_i) and diffraction CDFs.
 * params may be NULL (defaults).  Synchronises the stream once (to size the sample buffers). */
st_status st_scene_precompute(st_scene* scene, const st_curv_params* params);
/* Dynamic scenes: new positions for the same vertices (n_verts [3] floats, host or device per mem)
 * of a precomputed scene, then a refit: the LBVH topology and leaf order of the last precompute are
 * kept and the boxes, wide nodes, leaf triangles and normals recomputed (results stay exact: the
 * boxes are conservative for any positions, only the traversal cost can grow with large motions).
 * Welding, curvature, metric, CDFs and sample counts are recomputed too, unless flags holds
 * ST_REFIT_KEEP_CURVATURE (valid when whole meshes move rigidly, which leaves them unchanged up to
 * rounding).  The scene's version changes: simulate again before st_backward; recorded batches
 * re-record.  A non-finite vertex returns ST_ERR_MESH and leaves the scene unbuilt (simulate returns
 * ST_ERR_STATE) until a later update with finite positions, which then builds it in full with the
 * parameters of its last precompute.  ST_ERR_STATE before the scene's first successful precompute. */
#define ST_REFIT_KEEP_CURVATURE 1
st_status st_scene_update_vertices(st_scene* scene, const float* verts, int32_t mem, int32_t flags);
/* Instanced scene (Sec. III-B registers objects; a forest repeats a few plant meshes many times).
 * n_proto shared meshes, concatenated: prototype p owns vertices proto_vert_offset[p] ..
 * proto_vert_offset[p+1] of proto_verts [.][3] and triangles proto_tri_offset[p] .. proto_tri_offset[p+1]
 * of proto_tris [.][3] (vertex indices local to the prototype) with materials proto_tri_material [.];
 * offsets [n_proto + 1], starting at 0 and ascending.  n_inst instances: instance i is prototype
 * inst_proto[i] under the affine map x -> A x + b, inst_xform [n_inst][12] the row-major 3 x 4 matrices
 * [A | b].  The world scene is expanded on the device: instance i's vertices and triangles follow
 * instance i-1's, each world coordinate ((A_r0 x + A_r1 y) + A_r2 z) + b_r rounded to float32 in that
 * order, and instance i is mesh (object) i for the diffraction CDFs.  All pointers are host memory,
 * copied.  Then as a loaded scene: set materials, precompute.  ST_ERR_ARG: a null pointer, no
 * prototype, 0 or >= 2^24 instances, offsets not ascending from 0, more than 2^31 world vertices or 2^28
 * world triangles, none at all; ST_ERR_MESH: a local index or prototype id out of range, a non-finite
 * vertex or transform. */
st_status st_scene_load_instances(st_ctx* ctx, int32_t n_proto, const int64_t* proto_vert_offset,
                                  const float* proto_verts, const int64_t* proto_tri_offset, const int32_t* proto_tris,
                                  const int32_t* proto_tri_material, int32_t n_inst, const int32_t* inst_proto,
                                  const float* inst_xform, st_scene** out);
/* Moves the instances of a precomputed instanced scene: new transforms inst_xform [n_inst][12] (host
 * or device per mem), the world vertices expanded again on the device, then the refit of
 * st_scene_update_vertices with the same flags (ST_REFIT_KEEP_CURVATURE for rotations and
 * translations).  ST_ERR_STATE for a scene not loaded by st_scene_load_instances or never precomputed;
 * ST_ERR_MESH when a world vertex is not finite (the scene is then unbuilt until a later call with finite
 * maps, as for st_scene_update_vertices). */
st_status st_scene_set_instance_transforms(st_scene* scene, const float* inst_xform, int32_t mem, int32_t flags);
/* Checkpoint / resume of a precomputed scene loaded flat: st_scene_serialize writes the mesh, the material
 * tables, the curvature, metric and CDFs, the 4-wide BVH with its refit topology and the precompute's
 * parameters into buf (host memory, *bytes long); buf NULL returns the size needed in *bytes.
 * st_scene_deserialize makes a new scene of ctx from such a blob, precomputed: simulates on it give the
 * same bits as on the serialised scene.  The blob carries a format version and a checksum of its contents;
 * a blob that is truncated, modified or of another version returns ST_ERR_ARG before anything reaches the
 * device.  ST_ERR_STATE for a scene not precomputed, or loaded by st_scene_load_instances; ST_ERR_ARG for a
 * buffer smaller than *bytes (which then holds the size needed).  Synchronises the context's stream. */
st_status st_scene_serialize(st_scene* scene, void* buf, size_t* bytes);
st_status st_scene_deserialize(st_ctx* ctx, const void* buf, size_t bytes, st_scene** out);
/* Hierarchy of an instanced scene.  ST_STRUCTURE_FLAT (the default): one BVH over the expanded world
 * triangles.  ST_STRUCTURE_TWO_LEVEL: a 4-wide BVH per prototype over its triangles in object space, built
 * once, and a top-level BVH over the instances' world boxes, rebuilt by every precompute and instance
 * move; a ray enters a prototype's BVH after moving into the instance's object space, but triangles are
 * tested in world space with their vertices mapped as in the expansion, so every result (path records,
 * filters, spectra) is bit-identical to the flat structure's.  No hierarchy over the world triangles is
 * kept (less memory, faster precompute and moves); the expanded triangles, normals, curvature and CDFs
 * stay.  Takes effect at once on a precomputed scene (rebuilt with its last precompute's parameters).
 * ST_ERR_ARG for another value; ST_ERR_STATE for two levels on a scene not loaded by
 * st_scene_load_instances; ST_ERR_MESH when an instance map is singular.  A two-level scene is traced by
 * st_simulate and its variants; st_simulate_batch rejects it (ST_ERR_ARG) and st_scene_update_vertices
 * returns ST_ERR_STATE (it moves by st_scene_set_instance_transforms). */
#define ST_STRUCTURE_FLAT 0
#define ST_STRUCTURE_TWO_LEVEL 1
st_status st_scene_set_structure(st_scene* scene, int32_t structure);
/* The scene's triangles as loaded or expanded: counts (either may be NULL), then verts [n_verts][3],
 * tris [n_tris][3], tri_material [n_tris], tri_object [n_tris] (any may be NULL).  Synchronises. */
st_status st_scene_get_geometry(st_scene* scene, int64_t* n_verts, int64_t* n_tris, float* verts, int32_t* tris,
                                int32_t* tri_material, int32_t* tri_object, int32_t mem);
/* Copy per-vertex G [n_verts], per-triangle C [n_tris] and the diffraction sample count per
 * mesh out (any may be NULL).  n_samples has one entry per mesh id up to max(tri_object). */
st_status st_scene_get_curvature(st_scene* scene, float* G, float* C, int64_t* n_samples, int32_t mem);
/* Synchronise the context's stream, then free the scene's device memory; NULL is ST_ERR_ARG.  A recorded
 * batch is recorded again at its next st_simulate_batch; st_backward needs a new simulate. */
st_status st_scene_destroy(st_scene* scene);

/* Emitter (Algorithm 1 inputs): position, orientation quaternion (w, x, y, z; forward is +x
 * rotated by it), n_rays local unit directions dirs [n_rays][3], an optional directivity table
 * [n_theta][n_bins] over the angle to forward in [0, pi] (NULL = omni; n_bins must equal the
 * frequency grid at simulate time) and the diffraction field of view half-angle (>= pi: off). */
st_status st_set_emitter(st_ctx* ctx, const float pos[3], const float quat[4], int64_t n_rays, const float* dirs,
                         const float* dir_table, int32_t n_theta, float fov_half_rad, int32_t mem);
/* Receivers: positions [n_mics][3]; optional orientations [n_mics][4] and directivity tables
 * [n_mics][n_el][n_az][n_bands] on the (az, el) grid az = -pi + 2 pi i / n_az, el = -pi/2 +
 * pi j / (n_el - 1) of the arrival direction in the microphone frame, bands = the materials'
 * band centres (NULL = omni).  1..4096 microphones; with tables n_el >= 2, n_az >= 1 and 1..64 bands
 * (ST_ERR_ARG otherwise). */
st_status st_set_receivers(st_ctx* ctx, int32_t n_mics, const float* pos, const float* quats,
                           const float* tables, int32_t n_el, int32_t n_az, int32_t n_bands, int32_t mem);
/* Uniform frequency grid f_k = f_lo + k (f_hi - f_lo) / (n_bins - 1), k = 0..n_bins-1, Hz (one bin: f_lo).
 * 1..2^20 bins and 0 < f_lo < f_hi (ST_ERR_ARG otherwise). */
st_status st_set_frequencies(st_ctx* ctx, int32_t n_bins, double f_lo, double f_hi);
/* The same grid given as its bins, f_hz [n_bins] ascending, Hz, host memory (the paper's frequency
 * bins of the spectra, Sec. III-C / III-F).  The accumulators advance each path's phasor by one
 * constant bin spacing, so the bins must be uniformly spaced: every inner bin within 4 float32 ulps
 * of f_hz[0] + k (f_hz[n-1] - f_hz[0]) / (n - 1).  Then equal to st_set_frequencies(n_bins,
 * f_hz[0], f_hz[n_bins-1]).  Errors: ST_ERR_ARG for a null pointer, 0 or more than 2^20 bins,
 * f_hz[0] <= 0, bins not strictly ascending or not uniformly spaced (the context keeps its grid). */
st_status st_set_frequency_grid(st_ctx* ctx, int32_t n_bins, const float* f_hz);

/* One simulation: tracing, diffraction, direct path, accumulation.  spectra_out is caller-owned
 * device memory of 3 * n_mics * n_bins complex64 values laid out [component][mic][bin]; every
 * element is written (components not requested are zero).  params NULL = defaults.  The path
 * records are kept in ctx for st_get_paths / st_backward until the next simulate. */
st_status st_simulate(st_ctx* ctx, st_scene* scene, const st_sim_params* params, void* spectra_out,
                      st_stats* stats);
/* Same, with host input/output: spectra_out is host memory (3 * n_mics * n_bins complex64). */
st_status st_simulate_host(st_ctx* ctx, st_scene* scene, const st_sim_params* params, void* spectra_out,
                           st_stats* stats);

/* Path records of the last simulate, [n_rays][B] each (any pointer may be NULL): hit triangle
 * (-1 = none), hit point [3], reflected direction [3], path length (float64), receiver-point
 * visibility.  Synchronises. */
st_status st_get_paths(st_ctx* ctx, int32_t* tri, float* point, float* dir, double* r, uint8_t* los, int32_t mem);
/* Per-microphone receiver test of the last simulate (made with ST_LOS_PER_MIC, else ST_ERR_STATE):
 * [n_rays][B] masks, bit m set when microphone m is visible from the record's hit point (0 for records
 * without a hit); the record's visibility flag of st_get_paths is then "any bit set".  Synchronises.
 * The paper states no receiver test; this is the per-microphone reading of its receiver connection. */
st_status st_get_receiver_masks(st_ctx* ctx, uint64_t* mask, int32_t mem);
/* Diffraction samples of the last simulate: *n_out = count; triangle, point [3], kept flag
 * (arrays of at least `capacity` entries; any may be NULL).  Synchronises. */
st_status st_get_diffraction(st_ctx* ctx, int64_t* n_out, int32_t* tri, float* point, uint8_t* keep,
                             int64_t capacity, int32_t mem);
/* Direct-path visibility per microphone of the last simulate. */
st_status st_get_direct_visibility(st_ctx* ctx, uint8_t* vis, int32_t mem);

/* Adjoint of the last simulate with its path set frozen (the paper has no gradients; this is the
 * reverse pass of Eq. 2-4, 7-8 and 11-12).  grad_spectra = dL/dRe S + j dL/dIm S, device complex64
 * [3][n_mics][n_bins] laid out like the spectra.  Writes, as device float32 (any may be NULL):
 *   grad_k [n_mat][n_bands]: reflection band values (specular paths; assumes k > 0 at every bin),
 *   grad_mic [n_mics][3]:    microphone positions (specular, diffraction and direct paths),
 *   grad_emitter [3]:        emitter position: diffraction and direct paths, and specular paths
 *                            through their hit points (ray directions and triangle chains frozen:
 *                            hit q moves along d_q with the line from hit q-1, dP_q/dP_{q-1} =
 *                            I - d_q n_q^T / (n_q . d_q)).
 * After a simulate with ST_LOS_PER_MIC each specular path reaches only the microphones of its mask here too.
 * Needs omni receivers; position gradients also need an omni emitter (ST_ERR_ARG otherwise).  scene must be the one of the
 * last simulate, unchanged since (ST_ERR_STATE otherwise).  Deterministic: every sum runs in a fixed
 * order.  Stream-ordered; allocates reduction buffers on first use.  The first call after a simulate (omni
 * emitter) puts that simulate's internal specular path list in reflection-chain order, so that the reflection
 * sums are formed once per run of paths with equal material counts; later calls find it so, and repeated calls
 * give identical gradients.  With the stage overlap (st_set_stage_overlap) the diffraction and direct-path
 * adjoints run on the context's side stream beside the specular one. */
st_status st_backward(st_ctx* ctx, st_scene* scene, const void* grad_spectra, float* grad_k, float* grad_mic,
                      float* grad_emitter);
/* Adjoint with respect to the lobe widths: grad_beta [n_mat][n_bands] device float32, the gradient of
 * the loss through the specular lobe exp(-gamma^2 / (2 beta^2)) of each path's last hit (the lobe
 * exponent interpolated between bands through 1 / (2 beta^2)).  Same conditions as st_backward.  Its
 * float32 sums follow the path list's order, so a call before and a call after st_backward (which orders
 * the list by reflection chain) can differ in the last bits. */
st_status st_backward_beta(st_ctx* ctx, st_scene* scene, const void* grad_spectra, float* grad_beta);

/* Batched form: many poses (over one or more precomputed scenes) simulated together.  Every stage
 * runs over all jobs in one launch (one per bounce level for tracing), and the per-job accumulations
 * run on parallel branches of a CUDA graph.  The first call with a given batch structure (jobs'
 * scenes, sizes, pointers, params, tune) runs eagerly and records the graph; later calls with the
 * same structure replay it, reading the poses (emitter, emitter_quat, dirs, mics) from the job
 * pointers at run time, so callers update them in place between calls.  Omni emitter and receivers;
 * either receiver test (params->los_mode); params NULL = defaults; tune NULL = defaults.  ST_ERR_ARG for
 * a bad job, or with ST_LOS_PER_MIC more than 64 microphones in a job or sum(N M) >= 2^32; ST_ERR_STATE
 * for a scene not precomputed or of another context.  Writes every job's spectra_out
 * (complex64 [3][n_mics][n_bins]).  Stream-ordered on the context's stream. */
typedef struct st_job {
    st_scene* scene;            /* precomputed scene */
    const float* emitter;       /* device [3] */
    const float* emitter_quat;  /* device [4] */
    const float* dirs;          /* device [n_rays][3] local unit directions */
    int64_t n_rays;
    const float* mics;          /* device [n_mics][3] */
    int32_t n_mics;
    int32_t n_bins;
    double f_lo, f_hi;          /* uniform frequency grid */
    int32_t max_bounces;        /* 1..8 */
    uint32_t pose_index;        /* Philox counter word of the diffraction samples */
    float fov_half_rad;         /* diffraction field of view half-angle (>= pi: off) */
    void* spectra_out;          /* device complex64 [3][n_mics][n_bins] */
    /* Directivity (Sec. III-F), as st_set_emitter and st_set_receivers take it, in device memory; NULL:
     * omni.  The tables are read at run time, like the poses. */
    const float* dir_table;     /* [n_theta][n_bins] emitter pattern over the angle from its forward axis */
    int32_t n_theta;            /* >= 2 with dir_table */
    const float* mic_quats;     /* [n_mics][4] microphone orientations (NULL: identity) */
    const float* mic_tables;    /* [n_mics][n_el][n_az][n_bands] receiver transfer on the scene's bands */
    int32_t n_el, n_az;         /* >= 2 and >= 1 with mic_tables */
} st_job;

/* Launch shapes picked by st_autotune (0 = default). */
typedef struct st_tune {
    int32_t rays_per_block;     /* tracing block size: 64, 128 or 256 */
    int32_t mic_pairs_per_cta;  /* accumulator: microphone pairs per CTA, 1..16 */
    int32_t smem_kb;            /* accumulator: shared-memory budget per CTA, 32..160 KB */
    int32_t stack_depth;        /* traversal stack entries per query, 1..128 (0 = 128).  A query that would
                                   need more restarts from the root with a walk that needs no stack (fixed
                                   child order, parent references in the nodes), keeping its best hit, so
                                   results do not depend on it; st_stats.stack_restarts counts the restarts */
    int32_t refill_lanes;       /* rays per warp refill: the persistent traversal kernels give new queries to a
                                   warp's idle lanes once this many of its 32 lanes wait, 1..32 (0 = 16 for
                                   closest hits, 28 for visibility rays) */
    int32_t bins_per_thread;    /* frequency tile: bins a thread of the general accumulator advances, 8 or 16
                                   (0 = 16; the batched form takes 16) */
} st_tune;

st_status st_simulate_batch(st_ctx* ctx, int32_t n_jobs, const st_job* jobs, const st_sim_params* params,
                            const st_tune* tune);
/* Sets the context's launch shapes (as st_autotune does); later st_simulate calls use them.  ST_ERR_ARG for
 * a null pointer or a value outside the ranges above. */
st_status st_set_tune(st_ctx* ctx, const st_tune* tune);
/* Stage overlap of st_simulate (on by default): the diffraction stage (sampling, filters and line of
 * sight of Sec. III-D, then its accumulation, Eq. 7-8) and the direct path (Eq. 11-12) run on a side
 * stream of the context while the specular paths are traced (Algorithm 1) on the context's stream;
 * the specular accumulation (Eq. 2-4) starts once both are done.  The stages share no buffer, so the
 * results are identical either way.  0 issues every stage on the context's stream in the order trace,
 * diffraction, accumulation (stage times that do not overlap).  The side stream is created on the
 * first overlapped call.  ST_ERR_ARG for a null context. */
st_status st_set_stage_overlap(st_ctx* ctx, int32_t on);
/* Times candidate launch shapes on one sample job through the single-pose path and writes the
 * fastest to *out (also kept as the context's default for st_simulate).  Replaces the context's
 * emitter, receivers and frequency grid with the sample job's (omni).  Synchronises. */
st_status st_autotune(st_ctx* ctx, const st_job* sample, const st_sim_params* params, st_tune* out);

/* Emitter ray sets written on the device, float32 [n][3] unit directions in the emitter frame, for
 * st_set_emitter (ST_MEM_DEVICE).  ST_RAYS_FIBONACCI: the spherical Fibonacci lattice, z_i = 1 -
 * (2i + 1) / n, phi_i = i pi (3 - sqrt 5).  ST_RAYS_ZONAL: the centre points of the recursive zonal
 * equal-area partition of the sphere into n regions (Leopardi 2006), the paper's ray set (Sec.
 * III-C): two polar caps, collars of equal-area regions, each region's centre at the midpoint of its
 * colatitude and longitude ranges, collar i+1 rotated by half a region against collar i.  Directions
 * are evaluated in float64 and rounded once.  Synchronises (the zone table is uploaded).  Errors:
 * ST_ERR_ARG for a null pointer, n < 1 or an unknown kind. */
#define ST_RAYS_FIBONACCI 0
#define ST_RAYS_ZONAL 1
st_status st_ray_directions(st_ctx* ctx, int32_t kind, int64_t n, float* out);

/* Impulse responses and received signals (Eq. 5-6, 9-10, 13 and the signal equation of Sec. III-F).
 * Every path's transfer function is M(f) e^{+j 2 pi f r / c}; summed over paths, a component's
 * impulse response is the inverse Fourier transform of its spectrum, the components add, and the
 * received signal is the impulse response convolved with the emitted call.  On the spectra's uniform
 * grid f_k = f_lo + k df (df = (f_hi - f_lo) / (n_bins - 1); 1 for a single bin), with the kernel
 * e^{-j 2 pi f t} (echoes at t = r / c) and the spectra taken as the positive frequencies of a real
 * signal:
 *     out[r][n] = 2 df Re sum_k w_k E_k S'[r][k] e^{-j 2 pi f_k n / fs},  n < n_samples,
 *     E_k = (1 / fs) sum_i call[i] e^{+j 2 pi f_k i / fs}  (1 when call is NULL or call_len is 0),
 * The response is periodic in t with period 1 / df: an echo at r / c beyond it wraps around.
 * where S'[m] = sum over the n_comp components of spectra[c][m] (out [n_mics][n_samples]) or, with
 * ST_IR_PER_COMPONENT in flags, S'[c M + m] = spectra[c][m] (out [n_comp][n_mics][n_samples]).
 * spectra: device complex64 [n_comp][n_mics][n_bins] (st_simulate's layout); window: device float
 * [n_bins] or NULL; call: device float [call_len] sampled at fs, or NULL; out: device float32.
 * Stream-ordered on the context's stream; scratch is owned by the context.  Errors: ST_ERR_ARG for
 * null pointers, n_comp outside 1..3, n_mics < 1, n_bins < 1, n_samples < 1, fs <= 0, f_hi < f_lo. */
#define ST_IR_PER_COMPONENT 1
st_status st_impulse_response(st_ctx* ctx, const void* spectra, int32_t n_comp, int32_t n_mics, int32_t n_bins,
                              double f_lo, double f_hi, double fs, int32_t n_samples, const float* window,
                              const float* call, int32_t call_len, int32_t flags, float* out);

/* Testing hook for the failure paths (no counterpart in the paper): after `after` further device
 * allocations by this library succeed, the next one fails as cudaMalloc does when the device is out of
 * memory (the call that needs it returns ST_ERR_OOM; no memory is allocated for it), and injection
 * switches off.  after < 0 switches it off.  Process-wide, not thread-safe; the library never calls it. */
void st_inject_alloc_failure(int64_t after);

/* Allocation-free specular accumulation.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory where they need spectra -- code running inside another
 * allocator's fixed memory budget or arena, real-time loops where cudaMalloc would stall or
 * synchronise the device, or callbacks in which allocation is not allowed.
 *
 * Computes the specular component (index 0 of st_simulate's spectra, Eq. 2-4) from path records
 * laid out as st_get_paths returns them: rec_tri [n_rays][max_bounces] (-1 = no hit), rec_point and
 * rec_dir [n_rays][max_bounces][3], rec_r [n_rays][max_bounces] (float64), rec_los [n_rays]
 * [max_bounces]; tri_material [n_tris]; mics [n_mics][3]; all device pointers.  The material band
 * tables (band_hz [n_bands], k and beta [n_mat][n_bands]) are host pointers, read by stream-ordered
 * copies (keep them unchanged until the call's work on cuda_stream has finished).  Omni emitter and
 * receivers.  Uses params->c, alpha0/alpha1 and reflection_mode (NULL = defaults).  Writes
 * spectra_out, device complex64 [n_mics][n_bins], on cuda_stream.  max_bounces is 1..8.
 * Precondition: every triangle id of a visible record's chain is in 0..n_tris-1 and its material in
 * 0..n_mat-1; a record whose chain breaks this contributes nothing (nothing is read out of range).
 *
 * It calls no allocator.  Its scratch is one array of ST_NOALLOC_SCRATCH_BYTES compiled into the
 * library; every GPU that loads the library holds it until the process exits.  Sizes whose tables
 * plus one chunk of partial spectra (about 8 * n_mics * n_bins + 8 * n_mat * n_bins bytes) exceed
 * it return ST_ERR_ARG.  The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture begins.  The call itself is not
 * meant for capture into a CUDA graph: its host band tables are copied with cudaMemcpyAsync, which a
 * capture would either refuse (pageable memory) or replay from the host buffer as it is at replay time
 * (pinned memory).  All calls share the
 * array: calls that overlap on the GPU race and give wrong results, so order them on one stream.
 * Every call rewrites all of the scratch it reads, so no state carries over between calls. */
#define ST_NOALLOC_SCRATCH_BYTES (8u << 20)
st_status st_accumulate_specular_noalloc(const int32_t* rec_tri, const float* rec_point, const float* rec_dir,
                                         const double* rec_r, const uint8_t* rec_los, int64_t n_rays,
                                         int32_t max_bounces, const int32_t* tri_material, int64_t n_tris,
                                         const float* mics, int32_t n_mics, int32_t n_bins, double f_lo,
                                         double f_hi, int32_t n_mat, int32_t n_bands, const float* band_hz,
                                         const float* k, const float* beta, const st_sim_params* params,
                                         void* spectra_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SONOTRACE_H */
