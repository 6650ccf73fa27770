"""ctypes declarations of the C ABI in include/sonotrace.h (argument marshalling only).

The shared library is built in-tree by `paper_2602_19652_gb300.build`; if it is missing this
module raises instead of falling back to anything else."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# ST_CHECKS=1 in the environment loads the bounds-checked build (build(checks=True)) instead
LIB_PATH = os.path.join(HERE, "_build_checks" if os.environ.get("ST_CHECKS") == "1" else "_build", "libsonotrace.so")

P = C.c_void_p
I32, I64, U32, U64, F32, F64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_float, C.c_double

ST_OK = 0
# status codes (include/sonotrace.h)
ST_ERR_ARG, ST_ERR_CUDA, ST_ERR_OOM, ST_ERR_MESH, ST_ERR_TIMEOUT, ST_ERR_STATE, ST_ERR_OVERFLOW = -1, -2, -3, -4, -5, -6, -7
ST_MEM_HOST, ST_MEM_DEVICE = 0, 1
ST_IR_PER_COMPONENT = 1
ST_REFIT_KEEP_CURVATURE = 1
ST_STRUCTURE_FLAT, ST_STRUCTURE_TWO_LEVEL = 0, 1
ST_RAYS_FIBONACCI, ST_RAYS_ZONAL = 0, 1
ST_COMP_SPECULAR, ST_COMP_DIFFRACTION, ST_COMP_DIRECT = 1, 2, 4
ST_LOS_REFERENCE, ST_LOS_PER_MIC = 0, 1


class CurvParams(C.Structure):
    _fields_ = [("eta", F32), ("area_ref", F32), ("dither", F64), ("hc_frac", F32), ("samples_per_vertex", I32),
                ("sample_budget", I64), ("seed", U64)]


class SimParams(C.Structure):
    _fields_ = [("max_bounces", I32), ("max_distance", F64), ("c", F64), ("alpha0_db_m", F64),
                ("alpha1_db_m_khz", F64), ("t_min", F32), ("los_eps", F32), ("reflection_mode", I32),
                ("components", I32), ("theta_inc_rad", F32), ("direct_gain", F32), ("seed", U64),
                ("pose_index", U32), ("los_mode", I32)]


class Stats(C.Structure):
    _fields_ = [("rays", I64), ("closest_queries", I64), ("shadow_queries", I64), ("records", I64),
                ("visible_records", I64), ("candidates", I64), ("candidates_kept", I64), ("terms", I64),
                ("ms_trace", F32), ("ms_diffraction", F32), ("ms_accumulate", F32), ("ms_total", F32),
                ("ms_accum_kernel", F32), ("accum_launches", I32), ("kernel_launches", I64),
                ("visits", I64 * 4), ("stack_restarts", I64), ("ms_accum_specular", F32),
                ("ms_accum_diffraction", F32), ("terms_specular", I64), ("terms_diffraction", I64),
                ("diffraction_tensor", I32)]


class Job(C.Structure):
    _fields_ = [("scene", P), ("emitter", P), ("emitter_quat", P), ("dirs", P), ("n_rays", I64), ("mics", P),
                ("n_mics", I32), ("n_bins", I32), ("f_lo", F64), ("f_hi", F64), ("max_bounces", I32),
                ("pose_index", U32), ("fov_half_rad", F32), ("spectra_out", P), ("dir_table", P), ("n_theta", I32),
                ("mic_quats", P), ("mic_tables", P), ("n_el", I32), ("n_az", I32)]


class Tune(C.Structure):
    _fields_ = [("rays_per_block", I32), ("mic_pairs_per_cta", I32), ("smem_kb", I32), ("stack_depth", I32),
                ("refill_lanes", I32), ("bins_per_thread", I32)]


# name -> (restype, argtypes); every symbol declared in include/sonotrace.h
SIGNATURES = {
    "st_curv_params_default": (None, [P]),
    "st_sim_params_default": (None, [P]),
    "st_status_string": (C.c_char_p, [I32]),
    "st_checked_build": (I32, []),
    "st_last_error": (C.c_char_p, [P]),
    "st_create": (I32, [P, I32, P]),
    "st_destroy": (I32, [P]),
    "st_set_stream": (I32, [P, P]),
    "st_scene_load": (I32, [P, P, I64, P, I64, P, P, I32, P]),
    "st_scene_set_materials": (I32, [P, I32, I32, P, P, P, P]),
    "st_scene_precompute": (I32, [P, P]),
    "st_scene_get_curvature": (I32, [P, P, P, P, I32]),
    "st_scene_destroy": (I32, [P]),
    "st_set_emitter": (I32, [P, P, P, I64, P, P, I32, F32, I32]),
    "st_set_receivers": (I32, [P, I32, P, P, P, I32, I32, I32, I32]),
    "st_set_frequencies": (I32, [P, I32, F64, F64]),
    "st_simulate": (I32, [P, P, P, P, P]),
    "st_simulate_host": (I32, [P, P, P, P, P]),
    "st_get_paths": (I32, [P, P, P, P, P, P, I32]),
    "st_get_receiver_masks": (I32, [P, P, I32]),
    "st_get_diffraction": (I32, [P, P, P, P, P, I64, I32]),
    "st_get_direct_visibility": (I32, [P, P, I32]),
    "st_backward": (I32, [P, P, P, P, P, P]),
    "st_backward_beta": (I32, [P, P, P, P]),
    "st_simulate_batch": (I32, [P, I32, P, P, P]),
    "st_autotune": (I32, [P, P, P, P]),
    "st_scene_update_vertices": (I32, [P, P, I32, I32]),
    "st_scene_load_instances": (I32, [P, I32, P, P, P, P, P, I32, P, P, P]),
    "st_scene_set_instance_transforms": (I32, [P, P, I32, I32]),
    "st_scene_set_structure": (I32, [P, I32]),
    "st_scene_serialize": (I32, [P, P, C.POINTER(C.c_size_t)]),
    "st_scene_deserialize": (I32, [P, P, C.c_size_t, C.POINTER(P)]),
    "st_scene_get_geometry": (I32, [P, P, P, P, P, P, P, I32]),
    "st_ray_directions": (I32, [P, I32, I64, P]),
    "st_impulse_response": (I32, [P, P, I32, I32, I32, F64, F64, F64, I32, P, P, I32, I32, P]),
    "st_set_frequency_grid": (I32, [P, I32, P]),
    "st_set_tune": (I32, [P, P]),
    "st_set_stage_overlap": (I32, [P, I32]),
    "st_inject_alloc_failure": (None, [I64]),
    "st_accumulate_specular_noalloc": (I32, [P, P, P, P, P, I64, I32, P, I64, P, I32, I32, F64, F64, I32, I32, P, P, P,
                                             P, P, P]),
}

_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsonotrace.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                               "or `python -m paper_2602_19652_gb300.build`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class SonotraceError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def check(status, ctx=None):
    if status != ST_OK:
        L = load()
        msg = L.st_last_error(ctx).decode() if ctx else L.st_status_string(status).decode()
        raise SonotraceError(status, msg or L.st_status_string(status).decode())
