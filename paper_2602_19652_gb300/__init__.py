"""GB300 acoustic path tracing (SonoTraceUE hot path, arXiv 2602.19652) -- Python binding.

Thin wrapper over the C ABI of libsonotrace (include/sonotrace.h).  PyTorch provides device
memory and the current CUDA stream; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: without the built library or a GPU the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib
from .autograd import SpectraFn  # noqa: E402
from ._lib import (ST_COMP_DIFFRACTION, ST_COMP_DIRECT, ST_COMP_SPECULAR, ST_ERR_ARG, ST_ERR_MESH, ST_ERR_OOM,
                   ST_ERR_OVERFLOW, ST_ERR_STATE, ST_LOS_PER_MIC, ST_LOS_REFERENCE, ST_MEM_DEVICE, ST_MEM_HOST, CurvParams,
                   Job, SimParams, SonotraceError, Stats, Tune, check, load)

__all__ = ["Context", "Scene", "BatchJob", "SpectraFn", "CurvParams", "SimParams", "Stats", "Tune", "SonotraceError",
           "sim_params", "curv_params", "ST_COMP_SPECULAR", "ST_COMP_DIFFRACTION", "ST_COMP_DIRECT",
           "ST_LOS_REFERENCE", "ST_LOS_PER_MIC", "ST_ERR_ARG", "ST_ERR_MESH", "ST_ERR_STATE"]


def curv_params(**kw) -> CurvParams:
    p = CurvParams()
    load().st_curv_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def sim_params(**kw) -> SimParams:
    p = SimParams()
    load().st_sim_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _dev(t, dtype):
    t = torch.as_tensor(t, dtype=dtype, device="cuda").contiguous()
    return t


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Context:
    """One library context on one GPU, issuing work on a CUDA stream (default: torch's current)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.L = load()
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        h = C.c_void_p()
        check(self.L.st_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream)))
        self.h = h
        self._keep = []
        self.M = self.F = 0
        self.N = 0

    def close(self):
        """Destroys the context and every scene still loaded into it."""
        if getattr(self, "h", None):
            self.L.st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        check(status, self.h)

    # -------------------------------------------------------------- inputs
    def set_frequencies(self, n_bins: int, f_lo: float, f_hi: float):
        self._check(self.L.st_set_frequencies(self.h, int(n_bins), float(f_lo), float(f_hi)))
        self.F = int(n_bins)

    def set_frequency_grid(self, f_hz):
        """The frequency bins as an ascending, uniformly spaced array (Hz)."""
        f = np.ascontiguousarray(f_hz, dtype=np.float32).reshape(-1)
        self._check(self.L.st_set_frequency_grid(self.h, int(len(f)), f.ctypes.data_as(C.c_void_p)))
        self.F = int(len(f))

    def set_emitter(self, pos, quat, dirs, table=None, fov_half: float = math.pi):
        self.quat, self.dirs, self.fov_half = quat, dirs, fov_half
        # every pointer of the call in device memory, as ST_MEM_DEVICE says
        pos = _dev(pos, torch.float32).reshape(3).contiguous()
        quat = _dev(quat, torch.float32).reshape(4).contiguous()
        d = _dev(dirs, torch.float32)
        tab = None if table is None else _dev(table, torch.float32)
        self._check(self.L.st_set_emitter(self.h, _ptr(pos), _ptr(quat),
                                          int(d.shape[0]), _ptr(d), None if tab is None else _ptr(tab),
                                          0 if tab is None else int(tab.shape[0]), float(np.float32(fov_half)),
                                          ST_MEM_DEVICE))
        self.N = int(d.shape[0])

    def set_receivers(self, mics, quats=None, tables=None):
        """tables: [M][n_el][n_az][n_bands] receiver directivity on the materials' bands (None = omni)."""
        m = _dev(mics, torch.float32)
        q = None if quats is None else _dev(quats, torch.float32)
        t = None if tables is None else _dev(tables, torch.float32)
        n_el, n_az, nb = (0, 0, 0) if t is None else tuple(int(x) for x in t.shape[1:4])
        self._check(self.L.st_set_receivers(self.h, int(m.shape[0]), _ptr(m), None if q is None else _ptr(q),
                                            None if t is None else _ptr(t), n_el, n_az, nb, ST_MEM_DEVICE))
        self.M = int(m.shape[0])

    # -------------------------------------------------------------- simulate
    def simulate(self, scene: "Scene", params: SimParams | None = None, out: torch.Tensor | None = None,
                 stats: bool = False):
        """Returns complex64 [3][M][F] spectra on the device (specular, diffraction, direct)."""
        if out is None:
            out = torch.empty((3, self.M, self.F), dtype=torch.complex64, device=f"cuda:{self.device}")
        st = Stats() if stats else None
        self._check(self.L.st_simulate(self.h, scene.h, None if params is None else C.byref(params), _ptr(out),
                                       None if st is None else C.byref(st)))
        return (out, st) if stats else out

    def simulate_host(self, scene: "Scene", params: SimParams | None = None, out: np.ndarray | None = None):
        if out is None:
            out = np.empty((3, self.M, self.F), dtype=np.complex64)
        self._check(self.L.st_simulate_host(self.h, scene.h, None if params is None else C.byref(params),
                                            out.ctypes.data_as(C.c_void_p), None))
        return out

    def paths(self, B: int):
        N = self.N
        tri = np.empty((N, B), np.int32)
        p = np.empty((N, B, 3), np.float32)
        d = np.empty((N, B, 3), np.float32)
        r = np.empty((N, B), np.float64)
        los = np.empty((N, B), np.uint8)
        cp = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(self.L.st_get_paths(self.h, cp(tri), cp(p), cp(d), cp(r), cp(los), ST_MEM_HOST))
        return dict(tri=tri, p=p, d=d, r=r, los=los)

    def receiver_masks(self, B: int):
        """[N][B] uint64 per-microphone visibility of the last simulate (made with ST_LOS_PER_MIC)."""
        m = np.empty((self.N, B), np.uint64)
        self._check(self.L.st_get_receiver_masks(self.h, m.ctypes.data_as(C.c_void_p), ST_MEM_HOST))
        return m

    def diffraction(self):
        n = C.c_int64(0)
        self._check(self.L.st_get_diffraction(self.h, C.byref(n), None, None, None, 0, ST_MEM_HOST))
        K = n.value
        tri = np.empty(max(K, 1), np.int32)
        p = np.empty((max(K, 1), 3), np.float32)
        keep = np.empty(max(K, 1), np.uint8)
        cp = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(self.L.st_get_diffraction(self.h, C.byref(n), cp(tri), cp(p), cp(keep), K, ST_MEM_HOST))
        return tri[:K], p[:K], keep[:K]

    def backward(self, scene: "Scene", grad_spectra: torch.Tensor, n_mat: int, n_bands: int):
        """(dL/dk [n_mat][n_bands], dL/dmic [M][3], dL/demitter [3]) for grad_spectra = dL/dRe S + j dL/dIm S."""
        dev = grad_spectra.device
        g = grad_spectra.contiguous().to(torch.complex64)
        gk = torch.zeros((n_mat, n_bands), dtype=torch.float32, device=dev)
        gm = torch.zeros((self.M, 3), dtype=torch.float32, device=dev)
        ge = torch.zeros(3, dtype=torch.float32, device=dev)
        vp = lambda t: C.c_void_p(t.data_ptr())
        self._check(self.L.st_backward(self.h, scene.h, vp(g), vp(gk), vp(gm), vp(ge)))
        return gk, gm, ge

    def backward_beta(self, scene: "Scene", grad_spectra: torch.Tensor, n_mat: int, n_bands: int):
        """dL/dbeta [n_mat][n_bands] (lobe widths of the specular paths) for grad_spectra = dL/dRe S + j dL/dIm S."""
        g = grad_spectra.contiguous().to(torch.complex64)
        gb = torch.zeros((n_mat, n_bands), dtype=torch.float32, device=g.device)
        self._check(self.L.st_backward_beta(self.h, scene.h, C.c_void_p(g.data_ptr()), C.c_void_p(gb.data_ptr())))
        return gb

    def direct_visibility(self):
        v = np.empty(self.M, np.uint8)
        self._check(self.L.st_get_direct_visibility(self.h, v.ctypes.data_as(C.c_void_p), ST_MEM_HOST))
        return v

    # -------------------------------------------------------------- ray sets
    def ray_directions(self, n: int, kind: str = "zonal") -> torch.Tensor:
        """float32 [n][3] emitter-frame directions on the device: "zonal" (the paper's equal-area set)
        or "fibonacci"."""
        k = {"fibonacci": _lib.ST_RAYS_FIBONACCI, "zonal": _lib.ST_RAYS_ZONAL}[kind]
        out = torch.empty((int(n), 3), dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.L.st_ray_directions(self.h, k, int(n), C.c_void_p(out.data_ptr())))
        return out

    # -------------------------------------------------------------- signals
    def impulse_response(self, spectra: torch.Tensor, f_lo: float, f_hi: float, fs: float, n_samples: int,
                         window: torch.Tensor | None = None, call: torch.Tensor | None = None,
                         per_component: bool = False) -> torch.Tensor:
        """Band-limited impulse responses (or received signals, with the emitted `call` sampled at fs) of
        spectra [C][M][F]: float32 [M][n_samples] (components summed) or [C][M][n_samples]."""
        S = spectra.contiguous()
        if S.dim() == 2:
            S = S.unsqueeze(0)
        Cn, M, F = (int(x) for x in S.shape)
        dev = S.device
        w = None if window is None else window.to(device=dev, dtype=torch.float32).contiguous()
        e = None if call is None else call.to(device=dev, dtype=torch.float32).contiguous()
        out = torch.empty((Cn, M, n_samples) if per_component else (M, n_samples), dtype=torch.float32, device=dev)
        vp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._check(self.L.st_impulse_response(self.h, vp(S), Cn, M, F, float(f_lo), float(f_hi), float(fs),
                                               int(n_samples), vp(w), vp(e), 0 if e is None else int(e.numel()),
                                               _lib.ST_IR_PER_COMPONENT if per_component else 0, vp(out)))
        return out

    # -------------------------------------------------------------- batched form
    def simulate_batch(self, jobs: list["BatchJob"], params: SimParams | None = None, tune: Tune | None = None):
        """All jobs' spectra (each job's .out).  Same job list and sizes on a later call replays the
        recorded graph; update the jobs' pose tensors in place (BatchJob.set_pose) between calls."""
        key = tuple(id(j) for j in jobs)
        if getattr(self, "_batch_key", None) != key:
            self._batch_arr = (Job * len(jobs))(*[j.job for j in jobs])
            self._batch_key = key
            self._batch_jobs = list(jobs)
        self._check(self.L.st_simulate_batch(self.h, len(jobs), self._batch_arr,
                                             None if params is None else C.byref(params),
                                             None if tune is None else C.byref(tune)))
        return [j.out for j in jobs]

    def simulate_emitters(self, scene: "Scene", emitters, emitter_quats, dirs, mics, n_bins: int, f_lo: float,
                          f_hi: float, max_bounces: int, params: SimParams | None = None, pose_index: int = 0,
                          fov_half: float = math.pi) -> torch.Tensor:
        """Several emitters (positions [S][3], orientations [S][4]) sending the same ray set into one scene
        towards one receiver array, in one batched call: complex64 [S][3][M][F], emitter s's specular,
        diffraction and direct spectra (the sum over s is the array's spectra when all emitters send the
        same call).  Every emitter filters the same diffraction samples (one pose index).  The jobs share
        the ray and microphone tensors and are kept, so a later call with the same sizes replays the
        recorded graph with the new emitter poses.  Omni emitters and receivers, as in simulate_batch."""
        dev = f"cuda:{self.device}"
        E = np.ascontiguousarray(emitters, np.float32).reshape(-1, 3)
        Q = np.ascontiguousarray(emitter_quats, np.float32).reshape(-1, 4)
        if len(E) != len(Q) or len(E) == 0:
            raise ValueError("simulate_emitters: one orientation per emitter, at least one emitter")
        src_d = torch.as_tensor(dirs, dtype=torch.float32)
        src_m = torch.as_tensor(mics, dtype=torch.float32)
        key = (scene.h.value, len(E), tuple(src_d.shape), tuple(src_m.shape), int(n_bins), float(f_lo),
               float(f_hi), int(max_bounces), int(pose_index), float(np.float32(fov_half)))
        with torch.cuda.stream(self.stream):  # the copies are ordered before the library's work
            if getattr(self, "_emit_key", None) != key:
                # the context's own copies of the rays and microphones, shared by the jobs
                d = torch.empty(tuple(src_d.shape), dtype=torch.float32, device=dev)
                m = torch.empty(tuple(src_m.shape), dtype=torch.float32, device=dev)
                d.copy_(src_d)
                m.copy_(src_m)
                self._emit_jobs = [BatchJob(scene, E[i], Q[i], d, m, n_bins, f_lo, f_hi, max_bounces,
                                            pose_index=pose_index, fov_half=fov_half, device=self.device)
                                   for i in range(len(E))]
                self._emit_key, self._emit_refs = key, (d, m)
            else:
                d, m = self._emit_refs
                d.copy_(src_d)
                m.copy_(src_m)
                for i, j in enumerate(self._emit_jobs):
                    j.set_pose(emitter=E[i], emitter_quat=Q[i])
            return torch.stack(self.simulate_batch(self._emit_jobs, params))

    def set_tune(self, rays_per_block: int = 0, mic_pairs_per_cta: int = 0, smem_kb: int = 0, stack_depth: int = 0,
                 refill_lanes: int = 0, bins_per_thread: int = 0):
        """Launch shapes of later simulate calls (0 = the library's default for each)."""
        t = Tune(rays_per_block, mic_pairs_per_cta, smem_kb, stack_depth, refill_lanes, bins_per_thread)
        self._check(self.L.st_set_tune(self.h, C.byref(t)))

    def set_stage_overlap(self, on: bool):
        """Diffraction stage and direct path beside the trace on a side stream (default), or every stage in
        order on the context's stream (stage times that do not overlap); the results are the same."""
        self._check(self.L.st_set_stage_overlap(self.h, 1 if on else 0))

    def autotune(self, job: "BatchJob", params: SimParams | None = None) -> Tune:
        t = Tune()
        self._check(self.L.st_autotune(self.h, C.byref(job.job), None if params is None else C.byref(params),
                                       C.byref(t)))
        self.M, self.F, self.N = job.M, job.F, job.N
        return t


class BatchJob:
    """One pose of a batch: device tensors for the pose (updated in place between calls) and the
    job's output, complex64 [3][M][F]."""

    def __init__(self, scene: "Scene", emitter, emitter_quat, dirs, mics, n_bins: int, f_lo: float, f_hi: float,
                 max_bounces: int, pose_index: int = 0, fov_half: float = math.pi, device: int = 0,
                 emitter_table=None, mic_quats=None, mic_tables=None):
        """emitter_table [n_theta][n_bins], mic_quats [M][4], mic_tables [M][n_el][n_az][n_bands]: directivity
        as Context.set_emitter / set_receivers take it (None: omni)."""
        dev = f"cuda:{device}"
        self.scene = scene

        def f32(x):  # a float32 device tensor on this device is used as it is (jobs may share rays, mics)
            if isinstance(x, torch.Tensor):
                return x.to(device=dev, dtype=torch.float32).contiguous()
            return torch.as_tensor(np.asarray(x, np.float32), device=dev).contiguous()

        self.emitter = f32(emitter)
        self.emitter_quat = f32(emitter_quat)
        self.dirs = f32(dirs)
        self.mics = f32(mics)
        self.N, self.M, self.F = int(self.dirs.shape[0]), int(self.mics.shape[0]), int(n_bins)
        self.out = torch.empty((3, self.M, self.F), dtype=torch.complex64, device=dev)
        vp = lambda t: C.c_void_p(t.data_ptr())
        self.job = Job(scene=scene.h, emitter=vp(self.emitter), emitter_quat=vp(self.emitter_quat), dirs=vp(self.dirs),
                       n_rays=self.N, mics=vp(self.mics), n_mics=self.M, n_bins=self.F, f_lo=float(f_lo),
                       f_hi=float(f_hi), max_bounces=int(max_bounces), pose_index=int(pose_index),
                       fov_half_rad=float(np.float32(fov_half)), spectra_out=vp(self.out))
        self.emitter_table = None if emitter_table is None else f32(emitter_table)
        self.mic_quats = None if mic_quats is None else f32(mic_quats)
        self.mic_tables = None if mic_tables is None else f32(mic_tables)
        if self.emitter_table is not None:
            self.job.dir_table = vp(self.emitter_table)
            self.job.n_theta = int(self.emitter_table.shape[0])
        if self.mic_quats is not None:
            self.job.mic_quats = vp(self.mic_quats)
        if self.mic_tables is not None:
            self.job.mic_tables = vp(self.mic_tables)
            self.job.n_el, self.job.n_az = int(self.mic_tables.shape[1]), int(self.mic_tables.shape[2])

    def set_pose(self, emitter=None, emitter_quat=None, mics=None):
        """Copy a new pose into the job's tensors (same shapes), stream-ordered on torch's current stream."""
        for dst, src in ((self.emitter, emitter), (self.emitter_quat, emitter_quat), (self.mics, mics)):
            if src is not None:
                dst.copy_(torch.as_tensor(np.asarray(src, np.float32)), non_blocking=False)


class Scene:
    """A triangle scene owned by a Context: load, set materials, precompute (BVH, curvature, CDFs)."""

    def __init__(self, ctx: Context, verts, tris, tri_mat, tri_obj, _handle=None):
        self.ctx = ctx
        if _handle is not None:  # made by from_instances
            self.h = _handle
            return
        v = np.ascontiguousarray(verts, np.float32)
        t = np.ascontiguousarray(tris, np.int32)
        m = np.ascontiguousarray(tri_mat, np.int32)
        o = np.ascontiguousarray(tri_obj, np.int32)
        h = C.c_void_p()
        cp = lambda a: a.ctypes.data_as(C.c_void_p)
        ctx._check(ctx.L.st_scene_load(ctx.h, cp(v), len(v), cp(t), len(t), cp(m), cp(o), ST_MEM_HOST, C.byref(h)))
        self.h = h
        self.n_verts, self.n_tris = len(v), len(t)
        self.n_obj = int(o.max()) + 1

    def set_materials(self, band_hz, k, beta, diffr):
        self.band_hz, self.k_band, self.beta_band, self.diff_band = band_hz, k, beta, diffr
        b = np.ascontiguousarray(band_hz, np.float32)
        k = np.ascontiguousarray(k, np.float32)
        be = np.ascontiguousarray(beta, np.float32)
        d = np.ascontiguousarray(diffr, np.float32)
        cp = lambda a: a.ctypes.data_as(C.c_void_p)
        self.ctx._check(self.ctx.L.st_scene_set_materials(self.h, k.shape[0], k.shape[1], cp(b), cp(k), cp(be), cp(d)))

    def precompute(self, params: CurvParams | None = None):
        self.ctx._check(self.ctx.L.st_scene_precompute(self.h, None if params is None else C.byref(params)))

    def update_vertices(self, verts, keep_curvature: bool = False):
        """New positions for the same vertices, then a refit of the precomputed scene (see the C header)."""
        v = np.ascontiguousarray(verts, np.float32)
        assert v.shape == (self.n_verts, 3)
        self.ctx._check(self.ctx.L.st_scene_update_vertices(self.h, v.ctypes.data_as(C.c_void_p), ST_MEM_HOST,
                                                            _lib.ST_REFIT_KEEP_CURVATURE if keep_curvature else 0))

    @classmethod
    def from_instances(cls, ctx: Context, protos, inst_proto, inst_xform) -> "Scene":
        """A scene of instances of shared meshes: protos = [(verts [v][3], tris [t][3] local indices,
        tri_mat [t]), ...], inst_proto [n_inst] prototype ids, inst_xform [n_inst][3][4] row-major [A | b]
        (x -> A x + b).  Expanded on the device; instance i is object i."""
        pv = np.ascontiguousarray(np.concatenate([np.asarray(p[0], np.float32).reshape(-1, 3) for p in protos]))
        pt = np.ascontiguousarray(np.concatenate([np.asarray(p[1], np.int32).reshape(-1, 3) for p in protos]))
        pm = np.ascontiguousarray(np.concatenate([np.asarray(p[2], np.int32).reshape(-1) for p in protos]))
        voff = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(np.asarray(p[0]).reshape(-1, 3)) for p in protos])]),
                                    np.int64)
        toff = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(np.asarray(p[1]).reshape(-1, 3)) for p in protos])]),
                                    np.int64)
        ip = np.ascontiguousarray(inst_proto, np.int32).reshape(-1)
        xf = np.ascontiguousarray(inst_xform, np.float32).reshape(-1, 12)
        cp = lambda a: a.ctypes.data_as(C.c_void_p)
        h = C.c_void_p()
        ctx._check(ctx.L.st_scene_load_instances(ctx.h, len(protos), cp(voff), cp(pv), cp(toff), cp(pt), cp(pm), len(ip),
                                                 cp(ip), cp(xf), C.byref(h)))
        sc = cls(ctx, None, None, None, None, _handle=h)
        nv, nt = C.c_int64(0), C.c_int64(0)
        ctx._check(ctx.L.st_scene_get_geometry(h, C.byref(nv), C.byref(nt), None, None, None, None, ST_MEM_HOST))
        sc.n_verts, sc.n_tris, sc.n_obj, sc.n_inst = nv.value, nt.value, len(ip), len(ip)
        return sc

    def set_instance_transforms(self, inst_xform, keep_curvature: bool = False):
        """New instance transforms [n_inst][3][4] (numpy or a device tensor), then a refit (see the C header)."""
        if isinstance(inst_xform, torch.Tensor):
            x = inst_xform.to(dtype=torch.float32).contiguous()
            assert x.numel() == 12 * self.n_inst and x.is_cuda
            ptr_, mem = C.c_void_p(x.data_ptr()), ST_MEM_DEVICE
        else:
            x = np.ascontiguousarray(inst_xform, np.float32)
            assert x.size == 12 * self.n_inst
            ptr_, mem = x.ctypes.data_as(C.c_void_p), ST_MEM_HOST
        self.ctx._check(self.ctx.L.st_scene_set_instance_transforms(
            self.h, ptr_, mem, _lib.ST_REFIT_KEEP_CURVATURE if keep_curvature else 0))

    def serialize(self) -> bytes:
        """Host blob of the precomputed scene (checkpoint; see the C header)."""
        n = C.c_size_t(0)
        self.ctx._check(self.ctx.L.st_scene_serialize(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self.ctx._check(self.ctx.L.st_scene_serialize(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    @classmethod
    def deserialize(cls, ctx: Context, blob: bytes) -> "Scene":
        """A precomputed scene of ctx from a blob of Scene.serialize (resume; no precompute needed)."""
        h = C.c_void_p()
        buf = C.create_string_buffer(bytes(blob), len(blob))
        ctx._check(ctx.L.st_scene_deserialize(ctx.h, buf, len(blob), C.byref(h)))
        sc = cls(ctx, None, None, None, None, _handle=h)
        nv, nt = C.c_int64(0), C.c_int64(0)
        ctx._check(ctx.L.st_scene_get_geometry(h, C.byref(nv), C.byref(nt), None, None, None, None, ST_MEM_HOST))
        sc.n_verts, sc.n_tris = nv.value, nt.value
        o = np.empty(sc.n_tris, np.int32)
        ctx._check(ctx.L.st_scene_get_geometry(h, None, None, None, None, None, o.ctypes.data_as(C.c_void_p),
                                               ST_MEM_HOST))
        sc.n_obj = int(o.max()) + 1
        return sc

    def set_structure(self, two_level: bool):
        """Hierarchy of an instanced scene: one BVH over the expanded triangles (two_level=False, the default)
        or per-prototype BVHs in object space under a BVH over the instances (see the C header)."""
        self.ctx._check(self.ctx.L.st_scene_set_structure(
            self.h, _lib.ST_STRUCTURE_TWO_LEVEL if two_level else _lib.ST_STRUCTURE_FLAT))

    def geometry(self):
        """(verts [V][3], tris [T][3], tri_mat [T], tri_obj [T]) of the scene as loaded or expanded."""
        v = np.empty((self.n_verts, 3), np.float32)
        t = np.empty((self.n_tris, 3), np.int32)
        m = np.empty(self.n_tris, np.int32)
        o = np.empty(self.n_tris, np.int32)
        cp = lambda a: a.ctypes.data_as(C.c_void_p)
        self.ctx._check(self.ctx.L.st_scene_get_geometry(self.h, None, None, cp(v), cp(t), cp(m), cp(o), ST_MEM_HOST))
        return v, t, m, o

    def curvature(self):
        G = np.empty(self.n_verts, np.float32)
        Cm = np.empty(self.n_tris, np.float32)
        ns = np.empty(self.n_obj, np.int64)
        cp = lambda a: a.ctypes.data_as(C.c_void_p)
        self.ctx._check(self.ctx.L.st_scene_get_curvature(self.h, cp(G), cp(Cm), cp(ns), ST_MEM_HOST))
        return G, Cm, ns

    def close(self):
        # a destroyed context has already freed its scenes
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            self.ctx.L.st_scene_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(ctx: Context, wl, curv: CurvParams | None = None) -> Scene:
    """Load a synthetic workload's scene and sensor into ctx (scene precomputed)."""
    sc = Scene(ctx, wl.verts, wl.tris, wl.tri_mat, wl.tri_obj)
    sc.set_materials(wl.band_hz, wl.k_band, wl.beta_band, wl.diff_band)
    sc.precompute(curv)
    ctx.set_frequencies(wl.n_bins, wl.f_lo, wl.f_hi)
    ctx.set_emitter(wl.emitter, wl.emitter_quat, wl.dirs, wl.emitter_table, wl.fov_half)
    ctx.set_receivers(wl.mics, wl.mic_quats, wl.mic_tables)
    return sc
