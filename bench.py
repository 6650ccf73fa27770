"""Benchmark of the acoustic path-tracing hot path on one GB300 (or N, as independent poses).

Workload (default): the procedural clutter scene -- ground plane + ~200k triangles of icospheres
and cylinders in a 20 x 20 x 5 m volume, 4 materials with 16-band curves, 1M Fibonacci rays,
5 bounces, curvature-based Monte Carlo diffraction (64 samples per high-curvature vertex, 4M
budget), a 32-microphone 12 cm disc array and 512 bins over 20-80 kHz (synthetic, seeded).

One step = one full simulate of one sensor pose through the C ABI: tracing (Algorithm 1),
diffraction sampling and filters, direct path, accumulation of all three spectra.  With
--include-precompute the step also rebuilds the scene (weld, curvature, CDFs, LBVH).

Metric: Mrays/s = (closest-hit + any-hit ray segments traced) / device time, with mic-spectra/s
and the accelerator kernel roofline reported beside it.  Under torchrun every rank simulates its
own pose of the same scene (weak scaling, no collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Mrays/s (closest + any-hit segments/s; spectra <=1e-4 rel-L2 vs oracle)"
UNIT = "Mrays/s"
FLOPS_PER_TERM = 10  # per (path, mic, bin) term: complex rotation (6) + real-by-complex multiply-accumulate (4)
# dram__bytes_read.sum + dram__bytes_write.sum per launch on the clutter workload, from an ncu capture, with the
# hash of the kernel's sources it was taken on: the bench reports it only while the sources still hash to that
# value (else null, until the kernel is captured again).  Specular k_accum: captured on 200k rays (7.98 MB read,
# 0.02 MB written, 163,228 visible records) and scaled to the full-size launch by the visible records (816,192:
# the path list is read once).  k_accum_diff_mma: the full-size diffraction set (21.4 MB read, 0.003 MB written).
ACCUM_TRAFFIC = {"sources_sha16": "3dfb4d8787f86c0b", "specular_bytes_per_launch": 39.9e6}
ACCUM_SOURCES = ("st_accum.cu", "st_accum_dev.cuh", "st_internal.cuh")
DIFF_MMA_TRAFFIC = {"sources_sha16": "3bad1f7281ffc9cd", "bytes_per_launch": 21.4e6}
DIFF_MMA_SOURCES = ("st_accum_mma.cu", "st_accum_dev.cuh", "st_internal.cuh")
# k_accum_narrow on the vegetation workload (two launches a step, specular and diffraction): captured on 500k
# rays (specular 51.75 MB read + 0.14 MB written for 871,268 visible records; diffraction 11.04 MB read for the
# full-size set of 222,807 kept samples), the specular launch scaled to the full-size 6,971,043 records (the
# path list is read once: 414.2 MB), averaged over the step's two launches.
NARROW_TRAFFIC = {"sources_sha16": "90bea9bb00972dd0", "bytes_per_launch": 212.6e6}
NARROW_SOURCES = ("st_accum_narrow.cu", "st_accum_dev.cuh", "st_internal.cuh")


def accum_sources_sha16(files=ACCUM_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2602_19652_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


TENSOR_FLOPS_PER_TERM = 24  # k_accum_diff_mma: a complex multiply-add per term as four real products of bf16
# high/low parts, three each (hi*hi + hi*lo + lo*hi): 4 x 3 x 2 flops


def accum_roofline(stats_list, n_sm, sm_mhz, peak_src, kernel="k_accum (spectrum accumulator)", traffic=None,
                   only_specular=False):
    """FP32 roofline of the accumulator launches of the given simulate steps: 10 flops per (path, mic, bin)
    term over the launches' device time, against 128 FP32 lanes x 2 x the SM clock per SM.  only_specular:
    the specular launch alone (the diffraction launch then runs on the tensor cores, tensor_roofline)."""
    if only_specular:
        acc_ms = sum(s.ms_accum_specular for s in stats_list)
        launches = sum(1 for s in stats_list if s.terms_specular > 0)
        terms = sum(s.terms_specular for s in stats_list)
    else:
        acc_ms = sum(s.ms_accum_kernel for s in stats_list)
        launches = sum(s.accum_launches for s in stats_list)
        terms = sum(s.terms for s in stats_list)
    peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = FLOPS_PER_TERM * terms / (acc_ms / 1e3) / 1e12 if acc_ms > 0 else 0.0
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (max SM clock, {peak_src})",
            "work": f"{FLOPS_PER_TERM} FP32 flops per (path, mic, bin) term, {terms / max(launches, 1):.3e} "
                    f"terms per launch", "ms_per_launch": acc_ms / max(launches, 1), "traffic": traffic}


def tensor_roofline(stats_list, peaks, peak_src):
    """bf16 tensor roofline of the diffraction accumulator on the tensor cores (k_accum_diff_mma): 24 flops
    per (path, mic, bin) term over the launch's device time, against the measured bf16 dense rate."""
    ms = sum(s.ms_accum_diffraction for s in stats_list)
    terms = sum(s.terms_diffraction for s in stats_list)
    launches = sum(1 for s in stats_list if s.terms_diffraction > 0)
    peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = TENSOR_FLOPS_PER_TERM * terms / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    return {"bound": "tensor", "kernel": "k_accum_diff_mma (diffraction accumulator, mma.sync bf16)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": f"bf16 dense, burst ({peak_src})",
            "work": f"{TENSOR_FLOPS_PER_TERM} bf16 tensor flops per (path, mic, bin) term, "
                    f"{terms / max(launches, 1):.3e} terms per launch", "ms_per_launch": ms / max(launches, 1),
            "traffic": DIFF_MMA_TRAFFIC["bytes_per_launch"]
            if DIFF_MMA_TRAFFIC["sources_sha16"] == accum_sources_sha16(DIFF_MMA_SOURCES) else None}


def e2e_simulate(st, ctx, sc, wl, params, n_steps):
    """Seconds and bytes of n_steps simulates through the C ABI with host buffers: the emitter's ray set and
    the receivers copied in from host memory and the spectra returned to host memory by every call."""
    import ctypes as C
    import torch
    L = st.load()
    dirs_h = torch.from_numpy(np.ascontiguousarray(wl.dirs)).pin_memory()
    mics_h = np.ascontiguousarray(wl.mics, np.float32)
    spec_h = np.empty((3, len(wl.mics), wl.n_bins), np.complex64)
    pos = np.ascontiguousarray(wl.emitter, np.float32)
    quat = np.ascontiguousarray(wl.emitter_quat, np.float32)
    cp = lambda a: a.ctypes.data_as(C.c_void_p)
    etab = None if wl.emitter_table is None else np.ascontiguousarray(wl.emitter_table, np.float32)
    mq = None if wl.mic_quats is None else np.ascontiguousarray(wl.mic_quats, np.float32)
    mt = None if wl.mic_tables is None else np.ascontiguousarray(wl.mic_tables, np.float32)

    def one():
        st.check(L.st_set_emitter(ctx.h, cp(pos), cp(quat), len(wl.dirs), C.c_void_p(dirs_h.data_ptr()),
                                  None if etab is None else cp(etab), 0 if etab is None else etab.shape[0],
                                  float(np.float32(wl.fov_half)), st.ST_MEM_HOST), ctx.h)
        st.check(L.st_set_receivers(ctx.h, len(mics_h), cp(mics_h), None if mq is None else cp(mq),
                                    None if mt is None else cp(mt), 0 if mt is None else mt.shape[1],
                                    0 if mt is None else mt.shape[2], 0 if mt is None else mt.shape[3],
                                    st.ST_MEM_HOST), ctx.h)
        st.check(L.st_simulate_host(ctx.h, sc.h, C.byref(params), cp(spec_h), None), ctx.h)

    for _ in range(2):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_steps):
        one()  # each call returns with its spectra on the host
    dt = time.perf_counter() - t0
    h2d = wl.dirs.nbytes + mics_h.nbytes + pos.nbytes + quat.nbytes + sum(
        a.nbytes for a in (etab, mq, mt) if a is not None)
    return dt, int(h2d), int(spec_h.nbytes)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name: str, rank: int):
    if name == "clutter":
        wl = synth.clutter(seed=202)
    elif name == "shoebox":
        wl = synth.shoebox(seed=101)
    elif name == "vegetation":
        wl = synth.vegetation(seed=303)
    else:
        raise SystemExit(f"unknown workload {name}")
    return wl


def workload_config(wl, args):
    return {"workload": f"{wl.name}: {wl.n_tris} triangles, {len(wl.dirs)} rays x {wl.bounces} bounces, "
                        f"{len(wl.mics)} mics, {wl.n_bins} bins {wl.f_lo/1e3:.0f}-{wl.f_hi/1e3:.0f} kHz, "
                        f"diffraction {'on' if wl.diffraction else 'off'}",
            "triangles": wl.n_tris, "rays": len(wl.dirs), "bounces": wl.bounces, "mics": len(wl.mics),
            "bins": wl.n_bins, "diffraction": bool(wl.diffraction),
            "step": "scene precompute + simulate" if args.include_precompute else "simulate (scene prebuilt)",
            "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"{args.gpus} pose(s), one per GPU"}


class ClockSampler:
    """nvidia-smi clocks sampled every 50 ms while running."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for n, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def oracle_sample(wl, n_sample_rays: int, nthreads: int = 0):
    """The oracle as it stands on a bounded sample of the workload: every n-th ray (all mics, all
    bins) and the same fraction of the diffraction candidates.  Returns (segments, seconds, desc)."""
    import oracle
    N = len(wl.dirs)
    stride = max(1, N // n_sample_rays)
    sub = np.arange(0, N, stride)[:n_sample_rays]
    t0 = time.perf_counter()
    scene = oracle.Scene(wl.verts, wl.tris)
    ct_all = cp_all = None
    if wl.diffraction:  # per-scene pre-processing, like the BVH: not part of the timed sample
        G = oracle.curvature(wl.verts, wl.tris)
        Cm = oracle.tri_metric(wl.verts, wl.tris, G)
        cd = oracle.diffraction_cdf(wl.verts, wl.tris, Cm, wl.tri_obj)
        ct_all, cp_all = oracle.diffraction_samples(wl.verts, wl.tris, cd)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    R = oracle.mic_centroid(wl.mics)
    rec = oracle.trace(scene, wl.emitter, wl.emitter_quat, wl.dirs[sub], wl.bounces, r_max=wl.max_distance, R=R,
                       nthreads=nthreads)
    n_rec = int((rec["tri"] >= 0).sum())
    ended_by_miss = int(((rec["tri"] >= 0).sum(1) < wl.bounces).sum())
    segs = n_rec + ended_by_miss + n_rec  # closest queries (hits + final misses) + one visibility ray per hit
    ct = cp = keep = None
    frac = len(sub) / N
    if wl.diffraction:
        ks = np.arange(0, len(ct_all), max(1, int(round(1 / frac))))
        ct, cp = ct_all[ks], cp_all[ks]
        keep = oracle.diffraction_filter(scene, wl.emitter, wl.emitter_quat, ct, cp, fov_half=wl.fov_half,
                                         nthreads=nthreads)
        segs += len(ct)
    dvis = oracle.direct_visibility(scene, wl.emitter, wl.mics)
    segs += len(wl.mics)
    params = oracle.spec_params(wl)
    oracle.spectra(params, rec, wl.dirs[sub], wl.tri_mat, ct, cp, keep, dvis, nthreads=nthreads)
    dt = time.perf_counter() - t0
    desc = (f"every {stride}-th ray ({len(sub)} of {N}) traced with the oracle's BVH (BVH, curvature and CDFs "
            f"{t_build:.1f} s, not timed), 1/{int(round(1 / frac))} of the diffraction candidates, all {len(wl.mics)} mics x "
            f"{wl.n_bins} bins")
    return segs, dt, desc


def over_ranks(dist, world: int, vals_max, vals_sum, device="cpu"):
    """Max over ranks of vals_max and sum over ranks of vals_sum (float64 all-reduces); identity at N = 1."""
    import torch
    if world <= 1:
        return [float(v) for v in vals_max], [float(v) for v in vals_sum]
    a = torch.tensor([float(v) for v in vals_max], dtype=torch.float64, device=device)
    b = torch.tensor([float(v) for v in vals_sum], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.tolist(), b.tolist()


def measure_adjoint(st, torch, wl, steps: int = 5):
    """Device time of one forward simulate and of one st_backward (all gradients) on a workload."""
    ctx = st.Context(torch.cuda.current_device())
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    S = ctx.simulate(sc, p)
    G = torch.randn_like(S.real) + 1j * torch.randn_like(S.real)
    G = G.to(torch.complex64)
    n_mat, n_bands = wl.k_band.shape
    for _ in range(2):
        ctx.simulate(sc, p, out=S)
        ctx.backward(sc, G, n_mat, n_bands)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd, bwd = [], []
    for _ in range(steps):
        ev[0].record(stream)
        ctx.simulate(sc, p, out=S)
        ev[1].record(stream)
        ctx.backward(sc, G, n_mat, n_bands)
        ev[2].record(stream)
        torch.cuda.synchronize()
        fwd.append(ev[0].elapsed_time(ev[1]))
        bwd.append(ev[1].elapsed_time(ev[2]))
    f, b = float(np.median(fwd)), float(np.median(bwd))
    return {"fwd_ms": f, "bwd_ms": b, "bwd_over_fwd": b / f}


def measure_batched(st, torch, rays_per_pose: int = 32768, sample_budget: int = 65536, reps: int = 3,
                    plain_arm: bool = True):
    """Batched form against plain per-pose calls on the pose-sweep workload: 256 sensor poses over 16
    procedural scenes (triangle counts log-uniform 10k-2M, 1-4 materials), 2-64 mics, 256-2048 bins,
    1-5 bounces per pose, diffraction on.  Both arms use the autotuned launch shapes; both are timed
    on the device with L2 flushed before each timed pass."""
    dev = torch.cuda.current_device()
    wls, specs = synth.batched_poses(seed=505)
    ctx = st.Context(dev)
    scenes = []
    for wl in wls:
        sc = st.Scene(ctx, wl.verts, wl.tris, wl.tri_mat, wl.tri_obj)
        sc.set_materials(wl.band_hz, wl.k_band, wl.beta_band, wl.diff_band)
        sc.precompute(st.curv_params(sample_budget=sample_budget))
        scenes.append(sc)
    dirs = synth.fibonacci_directions(rays_per_pose)
    rng = np.random.default_rng(606)
    jobs = []
    for sp in specs:
        q = rng.normal(size=4)
        q = (q / np.linalg.norm(q)).astype(np.float32)
        wl = wls[sp["scene"]]
        jobs.append(st.BatchJob(scenes[sp["scene"]], sp["emitter"], q, dirs, sp["mics"], sp["n_bins"], wl.f_lo, wl.f_hi,
                                sp["bounces"], pose_index=sp["pose_index"], device=dev))
    p = st.sim_params(max_distance=60.0)
    order = np.argsort([j.M * j.F * j.job.max_bounces for j in jobs])
    tune = ctx.autotune(jobs[int(order[len(order) // 2])], p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ms = []
        for i in range(reps):
            flush.fill_(i & 255)
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ms))

    # batched: first call runs eagerly and records the graph; the timed calls replay it
    t0 = time.perf_counter()
    ctx.simulate_batch(jobs, p, tune)
    torch.cuda.synchronize()
    first_call_s = time.perf_counter() - t0
    ctx.simulate_batch(jobs, p, tune)
    batched_ms = timed(lambda: ctx.simulate_batch(jobs, p, tune))
    batched_out = [j.out.clone() for j in jobs]
    if not plain_arm:  # (profiling case: the batched arm alone)
        return {"batched_ms": batched_ms}

    # plain: one st_simulate per pose (sensor inputs already on the device)
    plain_out = [torch.empty_like(j.out) for j in jobs]
    host_pose = [(j.emitter.cpu().numpy(), j.emitter_quat.cpu().numpy()) for j in jobs]
    plain_params = [st.sim_params(max_distance=60.0, max_bounces=j.job.max_bounces, pose_index=j.job.pose_index)
                    for j in jobs]

    def plain():
        for j, o, (e, q), pp in zip(jobs, plain_out, host_pose, plain_params):
            ctx.set_frequencies(j.F, j.job.f_lo, j.job.f_hi)
            ctx.set_emitter(e, q, j.dirs, None, math.pi)
            ctx.set_receivers(j.mics)
            ctx.simulate(j.scene, pp, out=o)

    plain()
    plain_ms = timed(plain)
    err = 0.0
    for a, b in zip(batched_out, plain_out):
        for c in range(3):
            nb = float(torch.linalg.vector_norm(b[c]))
            if nb > 0:
                err = max(err, float(torch.linalg.vector_norm(a[c] - b[c])) / nb)
    n_rays = sum(j.N for j in jobs)
    n_spec = sum(j.M for j in jobs)
    return {"workload": f"{len(jobs)} poses over {len(scenes)} scenes ({min(w.n_tris for w in wls)}-"
                        f"{max(w.n_tris for w in wls)} triangles), {rays_per_pose} rays per pose, "
                        f"diffraction budget {sample_budget} per scene",
            "tune": {"rays_per_block": tune.rays_per_block, "mic_pairs_per_cta": tune.mic_pairs_per_cta,
                     "smem_kb": tune.smem_kb},
            "batched_ms": batched_ms, "plain_ms": plain_ms, "speedup": plain_ms / batched_ms,
            "batched_mrays_per_s": n_rays / batched_ms / 1e3, "plain_mrays_per_s": n_rays / plain_ms / 1e3,
            "batched_mic_spectra_per_s": n_spec / batched_ms * 1e3, "plain_mic_spectra_per_s": n_spec / plain_ms * 1e3,
            "max_rel_l2_batched_vs_plain": err, "first_call_s": first_call_s}


def measure_batched_directional(st, torch, n_poses: int = 64, rays_per_pose: int = 32768, reps: int = 3,
                                plain_arm: bool = True):
    """Batched form against plain per-pose calls on bat poses with directivity (Sec. III-F): a 200k-triangle
    leaf-disc scene, n_poses head poses near the centre (random headings; the ears at +-1 cm across the
    head, oriented with it), the piston emitter table and two ear tables, 1024 bins 20-120 kHz, 4 bounces,
    diffraction on (65,536 samples), field of view pi/2.  Plain calls set the pose's emitter (with its table)
    and receivers (with theirs) from device memory and simulate; L2 flushed before each timed pass."""
    dev = torch.cuda.current_device()
    wl = synth.vegetation(seed=303, target_tris=200_000, n_rays=rays_per_pose, bounces=4, n_bins=1024,
                          leaves_per_mesh=256)
    ctx = st.Context(dev)
    sc = st.Scene(ctx, wl.verts, wl.tris, wl.tri_mat, wl.tri_obj)
    sc.set_materials(wl.band_hz, wl.k_band, wl.beta_band, wl.diff_band)
    sc.precompute(st.curv_params(sample_budget=65536))
    rng = np.random.default_rng(808)
    d = f"cuda:{dev}"
    etab = torch.as_tensor(wl.emitter_table, device=d)
    mtab = torch.as_tensor(wl.mic_tables, device=d)
    dirs = torch.as_tensor(wl.dirs, device=d)
    fov = float(np.float32(math.pi / 2))
    jobs, poses = [], []
    for i in range(n_poses):
        q = rng.normal(size=4)
        q = (q / np.linalg.norm(q)).astype(np.float32)
        w, x, y, z = (float(v) for v in q)
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        e = rng.uniform(-0.1, 0.1, 3).astype(np.float32)
        mics = (e + (R @ np.array([[0.0, 0.01, 0.0], [0.0, -0.01, 0.0]]).T).T).astype(np.float32)
        mq = np.tile(q, (2, 1)).astype(np.float32)
        jobs.append(st.BatchJob(sc, e, q, dirs, mics, wl.n_bins, wl.f_lo, wl.f_hi, wl.bounces, pose_index=i,
                                fov_half=fov, device=dev, emitter_table=etab, mic_quats=mq, mic_tables=mtab))
        poses.append((torch.as_tensor(e, device=d), torch.as_tensor(q, device=d), torch.as_tensor(mics, device=d),
                      torch.as_tensor(mq, device=d)))
    p = st.sim_params(max_distance=wl.max_distance)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=d)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ms = []
        for i in range(reps):
            flush.fill_(i & 255)
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ms))

    ctx.simulate_batch(jobs, p)
    ctx.simulate_batch(jobs, p)
    batched_ms = timed(lambda: ctx.simulate_batch(jobs, p))
    batched_out = [j.out.clone() for j in jobs]
    if not plain_arm:  # (profiling case: the batched arm alone)
        return {"batched_ms": batched_ms}
    plain_out = [torch.empty_like(j.out) for j in jobs]
    pp = [st.sim_params(max_distance=wl.max_distance, max_bounces=wl.bounces, pose_index=i) for i in range(n_poses)]
    ctx.set_frequencies(wl.n_bins, wl.f_lo, wl.f_hi)

    def plain():
        for i, (e, q, m, mq) in enumerate(poses):
            ctx.set_emitter(e, q, dirs, etab, fov)
            ctx.set_receivers(m, mq, mtab)
            ctx.simulate(sc, pp[i], out=plain_out[i])

    plain()
    plain_ms = timed(plain)
    err = 0.0
    for a, b in zip(batched_out, plain_out):
        for c in range(3):
            nb = float(torch.linalg.vector_norm(b[c]))
            if nb > 0:
                err = max(err, float(torch.linalg.vector_norm(a[c] - b[c])) / nb)
    ctx.close()
    return {"workload": f"{n_poses} bat poses in a {wl.n_tris}-triangle leaf-disc scene, {rays_per_pose} rays x "
                        f"{wl.bounces} bounces, 2 ears x {wl.n_bins} bins, piston emitter and ear tables, diffraction "
                        f"65536 samples",
            "batched_ms": batched_ms, "plain_ms": plain_ms, "speedup": plain_ms / batched_ms,
            "max_rel_l2_batched_vs_plain": err}


def measure_emitters(st, torch, ctx, sc, wl, n_emitters: int = 4, reps: int = 3):
    """Several emitters sending the workload's ray set into its scene towards its array: one batched call
    (Context.simulate_emitters) against one plain st_simulate per emitter (set_emitter + simulate, the
    sensor inputs on the device).  Emitters within 0.5 m of the sensor, random orientations, one pose
    index; L2 flushed before each timed pass; both arms' spectra compared."""
    dev = torch.cuda.current_device()
    rng = np.random.default_rng(707)
    E = (wl.emitter + rng.uniform(-0.5, 0.5, (n_emitters, 3)) * np.array([1.0, 1.0, 0.2])).astype(np.float32)
    Q = rng.normal(size=(n_emitters, 4))
    Q = (Q / np.linalg.norm(Q, axis=1, keepdims=True)).astype(np.float32)
    dirs = torch.as_tensor(wl.dirs, device=f"cuda:{dev}")
    p = st.sim_params(max_distance=wl.max_distance)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ms = []
        for i in range(reps):
            flush.fill_(i & 255)
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ms))

    def batched():
        return ctx.simulate_emitters(sc, E, Q, dirs, wl.mics, wl.n_bins, wl.f_lo, wl.f_hi, wl.bounces, p)

    t0 = time.perf_counter()
    batched()  # first call: eager run and graph recording
    torch.cuda.synchronize()
    first_call_s = time.perf_counter() - t0
    batched_ms = timed(batched)
    out_b = batched().clone()
    outs = torch.empty_like(out_b)
    pp = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    ctx.set_frequencies(wl.n_bins, wl.f_lo, wl.f_hi)
    ctx.set_receivers(wl.mics)

    def plain():
        for e in range(n_emitters):
            ctx.set_emitter(E[e], Q[e], dirs, None, wl.fov_half)
            ctx.simulate(sc, pp, out=outs[e])

    plain()
    plain_ms = timed(plain)
    err = max(float(torch.linalg.vector_norm(out_b[e, c] - outs[e, c]) / torch.linalg.vector_norm(outs[e, c]))
              for e in range(n_emitters) for c in range(3) if float(torch.linalg.vector_norm(outs[e, c])) > 0)
    ctx.set_emitter(wl.emitter, wl.emitter_quat, wl.dirs, wl.emitter_table, wl.fov_half)
    n_rays = n_emitters * len(wl.dirs)
    return {"workload": f"{n_emitters} emitters x {len(wl.dirs)} rays x {wl.bounces} bounces into the {wl.name} scene, "
                        f"{len(wl.mics)} mics x {wl.n_bins} bins, diffraction on",
            "batched_ms": batched_ms, "plain_ms": plain_ms, "speedup": plain_ms / batched_ms,
            "batched_emitter_rays_per_s": n_rays / (batched_ms / 1e3), "first_call_s": first_call_s,
            "max_rel_l2_batched_vs_plain": err}


def measure_instances(st, torch, n_inst: int = 8000, n_rays: int = 1_000_000, reps: int = 3):
    """Instanced forest (shared plant meshes under affine maps, expanded on the device), in both scene
    structures (one BVH over the expanded triangles; per-prototype BVHs under a BVH over the instances):
    host time of st_scene_load_instances (checks, upload of prototypes and instance table, expansion),
    device times of the precompute, of moving every plant (new maps, expansion and refit or rebuild of the
    top level; keeping the curvature, as the moves are rotations and translations, and recomputing it) and
    of one simulate, the device memory the built scene holds, and the bytes uploaded against those of the
    same scene loaded flat."""
    dev = torch.cuda.current_device()
    fo = synth.instanced_forest(seed=606, n_inst=n_inst, n_rays=n_rays, bounces=3, n_mics=8, n_bins=128)
    b = fo.base
    ctx = st.Context(dev)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ms = []
        for i in range(reps):
            ev[0].record(stream)
            fn(i)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ms))

    curv = st.curv_params(sample_budget=1_000_000)
    rng = np.random.default_rng(8)
    X = fo.inst_xform.astype(np.float64)
    moved = X.copy()
    for i in range(1, n_inst):  # every plant turned about the vertical and shifted
        a = rng.uniform(-0.2, 0.2)
        R = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
        moved[i, :, :3] = R @ X[i, :, :3]
        moved[i, :2, 3] += rng.uniform(-0.05, 0.05, 2)
    poses = [torch.as_tensor(m.astype(np.float32), device=f"cuda:{dev}") for m in (moved, X)]
    ctx.set_frequencies(b.n_bins, b.f_lo, b.f_hi)
    ctx.set_emitter(b.emitter, b.emitter_quat, b.dirs)
    ctx.set_receivers(b.mics)
    p = st.sim_params(max_bounces=b.bounces, max_distance=b.max_distance)
    out = torch.empty((3, len(b.mics), b.n_bins), dtype=torch.complex64, device=f"cuda:{dev}")
    res, spectra = {}, []
    for two_level in (False, True):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        t0 = time.perf_counter()
        sc = st.Scene.from_instances(ctx, fo.protos, fo.inst_proto, fo.inst_xform)
        load_s = time.perf_counter() - t0
        sc.set_materials(b.band_hz, b.k_band, b.beta_band, b.diff_band)
        if two_level:
            sc.set_structure(True)
        precompute_ms = timed(lambda i: sc.precompute(curv))
        torch.cuda.synchronize()
        scene_bytes = free0 - torch.cuda.mem_get_info(dev)[0]
        move_keep_ms = timed(lambda i: sc.set_instance_transforms(poses[i & 1], keep_curvature=True))
        move_full_ms = timed(lambda i: sc.set_instance_transforms(poses[i & 1]))
        sc.set_instance_transforms(poses[1])
        ctx.simulate(sc, p, out=out)
        stats = []
        sim_ms = timed(lambda i: stats.append(ctx.simulate(sc, p, out=out, stats=True)[1]))
        spectra.append(out.cpu().numpy())
        segs = stats[-1].closest_queries + stats[-1].shadow_queries
        r = {"load_instances_s": load_s, "precompute_ms": precompute_ms, "move_refit_keep_curvature_ms": move_keep_ms,
             "move_refit_ms": move_full_ms, "simulate_ms": sim_ms, "value": segs / (sim_ms / 1e3) / 1e6, "unit": UNIT,
             "scene_device_bytes": int(scene_bytes)}
        if two_level:
            res["two_level"] = r
        else:
            pv = sum(len(q[0]) for q in fo.protos)
            pt = sum(len(q[1]) for q in fo.protos)
            res.update({"workload": f"instanced forest: {n_inst} instances of {len(fo.protos)} meshes, {sc.n_tris} "
                                    f"triangles, {n_rays} rays x {b.bounces} bounces, {len(b.mics)} mics x {b.n_bins} "
                                    f"bins, diffraction on",
                        **r, "upload_bytes_instanced": int(pv * 12 + pt * 16 + n_inst * 52 + (len(fo.protos) + 1) * 16),
                        "upload_bytes_flat": int(sc.n_verts * 12 + sc.n_tris * 20)})
        sc.close()
    res["two_level"]["spectra_equal_to_flat"] = bool(np.array_equal(spectra[0], spectra[1]))
    ctx.close()
    return res


def measure_workload(st, torch, wl, steps: int = 3, warmup: int = 2, los_mode: int = 0, roofline=None, e2e=False,
                     traffic=None):
    """Device time of one simulate on another workload (scene prebuilt, L2 flushed before each step);
    los_mode 1: the receiver test of every hit made per microphone.  roofline = (n_sm, sm_mhz, peak_src):
    also the accumulator's FP32 roofline; e2e: also the end-to-end rate through host buffers."""
    dev = torch.cuda.current_device()
    ctx = st.Context(dev)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, los_mode=los_mode)
    out = torch.empty((3, len(wl.mics), wl.n_bins), dtype=torch.complex64, device=f"cuda:{dev}")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.simulate(sc, p, out=out)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ms, segs, stats, all_stats = [], 0, None, []
    for i in range(steps):
        flush.fill_(i & 255)
        ev[0].record(stream)
        _, stats = ctx.simulate(sc, p, out=out, stats=True)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]))
        segs += stats.closest_queries + stats.shadow_queries
        all_stats.append(stats)
    t = float(sum(ms))
    res = {"config": f"{wl.name}: {wl.n_tris} triangles, {len(wl.dirs)} rays x {wl.bounces} bounces, "
                     f"{len(wl.mics)} mics, {wl.n_bins} bins, diffraction {'on' if wl.diffraction else 'off'}",
           "value": segs / (t / 1e3) / 1e6, "unit": UNIT, "ms_per_step": t / steps,
           "mic_spectra_per_s": len(wl.mics) * steps / (t / 1e3),
           "ms_trace": stats.ms_trace, "ms_diffraction": stats.ms_diffraction, "ms_accumulate": stats.ms_accumulate,
           "visible_records": stats.visible_records, "diffraction_kept": stats.candidates_kept,
           "anyhit_segments": stats.shadow_queries}
    if roofline is not None:
        n_sm, sm_mhz, peak_src = roofline
        kern = "k_accum_narrow (one microphone pair)" if len(wl.mics) <= 2 else "k_accum (spectrum accumulator)"
        res["roofline"] = accum_roofline(all_stats, n_sm, sm_mhz, peak_src, kernel=kern, traffic=traffic)
    if e2e:
        n = max(3, steps)
        dt, h2d, d2h = e2e_simulate(st, ctx, sc, wl, p, n)
        res["e2e"] = {"value": segs / steps * n / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * dt / n}
    ctx.close()
    return res


def l2_probe_gbs(torch, mb: int = 40, reps: int = 50):
    """Copy bandwidth with both buffers resident in L2 (2 x 40 MB < 129 MB): read + write bytes over the
    device time of back-to-back copies.  A torch copy kernel, so a lower bound on the L2 peak."""
    n = mb * (1 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    for _ in range(5):
        b.copy_(a)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(reps):
        b.copy_(a)
    ev[1].record()
    torch.cuda.synchronize()
    return 2.0 * a.numel() * 4 * reps / (ev[0].elapsed_time(ev[1]) / 1e3) / 1e9


def measure_traversal(st, torch, wl, ms_trace: float, ms_diffraction: float, hbm_gbs: float):
    """BVH fetch bandwidth of the tracing kernels: 4-wide nodes (112 B read of 128) and leaf triangles (48 B) visited,
    counted in a separate instrumented run (ST_COUNT_VISITS), divided by the uninstrumented kernel
    times of the headline steps.  The fetches are served mostly by L1/L2 (the node array of the
    benchmark scene fits in L2), so the ratio to the HBM copy bandwidth can exceed 1."""
    dev = torch.cuda.current_device()
    os.environ["ST_COUNT_VISITS"] = "1"
    try:
        ctx = st.Context(dev)
    finally:
        del os.environ["ST_COUNT_VISITS"]
    sc = st.from_workload(ctx, wl)
    p_spec = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, components=st.ST_COMP_SPECULAR)
    p_all = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    _, s_spec = ctx.simulate(sc, p_spec, stats=True)
    _, s_all = ctx.simulate(sc, p_all, stats=True)
    torch.cuda.synchronize()
    vs = list(s_spec.visits)
    va = list(s_all.visits)
    vd = [a - b for a, b in zip(va, vs)]  # diffraction filters and the direct path (any-hit only)
    bt = 112 * (vs[0] + vs[2]) + 48 * (vs[1] + vs[3])
    bd = 112 * (vd[0] + vd[2]) + 48 * (vd[1] + vd[3])
    ctx.close()
    q_t = s_spec.closest_queries + s_spec.shadow_queries
    q_d = (s_all.shadow_queries - s_spec.shadow_queries)
    l2 = l2_probe_gbs(torch)
    ft, fd = bt / (ms_trace / 1e3) / 1e9, bd / (ms_diffraction / 1e3) / 1e9
    return {"bytes_per_node": 112, "bytes_per_triangle": 48, "l2_probe_gbs": l2,
            "frac_of_l2_probe": {"bounces": ft / l2, "diffraction": fd / l2},
            "bounces": {"kernels": "k_closest + k_shade + k_visible (records), all bounces",
                        "queries": int(q_t), "nodes": int(vs[0] + vs[2]), "triangles": int(vs[1] + vs[3]),
                        "nodes_per_query": (vs[0] + vs[2]) / max(q_t, 1), "ms": ms_trace,
                        "fetch_gbs": ft},
            "diffraction": {"kernels": "k_diffraction + k_visible (line of sight to the emitter)",
                            "queries": int(q_d), "nodes": int(vd[0] + vd[2]), "triangles": int(vd[1] + vd[3]),
                            "nodes_per_query": (vd[0] + vd[2]) / max(q_d, 1), "ms": ms_diffraction,
                            "fetch_gbs": fd}}


def measure_signal(st, torch, ctx, S, wl, reps: int = 5):
    """Received signals of the headline spectra: all three components summed, convolved with a 1 ms
    chirp over the band, sampled at 2.5 x the top frequency over one period 1 / df of the response
    (a spectrum sampled every df gives a response periodic in 1 / df)."""
    fs = 2.5 * wl.f_hi
    period = (wl.n_bins - 1) / (wl.f_hi - wl.f_lo)
    n = int(math.ceil(min(wl.max_distance / 343.0, period) * fs))
    t = np.arange(int(1e-3 * fs)) / fs
    call = np.sin(2 * np.pi * (wl.f_hi * t - 0.5 * (wl.f_hi - wl.f_lo) / 1e-3 * t * t)).astype(np.float32)
    call_d = torch.from_numpy(call).cuda()
    for _ in range(2):
        ctx.impulse_response(S, wl.f_lo, wl.f_hi, fs, n, call=call_d)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    stream = torch.cuda.current_stream()
    ev[0].record(stream)
    for _ in range(reps):
        ctx.impulse_response(S, wl.f_lo, wl.f_hi, fs, n, call=call_d)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    M, F = int(S.shape[1]), int(S.shape[2])
    flops = 10.0 * M * n * F  # per (mic, sample, bin): rotation 6 + real part of the product 4
    return {"config": f"{M} mics x {F} bins -> {n} samples at {fs / 1e3:.0f} kHz, {len(call)}-sample chirp",
            "ms": ms, "msamples_per_s": M * n / ms / 1e3, "tflops": flops / (ms / 1e3) / 1e12}


def measure_scene_update(st, torch, ctx, sc, wl, reps: int = 3):
    """Device time of a full precompute (weld, curvature, CDFs, LBVH, wide nodes) against a refit of new
    vertex positions (same topology), with and without recomputing the curvature and CDFs."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    stream = torch.cuda.current_stream()
    v = wl.verts.astype(np.float64)
    moved = (v + 0.01 * np.sin(v[:, [1, 2, 0]])).astype(np.float32)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ms))

    res = {"precompute_ms": timed(lambda: sc.precompute()),
           "refit_ms": timed(lambda: sc.update_vertices(moved)),
           "refit_keep_curvature_ms": timed(lambda: sc.update_vertices(moved, keep_curvature=True))}
    sc.update_vertices(wl.verts)
    sc.precompute()
    return res


def run_case(st, torch, case: str, reps: int):
    """Small cases of single kernels for profiling (ncu captures): no timing output; "emitters" and
    "instances" print their measurement alone."""
    dev = torch.cuda.current_device()
    if case == "instances":
        print(json.dumps(measure_instances(st, torch)))
        return
    if case == "batched_bat":
        print(json.dumps(measure_batched_directional(st, torch)))
        return
    if case == "batched":
        print(json.dumps(measure_batched(st, torch)))
        return
    if case == "batched_bat_only":  # the batched arm alone (launch lists)
        print(json.dumps(measure_batched_directional(st, torch, plain_arm=False)))
        return
    if case == "batched_only":
        print(json.dumps(measure_batched(st, torch, plain_arm=False)))
        return
    if case == "emitters":
        wl = synth.clutter(seed=202)
        ctx = st.Context(dev)
        sc = st.from_workload(ctx, wl)
        print(json.dumps(measure_emitters(st, torch, ctx, sc, wl)))
        return
    if case in ("accum", "adjoint", "trace", "trace_per_mic"):
        wl = synth.clutter(seed=202, n_rays=200_000)
    elif case == "narrow":
        wl = synth.vegetation(seed=303, n_rays=500_000)
    else:
        raise SystemExit(f"unknown case {case}")
    ctx = st.Context(dev)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance,
                      los_mode=st.ST_LOS_PER_MIC if case == "trace_per_mic" else st.ST_LOS_REFERENCE)
    S = ctx.simulate(sc, p)
    if case == "adjoint":
        G = (torch.randn_like(S.real) + 1j * torch.randn_like(S.real)).to(torch.complex64)
        n_mat, n_bands = wl.k_band.shape
        for _ in range(reps):
            ctx.backward(sc, G, n_mat, n_bands)
    else:
        for _ in range(reps):
            ctx.simulate(sc, p, out=S)
    torch.cuda.synchronize()
    print(f"case {case}: {wl.name}, {len(wl.dirs)} rays, {reps} repetitions")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload, 0)
    cores = os.cpu_count()
    times, segs_all = [], []
    desc = ""
    for i in range(args.warmup + args.steps):
        segs, dt, desc = oracle_sample(wl, args.ref_rays)
        if i >= args.warmup:
            times.append(dt)
            segs_all.append(segs)
    value = sum(segs_all) / sum(times) / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 geometry, f64 spectra", "data": "synthetic",
            "impl": "reference", "config": workload_config(wl, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _r(x, n=4):
    """x rounded to n significant digits (floats only)."""
    if isinstance(x, float) and x != 0.0 and math.isfinite(x):
        return round(x, n - 1 - int(math.floor(math.log10(abs(x)))))
    return x


def compact_line(d):
    """The headline line: the contract's keys, with every other part of the metric (backward / forward
    time, batched vs plain, the vegetation workload's rate, roofline and end-to-end rate) in short form."""
    rf = d["roofline"]
    line = {k: d[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                              "higher_is_better", "scaling", "vs_baseline", "dtype", "data")}
    line["value"], line["ms_per_step"] = _r(line["value"], 6), _r(line["ms_per_step"], 5)
    c = d["config"]
    line["config"] = {"workload": f"{c['workload'].split(':')[0]}: {c['triangles']} tris, {c['rays']} rays x "
                                  f"{c['bounces']} bounces, {c['mics']} mics x {c['bins']} bins"
                                  f"{', diffraction' if c['diffraction'] else ''}",
                      "step": c["step"], "l2": "flushed (256 MiB write)", "parallelism": c["parallelism"]}
    line["roofline"] = {"bound": rf["bound"], "kernel": rf["kernel"].split(" ")[0], "achieved": _r(rf["achieved"]),
                        "peak": _r(rf["peak"]), "unit": rf["unit"], "frac": _r(rf["frac"]), "traffic": rf["traffic"]}
    rd = d.get("roofline_diffraction")
    if rd:
        line["roofline_diffraction"] = {"bound": rd["bound"], "kernel": rd["kernel"].split(" ")[0],
                                        "achieved": _r(rd["achieved"]), "peak": _r(rd["peak"]), "unit": rd["unit"],
                                        "frac": _r(rd["frac"], 4), "traffic": rd["traffic"]}
    cb = d.get("cpu_baseline")
    if cb:
        line["cpu_baseline"] = {"value": _r(cb["value"]), "unit": cb["unit"], "cores": cb["cores"],
                                "kind": cb["kind"], "sample": cb["sample_short"]}
    else:
        line["cpu_baseline"] = None
    e = d["e2e"]
    line["e2e"] = {"value": _r(e["value"]), "unit": e["unit"], "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                   "d2h_bytes_per_step": e["d2h_bytes_per_step"]}
    ck = d["clocks"]
    line["clocks"] = {"sm_mhz": ck.get("sm_mhz"), "sm_max_mhz": ck.get("sm_max_mhz"), "reasons": ck.get("reasons")}
    line["gpu_launches"] = d["gpu_launches"]
    line["mic_spectra_per_s"] = _r(d["mic_spectra_per_s"])
    if d.get("adjoint"):
        line["bwd_over_fwd"] = {("gradient" if k.startswith("gradient") else k.split(" ")[0]): _r(v["bwd_over_fwd"], 3)
                                for k, v in d["adjoint"].items()}
    if d.get("batched"):
        b = d["batched"]
        line["batched_vs_plain"] = {"speedup": _r(b["speedup"], 3), "batched_ms": _r(b["batched_ms"]),
                                    "plain_ms": _r(b["plain_ms"]), "poses": 256}
    if d.get("batched_directional"):
        b = d["batched_directional"]
        line["batched_vs_plain_bat"] = {"speedup": _r(b["speedup"], 3), "batched_ms": _r(b["batched_ms"]),
                                        "plain_ms": _r(b["plain_ms"]), "poses": 64}
    v = d.get("vegetation")
    if v:
        vr, ve = v["roofline"], v["e2e"]
        line["vegetation"] = {"value": _r(v["value"]), "ms_per_step": _r(v["ms_per_step"]),
                              "roofline": {"bound": vr["bound"], "kernel": vr["kernel"].split(" ")[0],
                                           "achieved": _r(vr["achieved"]), "peak": _r(vr["peak"]),
                                           "unit": vr["unit"], "frac": _r(vr["frac"]), "traffic": vr["traffic"]},
                              "e2e": {"value": _r(ve["value"]), "unit": ve["unit"],
                                      "h2d_bytes_per_step": ve["h2d_bytes_per_step"],
                                      "d2h_bytes_per_step": ve["d2h_bytes_per_step"]}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clutter")
    ap.add_argument("--include-precompute", action="store_true")
    ap.add_argument("--cpu-rays", type=int, default=16384, help="rays in the oracle's CPU-baseline sample")
    ap.add_argument("--ref-rays", type=int, default=2048, help="rays per step of the reference (oracle) arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the forward/backward timing")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain pose sweep")
    ap.add_argument("--no-per-mic", action="store_true", help="skip the per-microphone receiver-test timing")
    ap.add_argument("--no-vegetation", action="store_true", help="skip the full-size vegetation simulate timing")
    ap.add_argument("--no-emitters", action="store_true", help="skip the several-emitters timing")
    ap.add_argument("--no-instances", action="store_true", help="skip the instanced-forest timing")
    ap.add_argument("--case", default=None,
                    choices=["accum", "adjoint", "trace", "trace_per_mic", "narrow", "emitters", "instances", "batched_bat",
                             "batched", "batched_bat_only", "batched_only"],
                    help="run a small case of one kernel family a few times and exit (for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_2602_19652_gb300 as st

    if args.case:
        return run_case(st, torch, args.case, max(args.steps, 1))

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = workload(args.workload, rank)
    ctx = st.Context(local)
    sc = st.from_workload(ctx, wl)
    params = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, pose_index=rank)
    out = torch.empty((3, len(wl.mics), wl.n_bins), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(stats=True):
        if args.include_precompute:
            sc.precompute()
        return ctx.simulate(sc, params, out=out, stats=stats)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    st_list = []
    peaks, peak_src = load_peaks()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 255)                       # evict L2 between steps (outside the timed events)
            ev[i][0].record(stream)
            _, s = step()
            ev[i][1].record(stream)
            st_list.append(s)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    segs = sum(s.closest_queries + s.shadow_queries for s in st_list)
    # max over ranks of the time, sum of the work
    (total_ms_all,), (segs_all, spectra_all) = over_ranks(dist, world, [total_ms],
                                                          [segs, len(wl.mics) * args.steps], dev)
    value = segs_all / (total_ms_all / 1e3) / 1e6

    # ---- dominant kernel: the accumulator (FP32-pipe arithmetic)
    clocks = clk.summary()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    tensor_diff = all(s.diffraction_tensor for s in st_list)
    traffic = (ACCUM_TRAFFIC["specular_bytes_per_launch"]
               if tensor_diff and ACCUM_TRAFFIC["sources_sha16"] == accum_sources_sha16() else None)
    roofline = accum_roofline(st_list, n_sm, sm_mhz, peak_src, traffic=traffic,
                              kernel="k_accum (specular accumulator)" if tensor_diff else
                              "k_accum (spectrum accumulator)", only_specular=tensor_diff)
    roofline_diffraction = tensor_roofline(st_list, peaks, peak_src) if tensor_diff else None

    # ---- end to end through the C ABI with host buffers
    if world > 1:
        dist.barrier()
    n_e2e = max(3, args.steps // 2)
    if args.include_precompute:
        sc.precompute()
    t_e2e, h2d, d2h = e2e_simulate(st, ctx, sc, wl, params, n_e2e)
    (t_e2e_max,), (segs_e2e,) = over_ranks(dist, world, [t_e2e], [segs / len(st_list) * n_e2e], dev)
    e2e = {"value": segs_e2e / t_e2e_max / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": 1e3 * t_e2e_max / n_e2e}

    # the remaining measurements run on rank 0 alone
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # each stage's own device time, with the stages issued in order on one stream (in the timed steps the
    # diffraction stage and the direct path run on a side stream beside the trace); the traversal fetch
    # rates divide by these
    ctx.set_stage_overlap(False)
    serial = []
    for i in range(3):
        flush.fill_(i & 255)
        serial.append(step()[1])
    torch.cuda.synchronize()
    ctx.set_stage_overlap(True)
    stages_serial = {k: float(np.median([getattr(s, k) for s in serial]))
                     for k in ("ms_trace", "ms_diffraction", "ms_accumulate", "ms_total")}
    signal = measure_signal(st, torch, ctx, out, wl)
    scene_update = measure_scene_update(st, torch, ctx, sc, wl)
    traversal = measure_traversal(st, torch, wl, stages_serial["ms_trace"], stages_serial["ms_diffraction"],
                                  peaks["hbm_gbs"])
    adjoint = None
    if not args.no_adjoint:
        adjoint = {"gradient workload (shoebox, 4 materials x 16 bands, 32 mics, 128 bins, 10k rays x 3)":
                   measure_adjoint(st, torch, synth.gradient_problem(seed=404)),
                   f"{wl.name} workload": measure_adjoint(st, torch, wl)}

    batched = batched_dir = None
    if not args.no_batched:
        batched = measure_batched(st, torch)
        batched_dir = measure_batched_directional(st, torch)
    vegetation = None
    if not args.no_vegetation and args.workload != "vegetation":
        veg_traffic = (NARROW_TRAFFIC["bytes_per_launch"]
                       if NARROW_TRAFFIC["sources_sha16"] == accum_sources_sha16(NARROW_SOURCES) else None)
        vegetation = measure_workload(st, torch, synth.vegetation(seed=303), roofline=(n_sm, sm_mhz, peak_src),
                                      e2e=True, traffic=veg_traffic)
    per_mic = None
    if not args.no_per_mic and len(wl.mics) <= 64:
        per_mic = measure_workload(st, torch, wl, los_mode=st.ST_LOS_PER_MIC)
    emitters = None
    if not args.no_emitters and wl.emitter_table is None and wl.mic_tables is None:
        emitters = measure_emitters(st, torch, ctx, sc, wl)
    instances = None
    if not args.no_instances:
        instances = measure_instances(st, torch)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        segs_c, dt_c, desc = oracle_sample(wl, args.cpu_rays)
        cpu = {"value": segs_c / dt_c / 1e6, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": desc,
               "seconds": dt_c,
               "sample_short": f"1/{max(1, len(wl.dirs) // args.cpu_rays)} of the rays and diffraction samples, "
                               f"all mics x bins, {dt_c:.1f} s"}

    s0 = st_list[-1]
    detail = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (float-float r and phase)",
            "data": "synthetic", "config": workload_config(wl, args),
            "mic_spectra_per_s": spectra_all / (total_ms_all / 1e3),
            "per_step": {"closest_segments": s0.closest_queries, "anyhit_segments": s0.shadow_queries,
                         "visible_records": s0.visible_records, "diffraction_candidates": s0.candidates,
                         "diffraction_kept": s0.candidates_kept, "terms": s0.terms,
                         "ms_trace": s0.ms_trace, "ms_diffraction": s0.ms_diffraction,
                         "ms_accumulate": s0.ms_accumulate,
                         "stages": "diffraction stage and direct path on a side stream beside the trace; the "
                                   "specular accumulation after both"},
            "stages_serial": stages_serial,
            "roofline": roofline, "roofline_diffraction": roofline_diffraction, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "adjoint": adjoint,
            "traversal": traversal, "signal": signal, "scene_update": scene_update, "batched": batched, "batched_directional": batched_dir,
            "vegetation": vegetation, "receiver_test_per_mic": per_mic, "emitters": emitters,
            "instances": instances,
            "gpu_launches": int(sum(s.kernel_launches for s in st_list))}
    # every measurement in full on stderr; stdout carries one compact line (the headline with the
    # figures of the metric's other parts), short enough to be kept whole by a reader of the last 1.5 kB
    print("bench detail " + json.dumps(detail), file=sys.stderr)
    print(json.dumps(compact_line(detail), separators=(",", ":")))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
