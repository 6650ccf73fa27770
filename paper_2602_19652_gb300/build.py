"""Build libsonotrace.so (sm_103a) in-tree with nvcc: one object per translation unit, compiled in
parallel, then linked.  Geometry units are compiled with -fmad=false so their float32 results are
the same bits as any IEEE-754 implementation taking the same steps; host code is compiled without
floating-point contraction for the same reason (GCC contracts a*b+c by default on aarch64)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsonotrace.so")
# the bounds-checked build (-DST_CHECKS: indices read from device data are checked before use, a failed
# check is reported as ST_ERR_CUDA); same sources, its own output folder
OUT_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(OUT_CHECKS, "libsonotrace.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE]
# translation unit -> extra flags
UNITS = {
    "st_api.cu": ["-fmad=false", "-Xcompiler", "-fvisibility=default"],
    "st_sort.cu": [],
    "st_scene.cu": ["-fmad=false"],
    "st_trace.cu": ["-fmad=false"],
    "st_batch.cu": ["-fmad=false"],
    "st_accum.cu": [],
    "st_accum_mma.cu": [],
    "st_accum_narrow.cu": [],
    "st_adjoint.cu": [],
    "st_noalloc.cu": [],
    "st_signal.cu": [],
    "st_rays.cu": ["-fmad=false"],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _sources_newer(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "sonotrace.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, checks: bool = False) -> str:
    out, lib = (OUT_CHECKS, LIB_CHECKS) if checks else (OUT, LIB)
    os.makedirs(out, exist_ok=True)
    if not force and not _sources_newer(lib):
        return lib
    cc = nvcc()
    extra = ["-DST_CHECKS"] if checks else []

    def compile_one(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(out, unit.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *extra, *UNITS[unit], "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath", "-Xlinker", "/usr/local/cuda/lib64"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checks="--checks" in sys.argv))
