"""Build libdem.so (the CUDA DEM library) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2507_12610_gb300/libdem.so.  Host code is compiled without FMA
contraction so host-side set-up arithmetic is the same on x86-64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdem.so")

SOURCES = ["dem_api.cu", "dem_rebuild.cu", "dem_scan.cu", "dem_step.cu", "dem_step_fp64.cu",
           "dem_noalloc.cu", "dem_spawn.cu", "dem_export.cu", "mpnn.cu", "dem_probe.cu"]
# the FP64 step is the precision reference: no multiply-add contraction
# the mixed step uses approximate FP32 division and square root (about 1 ulp);
# its compensated sums use neither
FILE_FLAGS = {"dem_step_fp64.cu": ["--fmad=false"], "dem_noalloc.cu": ["--fmad=false"],
              "dem_spawn.cu": ["--fmad=false"], "dem_export.cu": ["--fmad=false"],
              "dem_step.cu": ["-prec-div=false", "-prec-sqrt=false"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra=(), csrc=CSRC):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE, "-I", csrc,
                   "-Xcompiler", "-fPIC,-ffp-contract=off", "--expt-relaxed-constexpr",
                   *extra]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False,
          extra_flags=(), build_dir: str = BUILD, lib: str = LIB, csrc: str = CSRC) -> str:
    """Compile (if stale) and link libdem.so; extra_flags go to every nvcc call."""
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "dem.h"))
    nv = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        if not os.path.exists(os.path.join(csrc, src)):
            continue
        s = os.path.join(csrc, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or ptxas_info or _stale(o, [s] + headers):
            extra = ((["-Xptxas", "-v"] if ptxas_info else []) + FILE_FLAGS.get(src, [])
                     + list(extra_flags))
            jobs.append([nv, *_flags(extra, csrc), "-c", s, "-o", o])
    outs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                outs.append(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed: {' '.join(j)}\n{r.stdout}\n{r.stderr}")
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    return lib


if __name__ == "__main__":
    import sys
    build(verbose=True, ptxas_info="-v" in sys.argv, force="-f" in sys.argv)
    print(LIB)
