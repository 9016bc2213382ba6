"""Builds libefgp.so (the CUDA library behind include/efgp.h) in-tree.

Every translation unit is compiled for sm_103a only, in parallel, and linked
with the static CUDA runtime so the library depends on nothing but the NVIDIA driver.
Run ``python -m paper_2210_10210_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libefgp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["api.cu", "fft.cu", "cg.cu", "cg_persistent.cu", "cg_queue.cu", "cg_grid.cu", "setup_fused.cu", "spread.cu", "interp.cu", "predict_noalloc.cu"]
CPP_SOURCES = ["host_params.cpp"]


def _nvcc() -> str:
    cand = [os.environ.get("NVCC", ""), shutil.which("nvcc") or "", "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libefgp")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, jobs: int | None = None) -> str:
    """Compile the library if any source is newer than it; returns its path."""
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "efgp.h"))
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    jobs_list = []
    objs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs_list.append([nvcc, *ARCH, "-lineinfo", *common, "--expt-relaxed-constexpr", "-c", s, "-o", o])
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs_list.append([nvcc, *common, "-x", "c++", "-c", s, "-o", o])
    if jobs_list:
        n = jobs or min(len(jobs_list), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            outs = list(ex.map(_run, jobs_list))
        if verbose:
            for o in outs:
                if o.strip():
                    print(o)
    if force or jobs_list or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", "-lpthread", "-ldl", "-lrt"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
