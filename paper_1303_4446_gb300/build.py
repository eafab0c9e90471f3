"""In-tree build of the CUDA library (sm_103a) and the workload integral generator.

    python -m paper_1303_4446_gb300.build          # builds what is out of date
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libx2c_gb300.so")
SOURCES = ["abi.cu", "solve.cu", "assemble.cu", "host.cu", "split.cu", "noalloc.cu", "serve.cu", "integrals.cu"]
HEADERS = ["common.cuh", "gemm_f64.cuh", "umma.cuh", "split_int.cuh", "serve_policy.h", "integrals_math.cuh",
           "solve_fw.cuh", "dkh_plan.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(ROOT, "include"), "-diag-suppress", "177"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _mtime(p):
    return os.path.getmtime(p) if os.path.exists(p) else -1.0


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu into _build/ in parallel and link libx2c_gb300.so (if stale)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    dep_time = max(_mtime(os.path.join(CSRC, h)) for h in HEADERS)
    dep_time = max(dep_time, _mtime(os.path.join(ROOT, "include", "x2c.h")))
    jobs = []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        if force or _mtime(obj) < max(_mtime(sp), dep_time):
            jobs.append([_nvcc()] + NVCC_FLAGS + ["-c", sp, "-o", obj])
    objs = [os.path.join(BUILD_DIR, s.replace(".cu", ".o")) for s in SOURCES]

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _mtime(LIB_PATH) < max(_mtime(o) for o in objs):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        run([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def build_all(force: bool = False, verbose: bool = False):
    from .workload import build_ints_library
    build_ints_library(force=force)
    return build_library(force=force, verbose=verbose)


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv, verbose=True))
