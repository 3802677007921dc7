"""Build the CUDA library in-tree: ``libfem_b300.so`` next to this file.

Everything is compiled for sm_103a only (B300); nvcc cross-compiles without a
GPU.  The shared library has a plain C ABI (``include/fem_b300.h``).  Each
source is compiled to its own object (in parallel, under ``_build/`` at the
repository root) and the objects are linked into the library.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(ROOT, "_build", "obj")
LIB = os.path.join(HERE, "libfem_b300.so")
SOURCES = ["fem_plan.cpp", "fem_api.cu", "fem_solver.cu", "fem_learned.cu", "fem_sparse.cu", "fem_spmv.cu", "fem_atomic.cu",
           "fem_ncm.cu", "fem_calib.cu"]
HEADERS = ["fem_plan.h", "fem_kernels.cuh", "fem_pair.cuh", "fem_material.cuh", "fem_vec.cuh", "fem_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    return [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _headers():
    files = [os.path.join(CSRC, h) for h in HEADERS if os.path.exists(os.path.join(CSRC, h))]
    files.append(os.path.join(ROOT, "include", "fem_b300.h"))
    return files


def _inputs():
    return _sources() + _headers()


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _flags():
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
            "-Xcompiler", "-pthread", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    t_hdr = max(os.path.getmtime(h) for h in _headers())
    jobs = []
    objs = []
    for src in _sources():
        obj = os.path.join(OBJ, os.path.basename(src) + ".o")
        objs.append(obj)
        stale = force or extra or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), t_hdr)
        if stale:
            jobs.append([_nvcc(), *_flags(), "-c", src, "-o", obj + ".tmp", *(extra or [])])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(cmd[-1 - len(extra or [])], cmd[-1 - len(extra or [])][:-4])

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(run, j) for j in jobs]:
            f.result()
    cmd = [_nvcc(), *ARCH, "-shared", "-Xcompiler", "-pthread", "-o", LIB + ".tmp", *objs]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
    print(LIB)
