"""Builds libgputx.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; the shared library links against
the shared CUDA runtime so that it and PyTorch use one runtime instance.
``build(debug=True)`` builds libgputx_debug.so instead, with -DGPUTX_DEBUG:
the same engine with a bounds check on every index its executors gather or
scatter by (a failed check fails the bulk with GPUTX_EBOUNDS).  The binding
loads it when GPUTX_DEBUG=1 is set in the environment.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgputx.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libgputx_debug.so")
SOURCES = ["api.cu", "analysis.cu", "exec.cu", "exec_dc.cu", "tables.cu", "serve.cu", "batch.cu", "pool.cu", "relaxed.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(home, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _flags():
    return ARCH + ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                   "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]


def _stale(outputs, inputs):
    if not all(os.path.exists(o) for o in outputs):
        return True
    newest = max(os.path.getmtime(i) for i in inputs)
    return min(os.path.getmtime(o) for o in outputs) < newest


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    BUILD, LIB = (BUILD_DEBUG, LIB_DEBUG) if debug else (globals()["BUILD"], globals()["LIB"])
    flags = _flags() + (["-DGPUTX_DEBUG"] if debug else [])
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "gputx.h"))
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale([o], [s] + headers):
            jobs.append([_nvcc()] + flags + ["-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, fu in zip(jobs, futs):
                r = fu.result()
                if verbose or r.returncode:
                    print(" ".join(j))
                    print(r.stdout, r.stderr)
                if r.returncode:
                    raise RuntimeError(f"nvcc failed for {j[-3]}")
    if force or jobs or _stale([LIB], objs):
        cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            print(" ".join(cmd), r.stdout, r.stderr)
            raise RuntimeError("link failed")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
