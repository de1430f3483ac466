"""Compile libh2.so in-tree for sm_103a (GB300) with nvcc and g++.

Translation units are compiled in parallel; the host build is compiled without
floating-point contraction so that the admissibility test is evaluated exactly as
written (the same expression the oracle evaluates).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libh2.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr", "-I", INCLUDE] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-I", INCLUDE]

CU_SOURCES = ["h2_device.cu", "h2_noalloc.cu", "h2_cg.cu", "h2_serve.cu", "h2_selftest.cu", "h2_compress.cu"]
CPP_SOURCES = ["h2_host.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libh2")


def _sources():
    cu = [s for s in CU_SOURCES if os.path.exists(os.path.join(CSRC, s))]
    return cu, CPP_SOURCES


def _stale(outputs_mtime: float) -> bool:
    newest = 0.0
    for root, _, files in os.walk(CSRC):
        for f in files:
            newest = max(newest, os.path.getmtime(os.path.join(root, f)))
    newest = max(newest, os.path.getmtime(os.path.join(INCLUDE, "h2.h")), os.path.getmtime(__file__))
    return newest > outputs_mtime


def build(force: bool = False, verbose: bool = False) -> str:
    """Build (if stale) and return the path of libh2.so."""
    if not force and os.path.exists(LIB) and not _stale(os.path.getmtime(LIB)):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp = _sources()
    jobs = []
    for s in cu:
        obj = os.path.join(BUILD, s + ".o")
        jobs.append([nvcc, "-c", os.path.join(CSRC, s), "-o", obj] + NVCC_FLAGS)
    for s in cpp:
        obj = os.path.join(BUILD, s + ".o")
        jobs.append([os.environ.get("CXX", "g++"), "-c", os.path.join(CSRC, s), "-o", obj] + CXX_FLAGS)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for msg in ex.map(run, jobs):
            if verbose and msg:
                print(msg, file=sys.stderr)
    objs = [os.path.join(BUILD, s + ".o") for s in cu + cpp]
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
