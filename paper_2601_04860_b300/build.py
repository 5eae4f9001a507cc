"""Build step of the CUDA library (nvcc, sm_103a) -- run by ``__graft_entry__.build()``.

Produces ``libdivas_fuse.so`` next to this file.  The flags matter for
numerics: ``-fmad=false`` keeps every multiply-add that is not an explicit
``__fmaf_rn`` unfused, so that all kernels that share the per-vote device
functions round identically; IEEE division and square root are the nvcc
defaults (no fast math).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
SOURCES = ["divas_fuse.cu"]
HEADERS = ["fuse_math.cuh", "tuple_mode.cuh", "weighting.cuh", "select.cuh", "occupancy.cuh", "surfels.cuh", "nerf_mode.cuh", "cull.cuh"]
LIB = os.path.join(HERE, "libdivas_fuse.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC_FLAGS = [
    "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
    "-fmad=false", "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-v",
]


def _inputs():
    files = [os.path.join(SRC_DIR, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "divas_fuse.h"))
    return files


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    tmp = LIB + ".tmp"
    cmd = [nvcc, *NVCC_FLAGS, "-I", INCLUDE, "-o", tmp,
           *[os.path.join(SRC_DIR, f) for f in SOURCES]]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed for libdivas_fuse.so")
    if verbose:
        sys.stderr.write(res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
