"""Compile the CUDA library (``csrc/*.cu``) for sm_103a into ``libskmmse.so`` in-tree.

The library is a plain C-ABI shared object (include/skmmse.h); the Python binding
loads it with ctypes.  nvcc cross-compiles without a GPU.
"""
from __future__ import annotations

import os
import subprocess
import sys
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
# SKMMSE_PHASE_CLOCKS=1 in the environment selects the phase-clock diagnostic variant,
# built into its own file so that it never stands in for the release library
PHASE_CLOCKS = os.environ.get("SKMMSE_PHASE_CLOCKS", "0") == "1"
LIB = os.path.join(PKG, "libskmmse_phase.so" if PHASE_CLOCKS else "libskmmse.so")
SOURCES = [os.path.join(CSRC, "skmmse_api.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(INCLUDE, "skmmse.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    with _lock:
        if not force and up_to_date():
            return LIB
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-I" + INCLUDE,
               "-Xcompiler", "-fPIC", "-shared", "-o", tmp] + SOURCES
        if PHASE_CLOCKS:
            cmd.insert(1, "-DSKMMSE_PHASE_CLOCKS")
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed building libskmmse.so")
        if verbose:
            sys.stderr.write(r.stderr)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
