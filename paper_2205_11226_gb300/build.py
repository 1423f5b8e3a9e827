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
LIB_RELEASE = os.path.join(PKG, "libskmmse.so")
LIB_PHASE = os.path.join(PKG, "libskmmse_phase.so")
LIB = LIB_PHASE if PHASE_CLOCKS else LIB_RELEASE
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


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d))


def _compile(lib: str, phase: bool, verbose: bool) -> subprocess.Popen:
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-I" + INCLUDE,
           "-Xcompiler", "-fPIC", "-shared", "-o", tmp] + SOURCES
    if phase:
        cmd.insert(1, "-DSKMMSE_PHASE_CLOCKS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)


def build(force: bool = False, verbose: bool = False, phase: bool | None = None,
          both: bool = False) -> str:
    """Compile the library selected by SKMMSE_PHASE_CLOCKS (or `phase`); `both` also
    compiles the other variant, in parallel.  Returns the selected library's path."""
    phase = PHASE_CLOCKS if phase is None else phase
    lib = LIB_PHASE if phase else LIB_RELEASE
    with _lock:
        todo = [(lib, phase)]
        if both:
            todo.append((LIB_RELEASE if phase else LIB_PHASE, not phase))
        todo = [(l, ph) for l, ph in todo if force or not up_to_date(l)]
        procs = [(l, _compile(l, ph, verbose)) for l, ph in todo]
        failed = []
        for l, pr in procs:
            out, err = pr.communicate()
            tmp = l + f".{os.getpid()}.tmp"
            if pr.returncode != 0:
                sys.stderr.write(out + err)
                failed.append(os.path.basename(l))
                continue
            if verbose:
                sys.stderr.write(err)
            os.replace(tmp, l)
        if failed:
            raise RuntimeError("nvcc failed building " + ", ".join(failed))
        return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
