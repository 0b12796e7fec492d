"""Compile libpn (the CUDA kernels and the C ABI) for sm_103a, in-tree.

``python -m paper_1801_07986_b300.build`` or :func:`build_library` writes
``paper_1801_07986_b300/libpn.so`` next to this file.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(CSRC, f) for f in ("pn_kernels.cu", "pn_order.cu", "pn_deriv.cu", "pn_api.cu", "pn_noalloc.cu",
                                           "pn_peaks.cu")]
HEADERS = [os.path.join(CSRC, "pn_internal.h"), os.path.join(CSRC, "pn_device.cuh"),
           os.path.join(os.path.dirname(HERE), "include", "pn.h")]
LIB = os.path.join(HERE, "libpn.so")
# the debug build: kernels check their global-memory indices (PN_DEBUG_CHECKS)
DEBUG_LIB = os.path.join(HERE, "libpn_debug.so")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-shared", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in SOURCES + HEADERS)


def build_library(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile libpn.so (or, with debug, libpn_debug.so) if it is missing or
    older than its sources."""
    lib = DEBUG_LIB if debug else LIB
    if not force and not stale(lib):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    flags = NVCC_FLAGS + (["-DPN_DEBUG_CHECKS"] if debug else [])
    cmd = [nvcc(), *flags, "-o", tmp, *SOURCES]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    debug = "--debug" in sys.argv
    print(build_library(force="--force" in sys.argv, verbose=not debug, debug=debug))
