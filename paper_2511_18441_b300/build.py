"""Build librecogs.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2511_18441_b300.build [--force] [--verbose] [--debug]

--debug builds librecogs_debug.so instead: the same sources with
RECOGS_DEBUG defined, whose kernels check the indices they read from their
own data and report a failed check through recogs_check (RECOGS_EBOUNDS)
instead of making the access. The binding loads it when the environment
variable RECOGS_LIBRARY is "debug".

Every kernel is compiled for ``-gencode arch=compute_103a,code=sm_103a``
only; the library refuses other devices at context creation.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "librecogs.so")
LIB_DEBUG = os.path.join(PKG, "librecogs_debug.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "--threads", "0"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and not _stale(lib):
        return lib
    tmp = lib + ".tmp"
    flags = [*NVCC_FLAGS, *(["-DRECOGS_DEBUG"] if debug else []), *extra]
    cmd = [nvcc(), *flags, "-shared", "-o", tmp, *sources()]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [],
          debug="--debug" in sys.argv)
