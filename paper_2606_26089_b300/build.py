"""Build the CUDA library (libpdr.so) in-tree for sm_103a with nvcc.

Usage: ``python -m paper_2606_26089_b300.build`` (or ``build()`` from Python).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libpdr.so")
# debug build: every batch-array, event and table index of the response kernel
# checked (an index out of range sets ERR_BOUNDS in the error word and is not used)
LIB_BOUNDS = os.path.join(HERE, "libpdr_bounds.so")
SOURCES = ["pdr_kernel.cu", "pdr_pileup.cu", "pdr_postprocess.cu", "pdr_ip.cu", "pdr_jets.cu", "pdr_runtime.cu",
           "pdr_noalloc.cu", "pdr_diag.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "pdr.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile csrc/*.cu into libpdr.so next to this file (bounds: the
    bounds-checking debug build, libpdr_bounds.so); returns its path."""
    lib = LIB_BOUNDS if bounds else LIB
    if not force and not _stale(lib):
        return lib
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", CSRC, "-o", lib + ".tmp"]
    if bounds:
        cmd += ["-DPDR_BOUNDS"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    cmd += ["-lcudart"]
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
