"""Build step of the CUDA library (sm_103a) -- run by __graft_entry__.build().

Compiles csrc/knnjoin.cu into _build/libknnjoin.so with nvcc for the B300
architecture only (compute_103a / sm_103a, no PTX for other targets).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libknnjoin.so")
LIB_CHECKS = os.path.join(BUILD, "libknnjoin_checks.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def sources() -> list[str]:
    out = [os.path.join(INCLUDE, "knnjoin.h")]
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def up_to_date_lib(lib: str) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in sources())


def _compile(lib: str, flags: list[str], verbose: bool) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *NVCC_FLAGS, *flags, "-o", lib + ".tmp", os.path.join(CSRC, "knnjoin.cu")]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    return _compile(LIB, list(extra or []), verbose)


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The checked variant (-DKNN_CHECKS): kernels test their array indexes and
    report a failed test as KNN_ERR_CUDA instead of accessing out of bounds."""
    if not force and up_to_date_lib(LIB_CHECKS):
        return LIB_CHECKS
    return _compile(LIB_CHECKS, ["-DKNN_CHECKS"], verbose)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None)
    print(LIB)
