"""Build step of the CUDA library (sm_103a) -- run by __graft_entry__.build().

Compiles the library for the B300 architecture only (compute_103a / sm_103a,
no PTX for other targets) into _build/libknnjoin.so: csrc/knnjoin.cu (host
orchestration, the C ABI and every kernel but the scan) and one object of
csrc/scan2_launch.cu per dimension d = 1..8 (-DKNN_SCAN2_DIM=d: that
dimension's scan kernel instances), compiled in parallel and linked with
nvcc.  An object is rebuilt when a file it includes (local "..." includes,
followed recursively) is newer than it.
"""
from __future__ import annotations

import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libknnjoin.so")
LIB_CHECKS = os.path.join(BUILD, "libknnjoin_checks.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [*ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xfatbin=-compress-all"]
SCAN2_DIMS = range(1, 9)


def _includes(path: str, seen: set[str]) -> set[str]:
    """`path` and every local header it includes, recursively."""
    path = os.path.normpath(path)
    if path in seen or not os.path.exists(path):
        return seen
    seen.add(path)
    with open(path) as f:
        for m in re.finditer(r'^\s*#\s*include\s+"([^"]+)"', f.read(), re.M):
            _includes(os.path.join(os.path.dirname(path), m.group(1)), seen)
    return seen


def sources() -> list[str]:
    """Every file the library is built from."""
    out = [os.path.join(INCLUDE, "knnjoin.h")]
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def _units(tag: str) -> list[tuple[str, str, list[str]]]:
    """(source, object, extra flags) of every translation unit."""
    units = [(os.path.join(CSRC, "knnjoin.cu"), os.path.join(BUILD, f"knnjoin{tag}.o"), [])]
    for d in SCAN2_DIMS:
        units.append((os.path.join(CSRC, "scan2_launch.cu"), os.path.join(BUILD, f"scan2_d{d}{tag}.o"),
                      [f"-DKNN_SCAN2_DIM={d}"]))
    return units


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in deps)


def up_to_date_lib(lib: str) -> bool:
    return not _stale(lib, sources())


def up_to_date() -> bool:
    return up_to_date_lib(LIB)


def _compile(lib: str, flags: list[str], verbose: bool, tag: str) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    jobs = []
    for src, obj, extra in _units(tag):
        if _stale(obj, _includes(src, set())):
            jobs.append([nvcc, *NVCC_FLAGS, *flags, *extra, "-c", "-o", obj + ".tmp", src])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        os.replace(cmd[-2], cmd[-2][:-4])

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(run, j) for j in jobs]:
            f.result()
    objs = [obj for _, obj, _ in _units(tag)]
    cmd = [nvcc, *ARCH, "-shared", "-o", lib + ".tmp", *objs]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    if force:
        for _, obj, _ in _units(""):
            if os.path.exists(obj):
                os.remove(obj)
    return _compile(LIB, list(extra or []), verbose, "")


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The checked variant (-DKNN_CHECKS): kernels test their array indexes and
    report a failed test as KNN_ERR_CUDA instead of accessing out of bounds."""
    if not force and up_to_date_lib(LIB_CHECKS):
        return LIB_CHECKS
    if force:
        for _, obj, _ in _units("_checks"):
            if os.path.exists(obj):
                os.remove(obj)
    return _compile(LIB_CHECKS, ["-DKNN_CHECKS"], verbose, "_checks")


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None)
    print(LIB)
