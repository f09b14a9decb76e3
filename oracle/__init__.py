"""CPU oracle for the exact KNN self-join -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library neither imports it nor
shares code with it.

The C source (``knn_oracle.c``) holds the definition written out (brute
force, canonical FP64 squared distance, ties by index, self excluded; paper
Sec. 2.1) and an exact grid join in the paper's manner (Sec. 3.1, 4.3) that
also counts the candidate evaluations of that schedule.  This module builds
it with gcc (``-ffp-contract=off``, OpenMP) and wraps it with ctypes.

Mutant builds (``build(mutant=...)``) compile the same source with one
planted mistake; the pinning tests use them to show that every pin fails on
a plausible error.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}

MUTANTS = ("DROP_LAST_TERM", "TIE_DESC", "KEEP_SELF", "LOOSE_CERTIFICATE",
           "NO_LOWER_NEIGHBOUR")
# planted mistakes in the FP32-only ranking (caught by its own pins)
FP32_MUTANTS = ("FP32_ONE_CHAIN", "FP32_UNFUSED")
# planted mistakes in the work count and the search-distance selection
# (caught by tests/test_oracle_schedule.py)
SCHEDULE_MUTANTS = ("COUNT_LAST_PASS", "COUNT_SELF", "EPS_BIN_OFF_BY_ONE")


def _lib_path(mutant: str | None) -> str:
    name = "liboracle.so" if not mutant else f"liboracle_{mutant.lower()}.so"
    return os.path.join(_BUILD, name)


def build(mutant: str | None = None, force: bool = False) -> str:
    """Compile the oracle (or one mutant of it); returns the .so path."""
    out = _lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
           "-o", out + ".tmp", _SRC, "-lm"]
    if mutant:
        if mutant not in MUTANTS + FP32_MUTANTS + SCHEDULE_MUTANTS:
            raise ValueError(mutant)
        cmd.insert(1, f"-DORACLE_MUTANT_{mutant}")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


class GridStats(ctypes.Structure):
    _fields_ = [("eps_mean", ctypes.c_double), ("eps_min", ctypes.c_double),
                ("width", ctypes.c_double), ("candidates", ctypes.c_int64),
                ("passes", ctypes.c_int), ("pass_queries", ctypes.c_int64 * 64),
                ("pass_candidates", ctypes.c_int64 * 64)]


def _load(mutant: str | None = None) -> ctypes.CDLL:
    key = mutant or ""
    with _lock:
        if key not in _libs:
            lib = ctypes.CDLL(build(mutant))
            P = ctypes.c_void_p
            lib.oracle_bf.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int]
            lib.oracle_bf.restype = ctypes.c_int
            lib.oracle_bf_rows.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P,
                                           ctypes.c_int64, P, P, ctypes.c_int]
            lib.oracle_bf_rows.restype = ctypes.c_int
            lib.oracle_bf_rs.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         P, P, ctypes.c_int]
            lib.oracle_bf_rs.restype = ctypes.c_int
            lib.oracle_fp32_rows.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P,
                                             ctypes.c_int64, P, ctypes.c_int]
            lib.oracle_fp32_rows.restype = ctypes.c_int
            lib.oracle_grid.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, P, P, P, ctypes.c_int]
            lib.oracle_grid.restype = ctypes.c_int
            lib.oracle_grid_rows.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, P, ctypes.c_int64, P, P, P,
                                             ctypes.c_int]
            lib.oracle_grid_rows.restype = ctypes.c_int
            lib.oracle_select_epsilon.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                  P, ctypes.c_int]
            lib.oracle_select_epsilon.restype = ctypes.c_double
            lib.oracle_grid_stats_size.restype = ctypes.c_int
            assert lib.oracle_grid_stats_size() == ctypes.sizeof(GridStats)
            _libs[key] = lib
        return _libs[key]


def _prep(points: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(points, dtype=np.float32)
    if p.ndim != 2:
        raise ValueError("points must be n x d")
    return p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def bf(points: np.ndarray, K: int, threads: int = 0, mutant: str | None = None):
    """Brute-force self-join: (ids int32 [n,K], dist float64 [n,K])."""
    p = _prep(points)
    n, d = p.shape
    ids = np.empty((n, K), np.int32)
    dist = np.empty((n, K), np.float64)
    rc = _load(mutant).oracle_bf(_ptr(p), n, d, K, _ptr(ids), _ptr(dist), threads)
    if rc:
        raise ValueError("oracle_bf: invalid arguments")
    return ids, dist


def bf_rs(queries: np.ndarray, points: np.ndarray, K: int, threads: int = 0, mutant: str | None = None):
    """Brute-force R x S join: for each query row, the K nearest data rows
    (ids into `points`, nothing excluded); arrays [len(queries), K]."""
    q, p = _prep(queries), _prep(points)
    if q.shape[1] != p.shape[1]:
        raise ValueError("queries and points must have the same d")
    nq, d = q.shape
    n = p.shape[0]
    ids = np.empty((nq, K), np.int32)
    dist = np.empty((nq, K), np.float64)
    rc = _load(mutant).oracle_bf_rs(_ptr(q), nq, _ptr(p), n, d, K, _ptr(ids), _ptr(dist), threads)
    if rc:
        raise ValueError("oracle_bf_rs: invalid arguments")
    return ids, dist


def bf_rows(points: np.ndarray, K: int, rows, threads: int = 0, mutant: str | None = None):
    """Brute force for the query rows `rows` only: arrays [len(rows), K]."""
    p = _prep(points)
    n, d = p.shape
    r = np.ascontiguousarray(rows, dtype=np.int64)
    ids = np.empty((len(r), K), np.int32)
    dist = np.empty((len(r), K), np.float64)
    rc = _load(mutant).oracle_bf_rows(_ptr(p), n, d, K, _ptr(r), len(r), _ptr(ids),
                                      _ptr(dist), threads)
    if rc:
        raise ValueError("oracle_bf_rows: invalid arguments")
    return ids, dist


def fp32_rows(points: np.ndarray, K: int, rows, threads: int = 0, mutant: str | None = None):
    """For the query rows `rows`, the K nearest under the FP32 filter distance
    alone, ties by index, self excluded: ids int32 [len(rows), K]."""
    p = _prep(points)
    n, d = p.shape
    r = np.ascontiguousarray(rows, dtype=np.int64)
    ids = np.empty((len(r), K), np.int32)
    rc = _load(mutant).oracle_fp32_rows(_ptr(p), n, d, K, _ptr(r), len(r), _ptr(ids), threads)
    if rc:
        raise ValueError("oracle_fp32_rows: invalid arguments")
    return ids


def fp32_mismatch(points: np.ndarray, exact_ids: np.ndarray, rows, threads: int = 0):
    """Counts of how the FP32-only rows differ from the exact rows
    `exact_ids[rows]`: (rows differing anywhere, positions differing, exact
    ids absent from the FP32-only row)."""
    r = np.ascontiguousarray(rows, dtype=np.int64)
    want = np.asarray(exact_ids)[r]
    got = fp32_rows(points, want.shape[1], r, threads)
    diff = got != want
    missing = sum(len(np.setdiff1d(want[k], got[k])) for k in range(len(r)))
    return int(diff.any(axis=1).sum()), int(diff.sum()), int(missing)


def grid(points: np.ndarray, K: int, width_mult: float = 1.0, threads: int = 0,
         mutant: str | None = None):
    """Exact grid join: (ids, dist, stats dict).  stats['candidates'] is the
    number of candidate distance evaluations of the schedule."""
    p = _prep(points)
    n, d = p.shape
    ids = np.empty((n, K), np.int32)
    dist = np.empty((n, K), np.float64)
    st = GridStats()
    rc = _load(mutant).oracle_grid(_ptr(p), n, d, K, width_mult, _ptr(ids), _ptr(dist),
                                   ctypes.byref(st), threads)
    if rc:
        raise ValueError("oracle_grid: invalid arguments")
    stats = dict(eps_mean=st.eps_mean, eps_min=st.eps_min, width=st.width,
                 candidates=int(st.candidates), passes=int(st.passes),
                 pass_queries=[int(st.pass_queries[i]) for i in range(min(st.passes, 64))],
                 pass_candidates=[int(st.pass_candidates[i]) for i in range(min(st.passes, 64))])
    return ids, dist, stats


def grid_rows(points: np.ndarray, K: int, rows, width_mult: float = 1.0, threads: int = 0):
    """Grid join of the query rows `rows` only: (ids, dist, stats), arrays [len(rows), K]."""
    p = _prep(points)
    n, d = p.shape
    r = np.ascontiguousarray(rows, dtype=np.int64)
    ids = np.empty((len(r), K), np.int32)
    dist = np.empty((len(r), K), np.float64)
    st = GridStats()
    rc = _load().oracle_grid_rows(_ptr(p), n, d, K, width_mult, _ptr(r), len(r), _ptr(ids),
                                  _ptr(dist), ctypes.byref(st), threads)
    if rc:
        raise ValueError("oracle_grid_rows: invalid arguments")
    return ids, dist, dict(candidates=int(st.candidates), passes=int(st.passes),
                           eps_min=st.eps_min, width=st.width)


def select_epsilon(points: np.ndarray, K: int, threads: int = 0, mutant: str | None = None):
    """(eps_min, eps_mean) of the paper's Sec. 4.4 procedure as the oracle reads it."""
    p = _prep(points)
    n, d = p.shape
    em = ctypes.c_double(0.0)
    e = _load(mutant).oracle_select_epsilon(_ptr(p), n, d, K, ctypes.byref(em), threads)
    return float(e), float(em.value)
