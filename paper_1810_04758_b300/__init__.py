"""Python binding of the B300 exact KNN self-join library (libknnjoin.so).

Argument marshalling only: every step of the join runs in the library's CUDA
kernels.  The functions carry the C ABI's names (include/knnjoin.h); the
``Context`` class wraps them for torch tensors (device memory and streams come
from PyTorch).  There is no CPU fallback: importing works without a GPU, but
every call needs the built library and a CUDA device, and fails loudly
otherwise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libknnjoin.so")

KNN_OK = 0
KNN_ERR_INVALID = 1
KNN_ERR_NOMEM = 2
KNN_ERR_CUDA = 3
KNN_ERR_NOT_READY = 4
KNN_ERR_TIMEOUT = 5
KNN_ERR_CANCELLED = 6
KNN_ERR_QUEUE_FULL = 7
STATUS_NAMES = {0: "KNN_OK", 1: "KNN_ERR_INVALID", 2: "KNN_ERR_NOMEM", 3: "KNN_ERR_CUDA",
                4: "KNN_ERR_NOT_READY", 5: "KNN_ERR_TIMEOUT", 6: "KNN_ERR_CANCELLED",
                7: "KNN_ERR_QUEUE_FULL"}

# Every symbol include/knnjoin.h declares.
EXPORTS = ("knnjoin_create", "knnjoin_destroy", "knnjoin_self_join", "knnjoin_join", "knnjoin_autotune",
           "knnjoin_self_join_batch",
           "knnjoin_submit", "knnjoin_poll", "knnjoin_cancel", "knnjoin_get_stats",
           "knnjoin_last_error", "knnjoin_version", "knnjoin_self_join_noalloc",
           "knnjoin_fp32_mismatch", "knnjoin_index_create", "knnjoin_index_query",
           "knnjoin_index_stats", "knnjoin_index_destroy", "knnjoin_self_join_rows",
           "knnjoin_shard_bounds", "knnjoin_self_join_range", "knnjoin_work_queue", "knnjoin_index_dump")
KNN_NOALLOC_MAX_POINTS = 65536


class KnnjoinConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("alloc", ctypes.c_void_p), ("free", ctypes.c_void_p), ("user", ctypes.c_void_p),
                ("hbm_budget_bytes", ctypes.c_size_t), ("max_jobs", ctypes.c_int),
                ("tune_cache_path", ctypes.c_char_p), ("width_mult", ctypes.c_float),
                ("workers", ctypes.c_int), ("policy", ctypes.c_int), ("out_chunk_mb", ctypes.c_int),
                ("large_first", ctypes.c_int), ("batch_union", ctypes.c_int),
                ("tail_queries", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class KnnjoinJob(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int),
                ("K", ctypes.c_int), ("out_ids", ctypes.c_void_p), ("out_dist", ctypes.c_void_p)]


class KnnjoinStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int), ("K", ctypes.c_int),
                ("passes", ctypes.c_int), ("start_level", ctypes.c_int),
                ("pass_queries", ctypes.c_int64 * 16), ("candidates", ctypes.c_int64),
                ("band_entries", ctypes.c_int64), ("overflow_queries", ctypes.c_int64),
                ("eps_mean", ctypes.c_double), ("eps_min", ctypes.c_double),
                ("cell_width", ctypes.c_double), ("key_bits", ctypes.c_int),
                ("fixed_point", ctypes.c_int), ("ms_total", ctypes.c_double),
                ("ms_index", ctypes.c_double), ("ms_scan", ctypes.c_double),
                ("launches", ctypes.c_int64), ("ms_queue", ctypes.c_double),
                ("ms_wall", ctypes.c_double),
                ("ms_pass", ctypes.c_double * 16),
                ("pass_candidates", ctypes.c_int64 * 16),
                ("width_mult", ctypes.c_double),
                ("chunks", ctypes.c_int64),
                ("buffer_entries", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if name == "pass_queries":
                v = [int(x) for x in v[: max(self.passes, 0)]]
            elif name == "pass_candidates":
                v = [int(x) for x in v[: max(min(self.passes, 16), 0)]]
            elif name == "ms_pass":
                v = [float(x) for x in v[: max(min(self.passes, 16), 0)]]
            d[name] = v
        return d


class KnnJoinError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib: Optional[ctypes.CDLL] = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libknnjoin.so (built by paper_1810_04758_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libknnjoin.so not built ({path}); run paper_1810_04758_b300/build.py")
    lib = ctypes.CDLL(path)
    P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.knnjoin_create.argtypes = [ctypes.POINTER(KnnjoinConfig), ctypes.POINTER(P)]
    lib.knnjoin_create.restype = I
    lib.knnjoin_destroy.argtypes = [P]
    lib.knnjoin_destroy.restype = None
    lib.knnjoin_self_join.argtypes = [P, P, I64, I, I, P, P]
    lib.knnjoin_self_join.restype = I
    lib.knnjoin_join.argtypes = [P, P, I64, P, I64, I, I, P, P]
    lib.knnjoin_join.restype = I
    lib.knnjoin_autotune.argtypes = [P, P, I64, I, I, ctypes.POINTER(ctypes.c_float)]
    lib.knnjoin_autotune.restype = I
    lib.knnjoin_fp32_mismatch.argtypes = [P, P, I64, I, I, P, ctypes.POINTER(ctypes.c_int64), I64,
                                          ctypes.POINTER(ctypes.c_int64)]
    lib.knnjoin_fp32_mismatch.restype = I
    lib.knnjoin_self_join_rows.argtypes = [P, P, I64, I, I, I64, I64, P, P]
    lib.knnjoin_self_join_rows.restype = I
    lib.knnjoin_shard_bounds.argtypes = [P, P, I64, I, I, I, P, P]
    lib.knnjoin_shard_bounds.restype = I
    lib.knnjoin_self_join_range.argtypes = [P, P, I64, I, I, I64, I64, P, P, P]
    lib.knnjoin_self_join_range.restype = I
    lib.knnjoin_work_queue.argtypes = [P, P, I64, I, I, P, I64, ctypes.POINTER(ctypes.c_int64)]
    lib.knnjoin_work_queue.restype = I
    lib.knnjoin_index_dump.argtypes = [P, P, I64, I, I, I, P, P, P, P, I64, P]
    lib.knnjoin_index_dump.restype = I
    lib.knnjoin_index_create.argtypes = [P, P, I64, I, I, ctypes.POINTER(ctypes.c_void_p)]
    lib.knnjoin_index_create.restype = I
    lib.knnjoin_index_query.argtypes = [P, P, I64, I, P, P]
    lib.knnjoin_index_query.restype = I
    lib.knnjoin_index_stats.argtypes = [P, ctypes.POINTER(KnnjoinStats)]
    lib.knnjoin_index_stats.restype = I
    lib.knnjoin_index_destroy.argtypes = [P]
    lib.knnjoin_index_destroy.restype = None
    lib.knnjoin_self_join_batch.argtypes = [P, ctypes.POINTER(KnnjoinJob), I]
    lib.knnjoin_self_join_batch.restype = I
    lib.knnjoin_submit.argtypes = [P, ctypes.POINTER(KnnjoinJob), ctypes.POINTER(ctypes.c_uint64)]
    lib.knnjoin_submit.restype = I
    lib.knnjoin_poll.argtypes = [P, ctypes.c_uint64]
    lib.knnjoin_poll.restype = I
    lib.knnjoin_cancel.argtypes = [P, ctypes.c_uint64]
    lib.knnjoin_cancel.restype = I
    lib.knnjoin_get_stats.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(KnnjoinStats)]
    lib.knnjoin_get_stats.restype = I
    lib.knnjoin_last_error.argtypes = [P]
    lib.knnjoin_last_error.restype = ctypes.c_char_p
    lib.knnjoin_self_join_noalloc.argtypes = [P, I64, I, I, P, P, P, ctypes.c_char_p, ctypes.c_size_t]
    lib.knnjoin_self_join_noalloc.restype = I
    lib.knnjoin_version.argtypes = []
    lib.knnjoin_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# Functions with the C ABI's names (raw pointers as Python ints)
# ---------------------------------------------------------------------------
def knnjoin_create(cfg: Optional[KnnjoinConfig] = None) -> int:
    lib = load_library()
    out = ctypes.c_void_p()
    st = lib.knnjoin_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(out))
    if st != KNN_OK:
        raise KnnJoinError(st, "knnjoin_create failed")
    return out.value


def knnjoin_destroy(ctx: int) -> None:
    load_library().knnjoin_destroy(ctx)


def knnjoin_last_error(ctx: int) -> str:
    return load_library().knnjoin_last_error(ctx).decode()


def knnjoin_version() -> str:
    return load_library().knnjoin_version().decode()


def _check(ctx: int, st: int) -> int:
    if st not in (KNN_OK, KNN_ERR_NOT_READY):
        raise KnnJoinError(st, knnjoin_last_error(ctx))
    return st


def knnjoin_self_join(ctx: int, points: int, n: int, d: int, K: int, out_ids: int,
                      out_dist: int) -> int:
    return _check(ctx, load_library().knnjoin_self_join(ctx, points, n, d, K, out_ids, out_dist))


def knnjoin_join(ctx: int, queries: int, nq: int, points: int, n: int, d: int, K: int, out_ids: int,
                 out_dist: int) -> int:
    return _check(ctx, load_library().knnjoin_join(ctx, queries, nq, points, n, d, K, out_ids, out_dist))


def knnjoin_autotune(ctx: int, points: int, n: int, d: int, K: int) -> float:
    best = ctypes.c_float(0.0)
    _check(ctx, load_library().knnjoin_autotune(ctx, points, n, d, K, ctypes.byref(best)))
    return float(best.value)


def knnjoin_fp32_mismatch(ctx: int, points: int, n: int, d: int, K: int, ids: int,
                          rows: Sequence[int]) -> tuple[int, int, int]:
    arr = (ctypes.c_int64 * len(rows))(*rows)
    out = (ctypes.c_int64 * 3)()
    _check(ctx, load_library().knnjoin_fp32_mismatch(ctx, points, n, d, K, ids, arr, len(rows), out))
    return int(out[0]), int(out[1]), int(out[2])


def knnjoin_self_join_rows(ctx: int, points: int, n: int, d: int, K: int, row_begin: int, row_end: int,
                           out_ids: int, out_dist: int) -> int:
    return _check(ctx, load_library().knnjoin_self_join_rows(ctx, points, n, d, K, row_begin, row_end,
                                                             out_ids, out_dist))


def knnjoin_shard_bounds(ctx: int, points: int, n: int, d: int, K: int, nshards: int):
    """(bounds int64 [nshards + 1], costs float64 [nshards]) of the
    cost-balanced shards (sorted query positions)."""
    import numpy as np
    bounds = np.zeros(nshards + 1, np.int64)
    costs = np.zeros(nshards, np.float64)
    _check(ctx, load_library().knnjoin_shard_bounds(ctx, points, n, d, K, nshards, bounds.ctypes.data,
                                                    costs.ctypes.data))
    return bounds, costs


def knnjoin_self_join_range(ctx: int, points: int, n: int, d: int, K: int, pos_begin: int, pos_end: int,
                            out_rows: int, out_ids: int, out_dist: int) -> int:
    return _check(ctx, load_library().knnjoin_self_join_range(ctx, points, n, d, K, pos_begin, pos_end, out_rows,
                                                              out_ids, out_dist))


def knnjoin_index_dump(ctx: int, points: int, n: int, d: int, K: int, level: int = 0, probe_keys=None):
    """The join's grid index: (sorted keys uint64 [n], permutation uint32 [n],
    grid dict, probe runs uint32 [m, 2] or None) -- see knnjoin_index_dump in
    include/knnjoin.h."""
    import numpy as np
    keys = np.zeros(n, np.uint64)
    perm = np.zeros(n, np.uint32)
    grid = np.zeros(3 + 2 * d, np.float64)
    pk = None if probe_keys is None else np.ascontiguousarray(probe_keys, dtype=np.uint64)
    runs = None if pk is None else np.zeros((len(pk), 2), np.uint32)
    m = 0 if pk is None else len(pk)
    _check(ctx, load_library().knnjoin_index_dump(ctx, points, n, d, K, level, keys.ctypes.data, perm.ctypes.data,
                                                  grid.ctypes.data, None if pk is None else pk.ctypes.data, m,
                                                  None if runs is None else runs.ctypes.data))
    g = {"w0": grid[0], "bits": int(grid[1]), "lo": grid[2:2 + d].copy(),
         "cmax0": grid[2 + d:2 + 2 * d].astype(np.int64), "dense_table": int(grid[2 + 2 * d])}
    return keys, perm, g, runs


def knnjoin_work_queue(ctx: int, points: int, n: int, d: int, K: int):
    """Cell count of each query in the first pass's work-queue order."""
    import numpy as np
    out = np.zeros(n, np.int64)
    ln = ctypes.c_int64(0)
    _check(ctx, load_library().knnjoin_work_queue(ctx, points, n, d, K, out.ctypes.data, n, ctypes.byref(ln)))
    return out[: ln.value]


def gather_shards(n: int, K: int, parts):
    """Reassemble a self-join's rows from shards given as (rows, ids, dist)
    numpy arrays (rows: the original row of each shard row): ids int32 [n, K]
    and dist float64 [n, K].  Every row must be covered exactly once."""
    import numpy as np
    ids = np.full((n, K), -1, np.int32)
    dist = np.full((n, K), np.nan, np.float64)
    seen = np.zeros(n, np.int64)
    for rows, i, d in parts:
        rows = np.asarray(rows, np.int64)
        np.add.at(seen, rows, 1)
        ids[rows] = i
        dist[rows] = d
    if not (seen == 1).all():
        raise ValueError("shards do not cover every row exactly once")
    return ids, dist


def knnjoin_index_create(ctx: int, points: int, n: int, d: int, K: int) -> int:
    out = ctypes.c_void_p(0)
    _check(ctx, load_library().knnjoin_index_create(ctx, points, n, d, K, ctypes.byref(out)))
    return int(out.value)


def knnjoin_index_query(ctx: int, index: int, queries: int, nq: int, K: int, out_ids: int,
                        out_dist: int) -> int:
    # errors are reported through the index's context
    return _check(ctx, load_library().knnjoin_index_query(index, queries, nq, K, out_ids, out_dist))


def knnjoin_index_stats(index: int) -> dict:
    st = KnnjoinStats()
    if load_library().knnjoin_index_stats(index, ctypes.byref(st)) != KNN_OK:
        raise KnnJoinError(KNN_ERR_INVALID, "invalid index")
    return st.as_dict()


def knnjoin_index_destroy(index: int) -> None:
    load_library().knnjoin_index_destroy(index)


def knnjoin_self_join_batch(ctx: int, jobs: list[KnnjoinJob]) -> int:
    arr = (KnnjoinJob * len(jobs))(*jobs)
    return _check(ctx, load_library().knnjoin_self_join_batch(ctx, arr, len(jobs)))


def knnjoin_submit(ctx: int, job: KnnjoinJob) -> int:
    jid = ctypes.c_uint64()
    _check(ctx, load_library().knnjoin_submit(ctx, ctypes.byref(job), ctypes.byref(jid)))
    return jid.value


def knnjoin_poll(ctx: int, job_id: int) -> int:
    """Raw status (KNN_OK / KNN_ERR_NOT_READY / error code); never raises."""
    return load_library().knnjoin_poll(ctx, job_id)


def knnjoin_cancel(ctx: int, job_id: int) -> int:
    return load_library().knnjoin_cancel(ctx, job_id)


def knnjoin_self_join_noalloc(points: int, n: int, d: int, K: int, out_ids: int, out_dist: int,
                              stream: int = 0) -> int:
    """The allocation-free variant (device pointers only, n <= 65,536); see
    include/knnjoin.h.  Raises KnnJoinError with the library's message."""
    buf = ctypes.create_string_buffer(512)
    st = load_library().knnjoin_self_join_noalloc(points, n, d, K, out_ids, out_dist, stream,
                                                  buf, len(buf))
    if st != KNN_OK:
        raise KnnJoinError(st, buf.value.decode())
    return st


def knnjoin_get_stats(ctx: int, job_id: int = 0) -> dict:
    st = KnnjoinStats()
    _check(ctx, load_library().knnjoin_get_stats(ctx, job_id, ctypes.byref(st)))
    return st.as_dict()


def shard_rows(n: int, world: int, rank: int) -> tuple[int, int]:
    """Row range [begin, end) of rank `rank` when a join of n query rows is
    split over `world` GPUs: contiguous, disjoint, covering [0, n), sizes
    differing by at most one (queries of random order cost alike on average)."""
    if world < 1 or not 0 <= rank < world or n < world:
        raise ValueError("need 0 <= rank < world <= n")
    return n * rank // world, n * (rank + 1) // world


# ---------------------------------------------------------------------------
# torch-facing wrapper
# ---------------------------------------------------------------------------
class Context:
    """A library context bound to a CUDA device and (by default) torch's
    current stream on it."""

    def __init__(self, device: int = 0, stream=None, width_mult: float = 0.0,
                 max_jobs: int = 0, hbm_budget_bytes: int = 0, workers: int = 0,
                 tune_cache_path: Optional[str] = None, policy: int = 0, out_chunk_mb: int = 0,
                 large_first: bool = False, batch_union: bool = False, tail_queries: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self._torch = torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        cfg = KnnjoinConfig()
        cfg.device = device
        cfg.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        cfg.width_mult = width_mult
        cfg.max_jobs = max_jobs
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.workers = workers
        cfg.policy = policy
        cfg.out_chunk_mb = out_chunk_mb
        cfg.large_first = 1 if large_first else 0
        cfg.batch_union = 1 if batch_union else 0
        cfg.tail_queries = tail_queries
        self._tune_path = tune_cache_path.encode() if tune_cache_path else None
        cfg.tune_cache_path = self._tune_path
        self._cfg = cfg
        self.ctx = knnjoin_create(cfg)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            knnjoin_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _outputs(self, n: int, K: int, like, out_ids, out_dist):
        torch = self._torch
        dev = like.device
        if out_ids is None:
            out_ids = torch.empty((n, K), dtype=torch.int32, device=dev)
        if out_dist is None:
            out_dist = torch.empty((n, K), dtype=torch.float64, device=dev)
        for t, dt in ((out_ids, torch.int32), (out_dist, torch.float64)):
            if t.dtype != dt or not t.is_contiguous() or tuple(t.shape) != (n, K):
                raise ValueError("output tensors must be contiguous [n, K] int32 / float64")
        return out_ids, out_dist

    def self_join(self, points, K: int, out_ids=None, out_dist=None):
        """Exact KNN self-join of a float32 [n, d] tensor (host or device).
        Returns (ids int32 [n, K], dist float64 [n, K]) on the points' device."""
        torch = self._torch
        if points.dtype != torch.float32 or points.dim() != 2:
            raise ValueError("points must be a float32 [n, d] tensor")
        points = points.contiguous()
        n, d = points.shape
        out_ids, out_dist = self._outputs(n, K, points, out_ids, out_dist)
        knnjoin_self_join(self.ctx, points.data_ptr(), n, d, K, out_ids.data_ptr(),
                          out_dist.data_ptr())
        return out_ids, out_dist

    def self_join_rows(self, points, K: int, row_begin: int, row_end: int, out_ids=None, out_dist=None):
        """Rows [row_begin, row_end) of the self-join of `points` (one shard of
        the join): (ids int32 [rows, K], dist float64 [rows, K])."""
        torch = self._torch
        if points.dtype != torch.float32 or points.dim() != 2:
            raise ValueError("points must be a float32 [n, d] tensor")
        points = points.contiguous()
        n, d = points.shape
        rows = max(0, row_end - row_begin)
        out_ids, out_dist = self._outputs(max(rows, 1), K, points, out_ids, out_dist)
        knnjoin_self_join_rows(self.ctx, points.data_ptr(), n, d, K, row_begin, row_end, out_ids.data_ptr(),
                               out_dist.data_ptr())
        return out_ids, out_dist

    def shard_bounds(self, points, K: int, nshards: int):
        """Cost-balanced cut points (sorted query positions, int64 [nshards + 1])
        and each shard's estimated cost."""
        points = points.contiguous()
        n, d = points.shape
        return knnjoin_shard_bounds(self.ctx, points.data_ptr(), n, d, K, nshards)

    def self_join_range(self, points, K: int, pos_begin: int, pos_end: int):
        """The queries at sorted positions [pos_begin, pos_end) (one
        cost-balanced shard): (rows int64 [m], ids int32 [m, K], dist float64
        [m, K]), rows = the original row of each output row."""
        torch = self._torch
        points = points.contiguous()
        n, d = points.shape
        m = pos_end - pos_begin
        rows = torch.empty(max(m, 1), dtype=torch.int64, device=points.device)
        out_ids, out_dist = self._outputs(max(m, 1), K, points, None, None)
        knnjoin_self_join_range(self.ctx, points.data_ptr(), n, d, K, pos_begin, pos_end, rows.data_ptr(),
                                out_ids.data_ptr(), out_dist.data_ptr())
        return rows, out_ids, out_dist

    def autotune(self, points, K: int) -> float:
        """Time the self-join of `points` at several cell-width multipliers and
        keep the fastest for later joins of the same (d, K, log2 n) class;
        returns it.  Results never depend on the multiplier."""
        points = points.contiguous()
        n, d = points.shape
        return knnjoin_autotune(self.ctx, points.data_ptr(), n, d, K)

    def fp32_mismatch(self, points, ids, rows) -> dict:
        """For the listed query rows of a self-join result `ids` (int32 [n, K])
        of `points` (float32 [n, d]), compare with ranking by the FP32 filter
        distance alone; returns the counts and rates of rows, positions and
        ids that would differ."""
        torch = self._torch
        if points.dtype != torch.float32 or points.dim() != 2:
            raise ValueError("points must be a float32 [n, d] tensor")
        if ids.dtype != torch.int32 or ids.dim() != 2 or ids.shape[0] != points.shape[0]:
            raise ValueError("ids must be an int32 [n, K] tensor")
        points, ids = points.contiguous(), ids.contiguous()
        n, d = points.shape
        K = ids.shape[1]
        rows = [int(r) for r in rows]
        rw, pw, miss = knnjoin_fp32_mismatch(self.ctx, points.data_ptr(), n, d, K, ids.data_ptr(), rows)
        m = len(rows)
        return {"rows": m, "K": K, "rows_differing": rw, "positions_differing": pw, "ids_missing": miss,
                "row_mismatch_rate": rw / m, "id_mismatch_rate": pw / (m * K), "set_mismatch_rate": miss / (m * K)}

    def index(self, points, K: int) -> "Index":
        """Index the float32 [n, d] `points` (host or device) once and keep the
        index on the device; its `query` answers R x S joins against them."""
        torch = self._torch
        if points.dtype != torch.float32 or points.dim() != 2:
            raise ValueError("points must be a float32 [n, d] tensor")
        points = points.contiguous()
        n, d = points.shape
        return Index(self, knnjoin_index_create(self.ctx, points.data_ptr(), n, d, K), n, d)

    def join(self, queries, points, K: int, out_ids=None, out_dist=None):
        """R x S join: for each row of the float32 [nq, d] `queries`, the K
        nearest rows of the float32 [n, d] `points` (nothing excluded).
        Returns (ids int32 [nq, K], dist float64 [nq, K]) on the queries' device."""
        torch = self._torch
        for t in (queries, points):
            if t.dtype != torch.float32 or t.dim() != 2:
                raise ValueError("queries and points must be float32 [rows, d] tensors")
        if queries.shape[1] != points.shape[1]:
            raise ValueError("queries and points must have the same d")
        queries, points = queries.contiguous(), points.contiguous()
        nq, d = queries.shape
        n = points.shape[0]
        out_ids, out_dist = self._outputs(nq, K, queries, out_ids, out_dist)
        knnjoin_join(self.ctx, queries.data_ptr(), nq, points.data_ptr(), n, d, K, out_ids.data_ptr(),
                     out_dist.data_ptr())
        return out_ids, out_dist

    def self_join_batch(self, point_list, Ks, outs_in=None):
        """Independent joins run concurrently by the context's worker pool.
        outs_in: optional list of (ids, dist) output tensors (e.g. pinned host
        buffers); returns the list of (ids, dist)."""
        torch = self._torch
        jobs, outs = [], []
        for q, (p, K) in enumerate(zip(point_list, Ks)):
            p = p.contiguous()
            n, d = p.shape
            given = outs_in[q] if outs_in is not None else (None, None)
            ids, dist = self._outputs(n, K, p, given[0], given[1])
            outs.append((ids, dist))
            jobs.append(KnnjoinJob(p.data_ptr(), n, d, K, ids.data_ptr(), dist.data_ptr()))
        self._keep = point_list
        knnjoin_self_join_batch(self.ctx, jobs)
        return outs

    def submit(self, points, K: int, out_ids=None, out_dist=None):
        """Enqueue a join; returns (job_id, ids, dist).  Keep the tensors alive
        until poll() returns a final status."""
        points = points.contiguous()
        n, d = points.shape
        out_ids, out_dist = self._outputs(n, K, points, out_ids, out_dist)
        job = KnnjoinJob(points.data_ptr(), n, d, K, out_ids.data_ptr(), out_dist.data_ptr())
        return knnjoin_submit(self.ctx, job), out_ids, out_dist

    def poll(self, job_id: int) -> int:
        return knnjoin_poll(self.ctx, job_id)

    def cancel(self, job_id: int) -> int:
        return knnjoin_cancel(self.ctx, job_id)

    def stats(self, job_id: int = 0) -> dict:
        return knnjoin_get_stats(self.ctx, job_id)

    def last_error(self) -> str:
        return knnjoin_last_error(self.ctx)


class Index:
    """A resident index of one point set (knnjoin_index_*): built once, then
    queried with batches of query points; freed by close() or with its
    context."""

    def __init__(self, ctx: Context, handle: int, n: int, d: int):
        self._ctx = ctx
        self.handle = handle
        self.n = n
        self.d = d

    def query(self, queries, K: int, out_ids=None, out_dist=None):
        """For each row of the float32 [nq, d] `queries`, the K nearest indexed
        points (nothing excluded): (ids int32 [nq, K], dist float64 [nq, K]) on
        the queries' device."""
        torch = self._ctx._torch
        if not self.handle:
            raise ValueError("index is closed")
        if queries.dtype != torch.float32 or queries.dim() != 2 or queries.shape[1] != self.d:
            raise ValueError("queries must be a float32 [nq, d] tensor with the index's d")
        queries = queries.contiguous()
        nq = queries.shape[0]
        out_ids, out_dist = self._ctx._outputs(nq, K, queries, out_ids, out_dist)
        knnjoin_index_query(self._ctx.ctx, self.handle, queries.data_ptr(), nq, K, out_ids.data_ptr(),
                            out_dist.data_ptr())
        return out_ids, out_dist

    def stats(self) -> dict:
        return knnjoin_index_stats(self.handle)

    def close(self) -> None:
        if self.handle and getattr(self._ctx, "ctx", None):
            knnjoin_index_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
