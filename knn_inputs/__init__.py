"""Seeded synthetic point sets for the KNN self-join (inputs only).

This module generates inputs and nothing else: it holds none of the join's
arithmetic, so both the CPU oracle and the GPU library can be fed from it
without sharing any code of the method.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: value number c of a stream with key k is mix(k + (c + 1) * gamma).
Everything is vectorised with numpy uint64 arithmetic (wrapping), so the
same (seed, name, job) always yields bit-identical points on any machine.

Workload shapes follow the paper's synthetic classes (Sec. 5.1): uniformly
distributed points, and exponentially distributed points with rate 40, in
2, 4 and 6 dimensions; n is scaled to the sizes this library is measured on.
"""
from __future__ import annotations

import hashlib
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, name: str, job: int = 0) -> int:
    """64-bit stream key for (seed, config name, job index)."""
    h = hashlib.sha256(f"{seed}|{name}|{job}".encode()).digest()
    return int.from_bytes(h[:8], "little")


def raw_u64(key: int, count: int, offset: int = 0) -> np.ndarray:
    """Values offset .. offset+count-1 of the SplitMix64 stream `key`."""
    with np.errstate(over="ignore"):
        c = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(key) + c * GAMMA
        return _mix(z)


def uniform_f32(key: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform [0,1) on the 2^-24 grid: (r >> 40) * 2^-24, exact in float32."""
    r = raw_u64(key, count, offset) >> np.uint64(40)
    return (r.astype(np.float64) * 2.0 ** -24).astype(np.float32)


def uniform_f64(key: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform [0,1) with 53 bits: (r >> 11) * 2^-53."""
    r = raw_u64(key, count, offset) >> np.uint64(11)
    return r.astype(np.float64) * 2.0 ** -53


def points_uniform(n: int, d: int, key: int) -> np.ndarray:
    """n x d float32, i.i.d. uniform [0,1) per coordinate (row-major)."""
    return uniform_f32(key, n * d).reshape(n, d)


def points_expo(n: int, d: int, key: int, rate: float = 40.0) -> np.ndarray:
    """n x d float32, i.i.d. exponential(rate) per coordinate, clipped below 1.

    x = -log1p(-u) / rate with u a 53-bit uniform in [0,1), rounded to
    float32; a value >= 1 (probability e^-40 per coordinate) becomes the
    largest float32 below 1.
    """
    u = uniform_f64(key, n * d)
    x = (-np.log1p(-u) / rate).astype(np.float32)
    x[x >= np.float32(1.0)] = np.nextafter(np.float32(1.0), np.float32(0.0))
    return x.reshape(n, d)


def points_clustered2d(n: int, key: int, frac_band: float = 0.7,
                       sigma: float = 0.02) -> np.ndarray:
    """n x 2 float32: a share `frac_band` of the points has x ~ U[0,1) and
    y ~ N(0.5, sigma) (redrawn until inside [0,1)); the rest is uniform.

    Normals come from the Box-Muller transform of two 53-bit uniforms.
    """
    u = uniform_f64(key, 4 * n).reshape(n, 4)
    x = u[:, 0].copy()
    y = u[:, 1].copy()
    band = u[:, 2] < frac_band
    rr = np.sqrt(-2.0 * np.log1p(-u[:, 3]))
    # second uniform for the angle comes from a separate stream offset
    th = 2.0 * np.pi * uniform_f64(key, n, offset=4 * n)
    g = 0.5 + sigma * rr * np.cos(th)
    bad = band & ((g < 0.0) | (g >= 1.0))
    extra = 0
    while bad.any():
        k = int(bad.sum())
        v = uniform_f64(key, 2 * k, offset=5 * n + extra).reshape(k, 2)
        extra += 2 * k
        g2 = 0.5 + sigma * np.sqrt(-2.0 * np.log1p(-v[:, 0])) * np.cos(2 * np.pi * v[:, 1])
        g[bad] = g2
        bad = band & ((g < 0.0) | (g >= 1.0))
    y[band] = g[band]
    pts = np.stack([x, y], axis=1).astype(np.float32)
    pts[pts >= np.float32(1.0)] = np.nextafter(np.float32(1.0), np.float32(0.0))
    return pts


def points_lattice(m: int, d: int, scale: float = 1.0) -> np.ndarray:
    """All integer points of {0..m-1}^d times `scale`, row-major order
    (last coordinate varies fastest), float32."""
    grids = np.meshgrid(*([np.arange(m, dtype=np.float64)] * d), indexing="ij")
    pts = np.stack([g.reshape(-1) for g in grids], axis=1) * scale
    return pts.astype(np.float32)


def points_duplicates(copies: int, sites: int, d: int, key: int) -> np.ndarray:
    """`copies` copies of each of `sites` uniform sites, shuffled order."""
    s = points_uniform(sites, d, key)
    pts = np.repeat(s, copies, axis=0)
    perm = np.argsort(raw_u64(key, pts.shape[0], offset=sites * d), kind="stable")
    return pts[perm]


def points_columns(columns: int, per_column: int, key: int, jitter_bits: int = 16,
                   jitter_scale: float = 2.0 ** -29) -> np.ndarray:
    """Two-dimensional points on `columns` integer x positions with
    `per_column` points each; y = k * jitter_scale, k uniform in
    [0, 2^jitter_bits).  Distances across columns differ only in terms far
    below single precision, so FP32 squared distances tie where the exact
    ones do not.  Shuffled order, float32."""
    m = columns * per_column
    x = np.repeat(np.arange(columns, dtype=np.float64), per_column)
    k = raw_u64(key, m) >> np.uint64(64 - jitter_bits)
    y = k.astype(np.float64) * jitter_scale
    pts = np.stack([x, y], axis=1)
    perm = np.argsort(raw_u64(key, m, offset=m), kind="stable")
    return pts[perm].astype(np.float32)


def permutation(n: int, key: int) -> np.ndarray:
    """A seeded permutation of range(n)."""
    return np.argsort(raw_u64(key, n), kind="stable")


# ---------------------------------------------------------------------------
# Named workloads (the paper's Unif / Expo classes at this library's sizes)
# ---------------------------------------------------------------------------
CONFIGS = {
    "unif2d_20k": dict(kind="uniform", n=20_000, d=2, K=8),
    "unif2d_2m": dict(kind="uniform", n=2_000_000, d=2, K=32),
    "unif4d_2m": dict(kind="uniform", n=2_000_000, d=4, K=32),
    "unif6d_2m": dict(kind="uniform", n=2_000_000, d=6, K=32),
    "expo2d_2m": dict(kind="expo", n=2_000_000, d=2, K=64),
    "expo4d_2m": dict(kind="expo", n=2_000_000, d=4, K=64),
    "expo6d_2m": dict(kind="expo", n=2_000_000, d=6, K=64),
}


def make_points(kind: str, n: int, d: int, seed: int = 0, name: str = "",
                job: int = 0) -> np.ndarray:
    key = stream_key(seed, name or f"{kind}{d}d_{n}", job)
    if kind == "uniform":
        return points_uniform(n, d, key)
    if kind == "expo":
        return points_expo(n, d, key)
    if kind == "clustered2d":
        if d != 2:
            raise ValueError("clustered2d is two-dimensional")
        return points_clustered2d(n, key)
    raise ValueError(f"unknown kind {kind!r}")


def config_points(name: str, seed: int = 0, n: int | None = None) -> tuple[np.ndarray, int]:
    """(points, K) for a named workload; `n` overrides the size (same stream)."""
    c = CONFIGS[name]
    nn = c["n"] if n is None else n
    return make_points(c["kind"], nn, c["d"], seed=seed, name=name), c["K"]


def batched_jobs(count: int = 256, seed: int = 0, n_lo: int = 1000,
                 n_hi: int = 200_000) -> list[dict]:
    """Job list of the batched workload: n log-uniform in [n_lo, n_hi],
    d in {2,3,4,6}, K in {4,8,16,32,64}, uniform or exponential(40) 50/50."""
    key = stream_key(seed, "batched", 0)
    u = uniform_f64(key, 4 * count).reshape(count, 4)
    jobs = []
    for j in range(count):
        n = int(np.exp(np.log(n_lo) + u[j, 0] * (np.log(n_hi) - np.log(n_lo))))
        d = (2, 3, 4, 6)[int(u[j, 1] * 4)]
        K = (4, 8, 16, 32, 64)[int(u[j, 2] * 5)]
        kind = "uniform" if u[j, 3] < 0.5 else "expo"
        jobs.append(dict(kind=kind, n=n, d=d, K=min(K, n - 1), job=j))
    return jobs


def batched_points(job: dict, seed: int = 0) -> np.ndarray:
    return make_points(job["kind"], job["n"], job["d"], seed=seed, name="batched",
                       job=job["job"])


def served_jobs(count: int = 500, seed: int = 0, n_lo: int = 10_000,
                n_hi: int = 5_000_000) -> list[dict]:
    """Job list of the served workload (arrival times are set by the caller):
    n log-uniform in [n_lo, n_hi], d uniform in 2..6, K log-uniform in
    [8, 128], a third each uniform, exponential(40), clustered 2-D."""
    key = stream_key(seed, "served", 0)
    u = uniform_f64(key, 5 * count).reshape(count, 5)
    jobs = []
    for j in range(count):
        n = int(np.exp(np.log(n_lo) + u[j, 0] * (np.log(n_hi) - np.log(n_lo))))
        kind = ("uniform", "expo", "clustered2d")[int(u[j, 3] * 3)]
        d = 2 if kind == "clustered2d" else 2 + int(u[j, 1] * 5)
        K = int(round(np.exp(np.log(8) + u[j, 2] * (np.log(128) - np.log(8)))))
        jobs.append(dict(kind=kind, n=n, d=d, K=min(K, n - 1), job=j,
                         u_arrival=float(u[j, 4])))
    return jobs


def served_points(job: dict, seed: int = 0) -> np.ndarray:
    return make_points(job["kind"], job["n"], job["d"], seed=seed, name="served",
                       job=job["job"])
