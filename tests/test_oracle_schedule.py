"""Pins of the oracle's work count (W_ref) and search-distance selection.

The grid join of the oracle (paper Sec. 3.1 grid index, Alg. 1 ring of 3^n
adjacent cells, failed queries retried on a grid of twice the cell side)
counts the candidate distance evaluations of its schedule; that count, W_ref,
is the numerator of every roofline figure.  The Sec. 4.4 selection of the
search distance (mean pairwise distance of a 0.1% sample, a histogram of
sampled distances in 1024 bins of width eps_mean / 1024, eps_min = the middle
of the first bin whose cumulative count per sampled point reaches K) sets the
schedule's cell side.  Both are pinned here against facts computed without
the oracle's code:

* on integer lattices where every query is certified in the first pass, the
  count is a closed form over cells: c^d points per cell, each seeing the
  c^d points of every in-grid neighbour cell but itself;
* on random integer sets with several passes, an independent NumPy
  restatement of the schedule (box membership by cell coordinates, exact
  integer certificate) gives the count per pass;
* on lattices small enough that every point is sampled, the distance
  histogram follows from counts of lattice offsets (an offset o occurs
  prod_k (m - |o_k|) times), which fixes eps_min in closed form; a 1-D line
  with strided sampling pins the sampling strides.

Three planted mistakes (counting only the last pass, counting the query
itself, histogram bins shifted by one) must each fail one of these pins.
"""
import itertools
import math

import numpy as np
import pytest

import knn_inputs as gen
import oracle


# --------------------------------------------------------------------------
# W_ref: candidate count of the grid schedule
# --------------------------------------------------------------------------
def lattice_first_pass_count(m: int, c: int, d: int) -> int:
    """Candidates when every query of {0..m-1}^d certifies at level 0 with
    cell side c (c divides m): a cell holds c^d points, and each of them
    evaluates the points of the in-grid cells within one step of its own
    cell, minus itself."""
    g = m // c  # cells per dimension
    per_dim = [min(u + 1, g - 1) - max(u - 1, 0) + 1 for u in range(g)]  # in-grid neighbours
    total = 0
    for cell in itertools.product(range(g), repeat=d):
        box_cells = math.prod(per_dim[u] for u in cell)
        total += c ** d * (box_cells * c ** d - 1)
    return total


def schedule_counts(p: np.ndarray, K: int, w: int):
    """(queries, candidates) per pass of the grid schedule on integer points
    with integer cell side w, written from its description: at level l the
    cell of a point is floor(x / w) >> l per coordinate; a query evaluates
    every other point whose level cell is within one step of its own in all
    dimensions; it is certified when it has at least K such points and the
    K-th smallest squared distance is strictly below R^2, R = the distance
    from the query to the nearest face of its 3^d box beyond which cells of
    points exist (no such face: certified); the others move up a level."""
    x = p.astype(np.int64)
    n, d = x.shape
    c0 = np.floor_divide(x, w)
    active = np.arange(n)
    queries, cands = [], []
    lvl = 0
    while active.size:
        cl = np.floor_divide(c0, 2 ** lvl)
        cmin, cmax = cl.min(axis=0), cl.max(axis=0)
        wl = w * 2 ** lvl
        total = 0
        failed = []
        for i in active:
            member = np.all(np.abs(cl - cl[i]) <= 1, axis=1)
            member[i] = False
            idx = np.nonzero(member)[0]
            total += int(idx.size)
            ok = False
            if idx.size >= K:
                dk = int(np.sort(((x[idx] - x[i]) ** 2).sum(axis=1))[K - 1])
                r2 = None
                for k in range(d):
                    gaps = []
                    if cl[i, k] - 1 > cmin[k]:
                        gaps.append(int(x[i, k] - (cl[i, k] - 1) * wl))
                    if cl[i, k] + 1 < cmax[k]:
                        gaps.append(int((cl[i, k] + 2) * wl - x[i, k]))
                    for g in gaps:
                        r2 = g * g if r2 is None else min(r2, g * g)
                ok = r2 is None or dk < r2
            if not ok:
                failed.append(i)
        queries.append(int(active.size))
        cands.append(total)
        active = np.array(failed, dtype=np.int64)
        lvl += 1
    return queries, cands


def integer_points(n, d, span, seed):
    key = gen.stream_key(seed, "int-points", n * 10 + d)
    return (gen.raw_u64(key, n * d) % np.uint64(span)).astype(np.float32).reshape(n, d)


@pytest.mark.parametrize("m,c,d,K", [(12, 3, 2, 4), (12, 4, 2, 8), (8, 2, 3, 6), (6, 3, 1, 2)])
def test_wref_lattice_closed_form(m, c, d, K):
    lat = gen.points_lattice(m, d)
    _, _, st = oracle.grid(lat, K, width_mult=-float(c))
    assert st["passes"] == 1  # every K-th lattice neighbour lies inside the box faces
    assert st["pass_queries"] == [m ** d]
    assert st["pass_candidates"] == [lattice_first_pass_count(m, c, d)]
    assert st["candidates"] == lattice_first_pass_count(m, c, d)


@pytest.mark.parametrize("n,d,span,w,K,seed", [(400, 2, 64, 4, 8, 1), (300, 3, 32, 4, 6, 2),
                                               (200, 1, 512, 8, 5, 3), (250, 4, 16, 4, 10, 4)])
def test_wref_multi_pass_restatement(n, d, span, w, K, seed):
    p = integer_points(n, d, span, seed)
    q, c = schedule_counts(p, K, w)
    assert len(q) >= 2  # the case exercises re-queued passes
    _, _, st = oracle.grid(p, K, width_mult=-float(w))
    assert st["passes"] == len(q)
    assert st["pass_queries"] == q
    assert st["pass_candidates"] == c
    assert st["candidates"] == sum(c)


# --------------------------------------------------------------------------
# Sec. 4.4 search distance
# --------------------------------------------------------------------------
def lattice_epsilon(m: int, d: int, K: int):
    """(eps_min, eps_mean) of the selection on {0..m-1}^d (row-major order,
    n = m^d <= 500, so the histogram samples every point and the mean
    distance uses the two strided samples 0 and n // 2)."""
    n = m ** d
    assert n <= 500 and round(0.001 * n) <= 2
    half = n // 2
    coords = [(half // m ** (d - 1 - k)) % m for k in range(d)]
    eps_mean = math.sqrt(float(sum(v * v for v in coords)))
    bw = eps_mean / 1024
    # ordered pairs at squared distance s: offsets o != 0 with |o|^2 = s
    pairs = {}
    for o in itertools.product(range(-(m - 1), m), repeat=d):
        s = sum(v * v for v in o)
        if s:
            pairs[s] = pairs.get(s, 0) + math.prod(m - abs(v) for v in o)
    hist = {}
    for s, cnt in pairs.items():
        dist = math.sqrt(float(s))
        if dist < eps_mean:
            b = min(int(dist / bw), 1023)
            hist[b] = hist.get(b, 0) + cnt
    cum = 0
    for b in range(1024):
        cum += hist.get(b, 0)
        if cum / n >= K:
            return (b + 0.5) * bw, eps_mean
    return eps_mean, eps_mean


@pytest.mark.parametrize("m,d,K", [(20, 2, 4), (20, 2, 12), (7, 3, 6), (4, 4, 10), (300, 1, 8),
                                   (22, 2, 30)])
def test_epsilon_lattice_closed_form(m, d, K):
    want_min, want_mean = lattice_epsilon(m, d, K)
    got_min, got_mean = oracle.select_epsilon(gen.points_lattice(m, d), K)
    assert got_mean == want_mean
    assert got_min == want_min


def line_epsilon(n: int, K: int):
    """Selection on the 1-D line 0..n-1 with strided samples: sm = round(n /
    1000) mean-distance samples at multiples of n // sm, and S = 500
    histogram samples at multiples of n // 500; the sample at p has 2
    neighbours at each distance t <= min(p, n-1-p) and 1 up to max(...)."""
    sm = round(0.001 * n)
    assert 2 < sm <= 2000 and n >= 500
    st = n // sm
    tot = sum(st * (b - a) for a in range(sm) for b in range(a + 1, sm))
    eps_mean = tot / (sm * (sm - 1) // 2)
    bw = eps_mean / 1024
    samples = [s * (n // 500) for s in range(500)]
    cum = 0
    t = 1
    bin_of = lambda t: min(int(float(t) / bw), 1023)
    b = 0
    while t < eps_mean:
        cnt = sum((t <= p) + (t <= n - 1 - p) for p in samples)
        if bin_of(t) != b:
            if cum / 500 >= K:
                return (b + 0.5) * bw, eps_mean
            b = bin_of(t)
        cum += cnt
        t += 1
    if cum / 500 >= K:
        return (b + 0.5) * bw, eps_mean
    return eps_mean, eps_mean


@pytest.mark.parametrize("n,K", [(5000, 8), (5000, 40), (12000, 3)])
def test_epsilon_strided_line(n, K):
    want_min, want_mean = line_epsilon(n, K)
    line = np.arange(n, dtype=np.float32).reshape(n, 1)
    got_min, got_mean = oracle.select_epsilon(line, K)
    assert got_mean == pytest.approx(want_mean, rel=1e-15)
    assert got_min == pytest.approx(want_min, rel=1e-15)


# --------------------------------------------------------------------------
# planted mistakes
# --------------------------------------------------------------------------
def schedule_pins_fail(mutant):
    lat = gen.points_lattice(12, 2)
    _, _, st = oracle.grid(lat, 4, width_mult=-3.0, mutant=mutant)
    if st["pass_candidates"] != [lattice_first_pass_count(12, 3, 2)] or \
            st["candidates"] != lattice_first_pass_count(12, 3, 2):
        return True
    p = integer_points(400, 2, 64, 1)
    q, c = schedule_counts(p, 8, 4)
    _, _, st = oracle.grid(p, 8, width_mult=-4.0, mutant=mutant)
    if st["pass_queries"] != q or st["pass_candidates"] != c or st["candidates"] != sum(c):
        return True
    for m, d, K in [(20, 2, 4), (7, 3, 6)]:
        if oracle.select_epsilon(gen.points_lattice(m, d), K, mutant=mutant) != lattice_epsilon(m, d, K):
            return True
    return False


@pytest.mark.parametrize("mutant", oracle.SCHEDULE_MUTANTS)
def test_schedule_pins_catch_planted_mistakes(mutant):
    assert schedule_pins_fail(mutant)


def test_schedule_pins_pass_unmutated():
    assert not schedule_pins_fail(None)
