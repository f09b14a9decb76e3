"""Kernel-level checks of the grid index (steps a3-a5: Sec. 3.1 grid index,
Sec. 4.6 GPU indexing) through knnjoin_index_dump.

The dump returns what a join builds: the sorted Morton keys, the sort's
permutation, the grid, and the runs the level's cell table (dense table or
hash map) returns for probe keys.  Each is checked against a CPU restatement
that shares nothing with the library:

* cell assignment: every point lies in the cell its key encodes, with the
  faces fl32(c w0 + lo) computed exactly (rational arithmetic, one rounding
  to float32) and the clamping to [0, cmax0];
* keys: the Morton interleave of those cells (bit b of coordinate k at key
  bit b d + k);
* sort: the permutation is numpy's stable argsort of the points' keys
  (equal keys keep their original order) and the keys come out sorted;
* runs and cell table: every present cell's [begin, end) equals the run of
  equal keys (numpy unique), at level 0, a coarser level and the top level;
  absent cells and keys beyond the level's grid return (0, 0).
"""
from fractions import Fraction

import numpy as np
import pytest

import knn_inputs as gen

pytestmark = pytest.mark.gpu


def f32_round(x: Fraction) -> np.float32:
    """Correctly rounded float32 (round half to even) of an exact rational
    in the normal range."""
    if x == 0:
        return np.float32(0.0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    scaled = a / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    q, r = divmod(scaled.numerator, scaled.denominator)
    if 2 * r > scaled.denominator or (2 * r == scaled.denominator and q % 2 == 1):
        q += 1
    return np.float32(sign * float(Fraction(q) * Fraction(2) ** (e - 23)))


def faces(w0: float, lo: float, cmax: int) -> np.ndarray:
    """fl32(c w0 + lo) for c = 0 .. cmax + 1 (a single rounding, as fmaf)."""
    W, O = Fraction(float(np.float32(w0))), Fraction(float(np.float32(lo)))
    return np.array([f32_round(c * W + O) for c in range(cmax + 2)], np.float32)


def morton(cells: np.ndarray, bits: int) -> np.ndarray:
    n, d = cells.shape
    key = np.zeros(n, np.uint64)
    for b in range(bits):
        for k in range(d):
            key |= ((cells[:, k].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(b * d + k)
    return key


def demorton(keys: np.ndarray, d: int, bits: int) -> np.ndarray:
    c = np.zeros((len(keys), d), np.int64)
    for b in range(bits):
        for k in range(d):
            c[:, k] |= ((keys >> np.uint64(b * d + k)) & np.uint64(1)).astype(np.int64) << b
    return c


SETS = [("uniform", 50000, 2, 8, 1), ("uniform", 30000, 6, 16, 2), ("expo", 60000, 2, 16, 3),
        ("expo", 40000, 3, 8, 4), ("clustered2d", 50000, 2, 8, 5), ("uniform", 20000, 4, 32, 6)]


@pytest.fixture(scope="module")
def kj():
    import paper_1810_04758_b300 as m
    from paper_1810_04758_b300 import build
    build.build()
    m.load_library()
    return m


def dump(kj, ctx, p, K, level=0, probe=None):
    import torch
    t = torch.from_numpy(p).cuda()
    return kj.knnjoin_index_dump(ctx.ctx, t.data_ptr(), len(p), p.shape[1], K, level, probe)


@pytest.mark.parametrize("kind,n,d,K,seed", SETS)
def test_keys_sort_and_cells(kj, kind, n, d, K, seed):
    p = gen.make_points(kind, n, d, seed=seed)
    with kj.Context(0) as ctx:
        keys, perm, g, _ = dump(kj, ctx, p, K)
    bits = g["bits"]
    # the sort: a permutation, keys ascending, equal keys in original order
    assert np.array_equal(np.sort(perm), np.arange(n, dtype=np.uint32))
    assert (keys[1:] >= keys[:-1]).all()
    by_point = np.empty(n, np.uint64)
    by_point[perm] = keys
    np.testing.assert_array_equal(perm, np.argsort(by_point, kind="stable").astype(np.uint32))
    # every point lies in the cell its key encodes (exact faces, clamped)
    cells = demorton(by_point, d, bits)
    np.testing.assert_array_equal(morton(cells, bits), by_point)
    for k in range(d):
        cm = int(g["cmax0"][k])
        assert (cells[:, k] >= 0).all() and (cells[:, k] <= cm).all()
        f = faces(g["w0"], g["lo"][k], cm)
        x = p[:, k]
        c = cells[:, k]
        lower_ok = (c == 0) | (f[c] <= x)
        upper_ok = (c == cm) | (x < f[np.minimum(c + 1, cm + 1)])
        assert lower_ok.all() and upper_ok.all(), (k, int((~lower_ok).sum()), int((~upper_ok).sum()))


@pytest.mark.parametrize("kind,n,d,K,seed", SETS)
def test_cell_tables(kj, kind, n, d, K, seed):
    p = gen.make_points(kind, n, d, seed=seed)
    rng = np.random.default_rng(seed)
    with kj.Context(0) as ctx:
        keys, perm, g, _ = dump(kj, ctx, p, K)
        bits = g["bits"]
        kinds = set()
        for level in sorted({0, min(1, bits), min(2, bits), bits}):
            nb = bits - level
            lk = keys >> np.uint64(d * level)
            uk, first, count = np.unique(lk, return_index=True, return_counts=True)
            cmaxL = np.array([int(c) >> level for c in g["cmax0"]])
            # absent cells inside the grid, and keys beyond it
            cand = np.stack([rng.integers(0, cm + 1, 4000) for cm in cmaxL], axis=1)
            ck = morton(cand, nb)
            absent = np.setdiff1d(ck, uk)
            beyond = []
            for k in range(d):
                if cmaxL[k] + 1 < (1 << nb):
                    c = np.zeros((1, d), np.int64)
                    c[0, k] = cmaxL[k] + 1
                    beyond.append(morton(c, nb)[0])
            if nb * d < 64:
                beyond.append(np.uint64(1) << np.uint64(nb * d))
            probe = np.concatenate([uk, absent, np.array(beyond, np.uint64)])
            _, _, g2, runs = dump(kj, ctx, p, K, level, probe)
            kinds.add(g2["dense_table"])
            m = len(uk)
            np.testing.assert_array_equal(runs[:m, 0], first.astype(np.uint32))
            np.testing.assert_array_equal(runs[:m, 1], (first + count).astype(np.uint32))
            assert (runs[m:] == 0).all()
            if level == bits:
                assert m == 1 and runs[0, 0] == 0 and runs[0, 1] == n  # the whole grid is one cell
    assert kinds <= {0, 1}


def test_both_table_kinds_are_exercised(kj):
    """The sets above reach a dense table and a hash map at some level."""
    seen = set()
    with kj.Context(0) as ctx:
        for kind, n, d, K, seed in SETS:
            p = gen.make_points(kind, n, d, seed=seed)
            keys, _, g, _ = dump(kj, ctx, p, K)
            for level in (0, 1):
                _, _, g2, _ = dump(kj, ctx, p, K, level, keys[:1] >> np.uint64(d * level))
                seen.add(g2["dense_table"])
    assert seen == {0, 1}


def test_dump_errors(kj):
    import torch
    p = gen.make_points("uniform", 3000, 3, seed=8)
    t = torch.from_numpy(p).cuda()
    with kj.Context(0) as ctx:
        _, _, g, _ = kj.knnjoin_index_dump(ctx.ctx, t.data_ptr(), 3000, 3, 8)
        with pytest.raises(kj.KnnJoinError) as e:
            kj.knnjoin_index_dump(ctx.ctx, t.data_ptr(), 3000, 3, 8, g["bits"] + 1, np.zeros(1, np.uint64))
        assert e.value.status == kj.KNN_ERR_INVALID
        with pytest.raises(kj.KnnJoinError):
            kj.knnjoin_index_dump(ctx.ctx, t.data_ptr(), 3000, 3, 3000)  # K > n - 1
        # the context still joins afterwards
        ids, _ = ctx.self_join(t, 8)
        torch.cuda.synchronize()
        assert ids.shape == (3000, 8)
