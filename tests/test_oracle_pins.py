"""Pins of the CPU oracle against facts outside itself.

The oracle's definition (paper Sec. 2.1): K nearest neighbours of every point
under the Euclidean distance, the point itself excluded; ties broken by index
and distances evaluated in canonical FP64 (that reading is stated in the
oracle's header).  Each test below checks it against something the paper or
mathematics fixes independently of the oracle's code:

* exact rational arithmetic (fractions) on inputs where FP64 is exact;
* closed forms on integer lattices (shell structure of Z^d);
* the full sort (K = n - 1) and a two-pointer merge in one dimension;
* duplicate sets (copies at distance 0, lowest ids first);
* invariants (sorted rows, prefix property, completeness);
* the grid join against brute force, and the certificate's strictness on a
  point that sits exactly on a face of the scanned box.

The mutation tests build the oracle with one planted mistake each and check
that at least one pin fails.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import knn_inputs as gen
import oracle


def exact_knn(points, K):
    """Exact rational (distance^2, id) ranking of all pairs."""
    pts = [[Fraction(float(v)) for v in row] for row in points]
    n = len(pts)
    ids = np.empty((n, K), np.int32)
    d2 = [[None] * K for _ in range(n)]
    for i in range(n):
        cand = []
        for j in range(n):
            if j == i:
                continue
            s = sum((a - b) ** 2 for a, b in zip(pts[i], pts[j]))
            cand.append((s, j))
        cand.sort()
        for k in range(K):
            ids[i, k] = cand[k][1]
            d2[i][k] = cand[k][0]
    return ids, d2


def quantized(n, d, seed, levels=16, scale=2.0 ** -4):
    """Coordinates on a coarse dyadic grid: every FP64 step is exact, and
    there are many equal distances."""
    key = gen.stream_key(seed, "quantized", n * 100 + d)
    r = gen.raw_u64(key, n * d) % np.uint64(levels)
    return (r.astype(np.float64) * scale).astype(np.float32).reshape(n, d)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n,K", [(12, 1), (33, 5), (48, 11)])
def test_bf_matches_exact_rational(d, n, K):
    p = quantized(n, d, seed=d)
    ids, dist = oracle.bf(p, K)
    eids, ed2 = exact_knn(p, K)
    np.testing.assert_array_equal(ids, eids)
    for i in range(n):
        for k in range(K):
            # D is exact here, so the reported distance is sqrt of the exact value
            assert dist[i, k] == math.sqrt(float(ed2[i][k]))


def test_bf_full_sort_is_k_equals_n_minus_1():
    p = quantized(40, 3, seed=11, levels=6)
    n = len(p)
    ids, dist = oracle.bf(p, n - 1)
    eids, _ = exact_knn(p, n - 1)
    np.testing.assert_array_equal(ids, eids)


def exact_knn_rs(queries, points, K):
    """Exact rational (distance^2, id) ranking of every (query, data point)
    pair, nothing excluded."""
    qs = [[Fraction(float(v)) for v in row] for row in queries]
    ps = [[Fraction(float(v)) for v in row] for row in points]
    ids = np.empty((len(qs), K), np.int32)
    d2 = [[None] * K for _ in range(len(qs))]
    for r, q in enumerate(qs):
        cand = sorted((sum((a - b) ** 2 for a, b in zip(q, p)), j) for j, p in enumerate(ps))
        for k in range(K):
            ids[r, k] = cand[k][1]
            d2[r][k] = cand[k][0]
    return ids, d2


@pytest.mark.parametrize("d", [1, 2, 3, 6])
@pytest.mark.parametrize("nq,n,K", [(7, 20, 1), (25, 40, 9), (30, 12, 12)])
def test_bf_rs_matches_exact_rational(d, nq, n, K):
    # R x S on the coarse dyadic grid: ties everywhere, K up to n (no exclusion)
    q = quantized(nq, d, seed=100 + d)
    p = quantized(n, d, seed=200 + d)
    ids, dist = oracle.bf_rs(q, p, K)
    eids, ed2 = exact_knn_rs(q, p, K)
    np.testing.assert_array_equal(ids, eids)
    for r in range(nq):
        for k in range(K):
            assert dist[r, k] == math.sqrt(float(ed2[r][k]))


@pytest.mark.parametrize("kind,d", [("uniform", 3), ("expo", 2), ("clustered2d", 2)])
def test_bf_rs_of_a_set_with_itself_is_the_self_join(kind, d):
    # R = S with K + 1 neighbours: each row holds the query's own index; with
    # it removed the row is the self-join's row (pinned above)
    p = gen.make_points(kind, 600, d, seed=5)
    K = 12
    ids_rs, dist_rs = oracle.bf_rs(p, p, K + 1)
    ids, dist = oracle.bf(p, K)
    for i in range(len(p)):
        keep = ids_rs[i] != i
        assert (~keep).sum() == 1
        np.testing.assert_array_equal(ids_rs[i][keep], ids[i])
        np.testing.assert_array_equal(dist_rs[i][keep], dist[i])


def test_exact_vs_canonical_on_generic_floats():
    """On generic (non-dyadic-grid) floats canonical FP64 may in principle
    reorder near-equal distances; count how often -- expected 0 here."""
    key = gen.stream_key(3, "generic", 0)
    p = (gen.uniform_f64(key, 50 * 4).reshape(50, 4) * 3.7 - 1.1).astype(np.float32)
    ids, _ = oracle.bf(p, 10)
    eids, _ = exact_knn(p, 10)
    assert (ids != eids).sum() == 0


def shell_offsets(d, rho):
    offs = [o for o in itertools.product(range(-rho, rho + 1), repeat=d) if any(o)]
    return offs


@pytest.mark.parametrize("d,m,K", [(1, 25, 6), (2, 15, 12), (2, 15, 21), (3, 9, 26), (3, 9, 33)])
@pytest.mark.parametrize("scale", [1.0, 2.0 ** -3])
def test_lattice_closed_form(d, m, K, scale):
    """Interior points of {0..m-1}^d: the neighbours are idx(p) + L(o) for the
    integer offsets o sorted by (|o|^2, L(o)), L the row-major offset."""
    p = gen.points_lattice(m, d, scale)
    ids, dist = oracle.bf(p, K)
    rho = 1
    while True:
        offs = shell_offsets(d, rho)
        norms = sorted(sum(c * c for c in o) for o in offs)
        if len(norms) >= K and norms[K - 1] < (rho + 1) ** 2:  # all offsets up to that norm lie in the box
            break
        rho += 1
    strides = [m ** (d - 1 - k) for k in range(d)]
    ranked = sorted(offs, key=lambda o: (sum(c * c for c in o), sum(c * s for c, s in zip(o, strides))))
    want_off = [sum(c * s for c, s in zip(o, strides)) for o in ranked[:K]]
    want_d = [math.sqrt(sum(c * c for c in o)) * scale for o in ranked[:K]]
    # K-th distance = sqrt of the smallest shell s whose cumulative count reaches K
    shells = {}
    for o in offs:
        s = sum(c * c for c in o)
        shells[s] = shells.get(s, 0) + 1
    cum = 0
    for s in sorted(shells):
        cum += shells[s]
        if cum >= K:
            kth = math.sqrt(s) * scale
            break
    checked = 0
    for idx in range(len(p)):
        coord = [(idx // strides[k]) % m for k in range(d)]
        if all(rho <= c < m - rho for c in coord):
            np.testing.assert_array_equal(ids[idx], np.array(want_off) + idx)
            np.testing.assert_array_equal(dist[idx], np.array(want_d))
            assert dist[idx, K - 1] == kth
            checked += 1
    assert checked > 0


def test_lattice_permuted_order():
    """Shuffling the input order permutes the rows and relabels the ids: each
    row keeps its distances, and equal distances are ordered by the new ids."""
    d, m, K = 2, 13, 9
    base = gen.points_lattice(m, d)
    perm = gen.permutation(len(base), gen.stream_key(0, "perm", 0))
    p = base[perm]
    ids0, dist0 = oracle.bf(base, K)
    ids1, dist1 = oracle.bf(p, K)
    for r in range(len(p)):
        orig = perm[r]
        np.testing.assert_array_equal(dist1[r], dist0[orig])
        for k in range(K - 1):
            if dist1[r, k] == dist1[r, k + 1]:
                assert ids1[r, k] < ids1[r, k + 1]
        # strictly closer neighbours than the K-th are the same points
        inner0 = set(ids0[orig][dist0[orig] < dist0[orig, K - 1]].tolist())
        inner1 = set(perm[ids1[r][dist1[r] < dist1[r, K - 1]]].tolist())
        assert inner0 == inner1


def two_pointer_1d(x, K):
    """K nearest neighbours in 1-D by merging the sorted left and right sides."""
    n = len(x)
    vals = sorted(set(x.tolist()))
    groups = {v: sorted(np.nonzero(x == v)[0].tolist()) for v in vals}
    pos = {v: i for i, v in enumerate(vals)}
    out = np.empty((n, K), np.int32)
    for i in range(n):
        v = float(x[i])
        res = [j for j in groups[v] if j != i]
        lo, hi = pos[v] - 1, pos[v] + 1
        while len(res) < K:
            dl = v - vals[lo] if lo >= 0 else math.inf
            dh = vals[hi] - v if hi < len(vals) else math.inf
            if dl < dh:
                res += groups[vals[lo]]; lo -= 1
            elif dh < dl:
                res += groups[vals[hi]]; hi += 1
            else:
                res += sorted(groups[vals[lo]] + groups[vals[hi]]); lo -= 1; hi += 1
        out[i] = res[:K]
    return out


def test_one_dimension_two_pointer():
    x = quantized(200, 1, seed=5, levels=64).reshape(-1)
    ids, _ = oracle.bf(x.reshape(-1, 1), 7)
    np.testing.assert_array_equal(ids, two_pointer_1d(x, 7))


def test_duplicates_first_copies():
    copies, sites, d, K = 6, 40, 3, 9
    p = gen.points_duplicates(copies, sites, d, gen.stream_key(0, "dup", 0))
    assert len(np.unique(p, axis=0)) == sites
    ids, dist = oracle.bf(p, K)
    for i in range(len(p)):
        twins = [j for j in range(len(p)) if j != i and np.array_equal(p[j], p[i])]
        want = twins[:min(K, copies - 1)]
        assert ids[i, :len(want)].tolist() == want
        assert (dist[i, :len(want)] == 0).all()
        assert (dist[i, len(want):] > 0).all()


def check_invariants(p, ids, dist, K):
    n = len(p)
    assert ids.shape == (n, K) and dist.shape == (n, K)
    assert (ids >= 0).all() and (ids < n).all()
    assert (ids != np.arange(n)[:, None]).all(), "self in a row"
    srt = np.sort(ids, axis=1)
    assert (srt[:, 1:] != srt[:, :-1]).all(), "repeated id in a row"
    assert (np.diff(dist, axis=1) >= 0).all(), "row not ascending"


@pytest.mark.parametrize("kind,d", [("uniform", 2), ("uniform", 5), ("expo", 3), ("expo", 6),
                                    ("clustered2d", 2)])
def test_invariants_prefix_and_completeness(kind, d):
    p = gen.make_points(kind, 3000, d, seed=1)
    ids8, dist8 = oracle.bf(p, 8)
    ids20, dist20 = oracle.bf(p, 20)
    check_invariants(p, ids8, dist8, 8)
    check_invariants(p, ids20, dist20, 20)
    np.testing.assert_array_equal(ids8, ids20[:, :8])          # prefix property
    assert (dist20[:, 19] >= dist8[:, 7]).all()                # K-th non-decreasing in K
    # completeness on sampled rows: nothing outside the row beats its K-th
    p64 = p.astype(np.float64)
    for i in range(0, len(p), 97):
        t = p64 - p64[i]
        D = np.zeros(len(p))
        for k in range(d):
            D = D + t[:, k] * t[:, k]
        kth = (dist20[i, 19] ** 2, ids20[i, 19])
        outside = np.setdiff1d(np.arange(len(p)), np.append(ids20[i], i))
        for j in outside[np.argsort(D[outside])[:5]]:
            assert (D[j], j) > (D[ids20[i, 19]], ids20[i, 19])
        assert kth[1] == ids20[i, 19]


@pytest.mark.parametrize("kind,d,n,K", [("uniform", 1, 5000, 4), ("uniform", 2, 20000, 8),
                                        ("uniform", 3, 8000, 16), ("uniform", 4, 8000, 32),
                                        ("uniform", 6, 6000, 32), ("expo", 2, 20000, 64),
                                        ("expo", 4, 8000, 16), ("expo", 6, 6000, 64),
                                        ("clustered2d", 2, 20000, 32)])
def test_grid_matches_bf(kind, d, n, K):
    p = gen.make_points(kind, n, d, seed=2)
    ib, db = oracle.bf(p, K)
    ig, dg, st = oracle.grid(p, K)
    np.testing.assert_array_equal(ig, ib)
    np.testing.assert_array_equal(dg, db)
    assert st["candidates"] > 0 and st["passes"] >= 1


@pytest.mark.parametrize("mult", [0.3, 1.0, 2.5])
def test_grid_matches_bf_lattice_and_duplicates(mult):
    lat = gen.points_lattice(11, 3, 0.5)
    ib, db = oracle.bf(lat, 30)
    ig, dg, _ = oracle.grid(lat, 30, width_mult=mult)
    np.testing.assert_array_equal(ig, ib)
    np.testing.assert_array_equal(dg, db)
    dup = gen.points_duplicates(9, 300, 2, gen.stream_key(1, "dup", 1))
    ib, db = oracle.bf(dup, 12)
    ig, dg, _ = oracle.grid(dup, 12, width_mult=mult)
    np.testing.assert_array_equal(ig, ib)
    np.testing.assert_array_equal(dg, db)


def face_case():
    """1-D points where a point outside the scanned box sits exactly on its
    upper face, at the K-th distance, with a smaller id than the point
    inside: with cell side 1 the query at 5.75 scans cells 4..6 = [4, 7),
    whose upper face 7.0 is 1.25 away; 4.5 is also 1.25 away but has id 2."""
    return np.array([[7.0], [5.75], [4.5], [0.0], [20.0], [30.0]], np.float32)


def test_certificate_is_strict_on_the_face():
    p = face_case()
    ig, dg, _ = oracle.grid(p, 1, width_mult=-1.0)
    ib, _ = oracle.bf(p, 1)
    assert ib[1, 0] == 0
    np.testing.assert_array_equal(ig, ib)


def pins_fail(mutant):
    """True when at least one pin detects the mutant."""
    p = quantized(33, 3, seed=3)
    ids, _ = oracle.bf(p, 5, mutant=mutant)
    if not np.array_equal(ids, exact_knn(p, 5)[0]):
        return True
    lat = gen.points_lattice(15, 2)
    ids, _ = oracle.bf(lat, 12, mutant=mutant)
    if not np.array_equal(ids[7 * 15 + 7], np.array(sorted(
            [o for o in itertools.product(range(-2, 3), repeat=2) if any(o)],
            key=lambda o: (o[0] ** 2 + o[1] ** 2, o[0] * 15 + o[1]))[:12]) @ np.array([15, 1]) + 7 * 15 + 7):
        return True
    u = gen.make_points("uniform", 4000, 2, seed=4)
    if not np.array_equal(oracle.grid(u, 8, mutant=mutant)[0], oracle.bf(u, 8)[0]):
        return True
    fc = face_case()
    if oracle.grid(fc, 1, width_mult=-1.0, mutant=mutant)[0][1, 0] != 0:
        return True
    return False


@pytest.mark.parametrize("mutant", oracle.MUTANTS)
def test_pins_catch_planted_mistakes(mutant):
    assert pins_fail(mutant)


def test_pins_pass_unmutated():
    assert not pins_fail(None)


def test_grid_rows_matches_full_grid():
    p = gen.make_points("expo", 20000, 3, seed=6)
    ig, dg, _ = oracle.grid(p, 16)
    rows = np.array([5, 19999, 0, 777, 777, 12345])
    ir, dr, _ = oracle.grid_rows(p, 16, rows)
    np.testing.assert_array_equal(ir, ig[rows])
    np.testing.assert_array_equal(dr, dg[rows])
