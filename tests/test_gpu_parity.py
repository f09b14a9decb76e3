"""GPU parity of the exact KNN self-join against the CPU oracle.

Every case compares the CUDA path, called through the C ABI, with the oracle
on the same seeded inputs, element by element: neighbour ids bit-exact and
distances bit-identical (the library's distances are the correctly rounded
square roots of the same canonical FP64 squared distances, so exact equality
is the tolerance; it is tighter than the 1e-12 relative bound).
"""
import os
import subprocess

import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = Context(device=0)
    yield c
    c.close()


def run(ctx, pts, K, on_device=True):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(pts, np.float32))
    if on_device:
        t = t.cuda()
    ids, dist = ctx.self_join(t, K)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


def assert_same(got, want):
    gi, gd = got
    wi, wd = want
    bad = np.nonzero((gi != wi).any(axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} rows differ, first {bad[:5]}: got {gi[bad[0]]} want {wi[bad[0]]}"
    np.testing.assert_array_equal(gd, wd)


def test_exact_arithmetic_on_device(tmp_path):
    exe = tmp_path / "ted"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", str(exe),
                    os.path.join(ROOT, "tests/native/test_exact_device.cu")], check=True)
    r = subprocess.run([str(exe), str(1 << 24)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr


def test_unif2d_20k_full(ctx):
    p, K = gen.config_points("unif2d_20k")
    assert_same(run(ctx, p, K), oracle.bf(p, K))


@pytest.mark.parametrize("kind,d,n,K", [
    ("uniform", 1, 7000, 5), ("uniform", 2, 30011, 32), ("uniform", 3, 12000, 16),
    ("uniform", 4, 20000, 32), ("uniform", 5, 9000, 24), ("uniform", 6, 20000, 32),
    ("uniform", 7, 5000, 12), ("uniform", 8, 4000, 8),
    ("expo", 2, 30000, 64), ("expo", 4, 20000, 64), ("expo", 6, 20000, 64), ("expo", 3, 8000, 128),
    ("clustered2d", 2, 40000, 32),
])
def test_parity_small(ctx, kind, d, n, K):
    p = gen.make_points(kind, n, d, seed=7)
    assert_same(run(ctx, p, K), oracle.bf(p, K))


@pytest.mark.parametrize("d,K", [(2, 16), (3, 16), (4, 8)])
def test_dense_core_in_sparse_background(ctx, d, K):
    # 2/3 of the points in a cube of side 1e-3, the rest uniform: queries of
    # the background sit at coarse levels whose ring covers the core, so the
    # core's cells are long runs scanned in pruned super-tiles
    n_core, n_bg = 20000, 10000
    core = (0.5 + 1e-3 * gen.make_points("uniform", n_core, d, seed=31).astype(np.float64)).astype(np.float32)
    bg = gen.make_points("uniform", n_bg, d, seed=32)
    p = np.concatenate([core, bg])
    assert_same(run(ctx, p, K), oracle.bf(p, K))


@pytest.mark.parametrize("d,K", [(2, 64), (4, 32), (6, 16)])
def test_long_runs_with_outliers(ctx, d, K):
    # 180k points in a cube of side 1e-4 (cells of the core hold runs of many
    # 4,096-point mega-tiles), 20k uniform points around it and 300 far
    # outliers; outlier and background queries sit at coarse levels whose
    # boxes reach the core, so the mega-tile walk skips most of its runs.
    # Sampled rows (every outlier, a stride of the rest) against brute force.
    core = (0.25 + 1e-4 * gen.make_points("uniform", 180000, d, seed=35).astype(np.float64)).astype(np.float32)
    bg = gen.make_points("uniform", 20000, d, seed=36)
    far = (4.0 + 3.0 * gen.make_points("uniform", 300, d, seed=37).astype(np.float64)).astype(np.float32)
    p = np.concatenate([core, bg, far])
    ids, dist = run(ctx, p, K)
    rows = np.concatenate([np.arange(0, len(p) - 300, 97), np.arange(len(p) - 300, len(p))])
    wi, wd = oracle.bf_rows(p, K, rows)
    bad = np.nonzero((ids[rows] != wi).any(axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} rows differ, first row {rows[bad[0]]}"
    np.testing.assert_array_equal(dist[rows], wd)


def test_requeued_passes_match(ctx):
    # queries that the first pass cannot certify are re-scanned one level up,
    # starting from the band of the K-th value the first pass found
    seen = 0
    for kind, d, n, K in [("uniform", 6, 20000, 32), ("expo", 4, 20000, 64), ("expo", 2, 30000, 64)]:
        p = gen.make_points(kind, n, d, seed=7)
        got = run(ctx, p, K)
        st = ctx.stats()
        if st["passes"] >= 2 and st["pass_queries"][1] > 0:
            seen += 1
        assert_same(got, oracle.bf(p, K))
    assert seen > 0


@pytest.mark.parametrize("K", [1, 2, 255])
def test_parity_k_extremes(ctx, K):
    p = gen.make_points("uniform", 3000, 3, seed=9)
    assert_same(run(ctx, p, K), oracle.bf(p, K))


def test_k_equals_n_minus_1(ctx):
    p = gen.make_points("uniform", 200, 2, seed=3)
    assert_same(run(ctx, p, 199), oracle.bf(p, 199))


def test_two_points(ctx):
    p = np.array([[0.5, 0.25], [0.125, 1.0]], np.float32)
    assert_same(run(ctx, p, 1), oracle.bf(p, 1))


@pytest.mark.parametrize("d,m,K,scale", [(2, 60, 21, 1.0), (3, 17, 33, 0.125), (1, 500, 6, 1.0),
                                         (4, 7, 40, 2.0)])
def test_lattice_ties(ctx, d, m, K, scale):
    p = gen.points_lattice(m, d, scale)
    assert_same(run(ctx, p, K), oracle.bf(p, K))


def test_lattice_permuted(ctx):
    base = gen.points_lattice(40, 2)
    p = base[gen.permutation(len(base), gen.stream_key(1, "perm", 0))]
    assert_same(run(ctx, p, 13), oracle.bf(p, 13))


@pytest.mark.parametrize("copies,sites,d,K", [(6, 500, 2, 9), (300, 10, 3, 40), (2000, 2, 2, 100)])
def test_duplicates(ctx, copies, sites, d, K):
    p = gen.points_duplicates(copies, sites, d, gen.stream_key(2, "dup", copies))
    assert_same(run(ctx, p, K), oracle.bf(p, K))


def test_all_points_identical(ctx):
    p = np.full((500, 3), 0.375, np.float32)
    assert_same(run(ctx, p, 20), oracle.bf(p, 20))


def test_negative_large_and_tiny_coordinates(ctx):
    key = gen.stream_key(5, "mixed", 0)
    u = gen.uniform_f64(key, 6000 * 3).reshape(6000, 3)
    p = ((u - 0.5) * np.array([1e6, 1e-30, 3.0])).astype(np.float32)
    assert_same(run(ctx, p, 10), oracle.bf(p, 10))
    q = (gen.uniform_f64(key, 5000 * 2, offset=99).reshape(5000, 2) * 1e-38).astype(np.float32)
    assert_same(run(ctx, q, 7), oracle.bf(q, 7))


def test_host_pointers_match_device(ctx):
    p = gen.make_points("expo", 10000, 3, seed=4)
    a = run(ctx, p, 16, on_device=True)
    b = run(ctx, p, 16, on_device=False)
    assert_same(a, b)


def test_deterministic(ctx):
    p = gen.make_points("uniform", 50000, 4, seed=8)
    a = run(ctx, p, 32)
    b = run(ctx, p, 32)
    assert_same(a, b)


def test_invalid_arguments(ctx):
    import torch
    from paper_1810_04758_b300 import KnnJoinError, KNN_ERR_INVALID
    p = torch.rand(100, 3, device="cuda")
    with pytest.raises(KnnJoinError) as e:
        ctx.self_join(p, 100)
    assert e.value.status == KNN_ERR_INVALID
    with pytest.raises(KnnJoinError):
        ctx.self_join(torch.rand(100, 9, device="cuda"), 3)
    bad = p.clone()
    bad[17, 1] = float("nan")
    with pytest.raises(KnnJoinError) as e:
        ctx.self_join(bad, 5)
    assert e.value.status == KNN_ERR_INVALID
    # the context stays usable after a rejected call
    ids, _ = ctx.self_join(p, 5)
    assert ids.shape == (100, 5)


@pytest.mark.parametrize("n,K,offset", [(2001, 3, 0), (2001, 3, 1), (3000, 8, 1)])
def test_distance_outputs_odd_sized_and_unaligned(ctx, n, K, offset):
    # the square-root pass works on 16-byte vectors when it can: an odd
    # number of entries leaves a tail, and an output that starts 8 bytes
    # into an allocation takes the one-value-at-a-time path
    import torch
    p = gen.make_points("uniform", n, 3, seed=91)
    base = torch.empty(n * K + offset, dtype=torch.float64, device="cuda")
    dist = base[offset:].view(n, K)
    ids = torch.empty((n, K), dtype=torch.int32, device="cuda")
    ctx.self_join(torch.from_numpy(p).cuda(), K, ids, dist)
    torch.cuda.synchronize()
    want = oracle.bf(p, K)
    np.testing.assert_array_equal(ids.cpu().numpy(), want[0])
    np.testing.assert_array_equal(dist.cpu().numpy(), want[1])
