"""GPU parity of the R x S join (knnjoin_join) against the CPU oracle.

For each query row, the K nearest data rows under (canonical D, data row),
nothing excluded.  Ids bit-exact and distances bit-identical to the
oracle's brute force, as for the self-join.
"""
import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = Context(device=0)
    yield c
    c.close()


def run(ctx, q, p, K, on_device=True):
    import torch
    tq = torch.from_numpy(np.ascontiguousarray(q, np.float32))
    tp = torch.from_numpy(np.ascontiguousarray(p, np.float32))
    if on_device:
        tq, tp = tq.cuda(), tp.cuda()
    ids, dist = ctx.join(tq, tp, K)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


def assert_same(got, want):
    gi, gd = got
    wi, wd = want
    bad = np.nonzero((gi != wi).any(axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} rows differ, first {bad[:5]}: got {gi[bad[0]]} want {wi[bad[0]]}"
    np.testing.assert_array_equal(gd, wd)


@pytest.mark.parametrize("kind,d,nq,n,K", [
    ("uniform", 2, 12000, 30000, 32), ("uniform", 3, 9000, 20000, 16), ("uniform", 4, 8000, 20000, 32),
    ("uniform", 6, 6000, 20000, 32), ("uniform", 1, 5000, 7000, 5), ("uniform", 8, 3000, 4000, 8),
    ("expo", 2, 10000, 30000, 64), ("expo", 4, 8000, 20000, 64), ("clustered2d", 2, 10000, 40000, 32),
])
def test_join_parity(ctx, kind, d, nq, n, K):
    q = gen.make_points(kind, nq, d, seed=41)
    p = gen.make_points(kind, n, d, seed=42)
    assert_same(run(ctx, q, p, K), oracle.bf_rs(q, p, K))


@pytest.mark.parametrize("d", [2, 3, 6])
def test_queries_outside_the_data_box(ctx, d):
    # queries spread over [-0.5, 1.5)^d: many lie outside the data's box
    q = (2.0 * gen.make_points("uniform", 6000, d, seed=43).astype(np.float64) - 0.5).astype(np.float32)
    p = gen.make_points("uniform", 15000, d, seed=44)
    assert_same(run(ctx, q, p, 16), oracle.bf_rs(q, p, 16))


def test_queries_equal_to_data_points(ctx):
    # R = S: each query's own row is its first neighbour at distance 0
    p = gen.make_points("uniform", 20000, 3, seed=45)
    got = run(ctx, p, p, 9)
    assert_same(got, oracle.bf_rs(p, p, 9))
    assert (got[0][:, 0] == np.arange(len(p))).all() and (got[1][:, 0] == 0).all()


def test_single_query_and_k_equals_n(ctx):
    p = gen.make_points("expo", 200, 4, seed=46)
    q = gen.make_points("uniform", 1, 4, seed=47)
    assert_same(run(ctx, q, p, 200), oracle.bf_rs(q, p, 200))


def test_dense_core_in_sparse_background(ctx):
    core = (0.5 + 1e-3 * gen.make_points("uniform", 20000, 2, seed=48).astype(np.float64)).astype(np.float32)
    p = np.concatenate([core, gen.make_points("uniform", 10000, 2, seed=49)])
    q = gen.make_points("uniform", 8000, 2, seed=50)
    assert_same(run(ctx, q, p, 16), oracle.bf_rs(q, p, 16))


def test_host_pointers_match_device(ctx):
    q = gen.make_points("uniform", 4000, 3, seed=51)
    p = gen.make_points("uniform", 9000, 3, seed=52)
    assert_same(run(ctx, q, p, 12, on_device=False), run(ctx, q, p, 12))


def test_invalid_arguments(ctx):
    import torch
    from paper_1810_04758_b300 import KnnJoinError
    p = torch.from_numpy(gen.make_points("uniform", 100, 2, seed=53)).cuda()
    q = torch.from_numpy(gen.make_points("uniform", 10, 2, seed=54)).cuda()
    with pytest.raises(KnnJoinError):
        ctx.join(q, p, 101)  # K > n
    with pytest.raises(KnnJoinError):
        ctx.join(q[:0], p, 5)  # no queries
    with pytest.raises(ValueError):
        ctx.join(q, torch.zeros((100, 3), dtype=torch.float32, device="cuda"), 5)


def test_far_queries_on_skewed_data(ctx):
    # queries far outside an exponential data set: every candidate lies at
    # nearly the same distance, buffers overflow into the general kernel
    # within a two-tile step, and the second tile must not append to a
    # buffer the first tile's insert has just handed over
    p = gen.make_points("expo", 40000, 3, seed=77)
    q = (4.0 * gen.make_points("uniform", 3000, 3, seed=78).astype(np.float64) - 1.0).astype(np.float32)
    got = run(ctx, q, p, 32)
    assert ctx.stats()["overflow_queries"] > 0
    assert_same(got, oracle.bf_rs(q, p, 32))
