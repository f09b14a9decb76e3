"""GPU parity of the resident index (knnjoin_index_*) against the oracle.

An index of S is built once and kept on the device; each query batch R gets,
for each query row, the K nearest rows of S under (canonical D, row), nothing
excluded -- the oracle's brute-force R x S join, bit for bit.  The grid is
S's alone, so batches that leave S's box or its fixed-point frame are cases
of their own.
"""
import threading

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


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def assert_same(got, want):
    gi, gd = (t.cpu().numpy() for t in got)
    wi, wd = want
    bad = np.nonzero((gi != wi).any(axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} rows differ, first {bad[:5]}: got {gi[bad[0]]} want {wi[bad[0]]}"
    np.testing.assert_array_equal(gd, wd)


@pytest.mark.parametrize("kind,d,n,K", [("uniform", 2, 30000, 16), ("uniform", 4, 25000, 32),
                                        ("uniform", 6, 20000, 32), ("expo", 3, 25000, 64),
                                        ("clustered2d", 2, 30000, 16)])
def test_batches_match_oracle(ctx, kind, d, n, K):
    p = gen.make_points(kind, n, d, seed=60 + d)
    with ctx.index(cuda(p), K) as ix:
        for b, (nq, Kq) in enumerate([(5000, K), (1, K), (3000, max(1, K // 4)), (7000, min(2 * K, 256))]):
            q = gen.make_points(kind, nq, d, seed=600 + 10 * d + b)
            assert_same(ix.query(cuda(q), Kq), oracle.bf_rs(q, p, Kq))
        st = ix.stats()
        assert st["n"] == nq and st["passes"] >= 1


@pytest.mark.parametrize("d", [2, 3, 6])
def test_queries_outside_the_data_box(ctx, d):
    p = gen.make_points("uniform", 15000, d, seed=61)
    q = (3.0 * gen.make_points("uniform", 4000, d, seed=62).astype(np.float64) - 1.0).astype(np.float32)
    with ctx.index(cuda(p), 16) as ix:
        assert_same(ix.query(cuda(q), 16), oracle.bf_rs(q, p, 16))
        far = np.full((3, d), 1e6, np.float32)
        far[1] = -1e6
        far[2, 0] = 0.5
        assert_same(ix.query(cuda(far), 5), oracle.bf_rs(far, p, 5))


def test_queries_outside_the_fixed_point_frame(ctx):
    # data on the 2^-24 lattice (integer path); queries with finer bits and a
    # larger range force the batch onto the FP64 scoring path
    p = gen.make_points("uniform", 20000, 4, seed=63)
    q = (gen.make_points("expo", 5000, 4, seed=64).astype(np.float64) * 3.0 + 1e-9).astype(np.float32)
    with ctx.index(cuda(p), 32) as ix:
        got = ix.query(cuda(q), 32)
        assert ix.stats()["fixed_point"] == 0
        assert_same(got, oracle.bf_rs(q, p, 32))
        q2 = gen.make_points("uniform", 3000, 4, seed=65)
        got2 = ix.query(cuda(q2), 32)
        assert ix.stats()["fixed_point"] == 1
        assert_same(got2, oracle.bf_rs(q2, p, 32))


def test_same_as_join_and_repeatable(ctx):
    p = gen.make_points("expo", 20000, 2, seed=66)
    q = gen.make_points("expo", 6000, 2, seed=67)
    with ctx.index(cuda(p), 24) as ix:
        a = ix.query(cuda(q), 24)
        b = ix.query(cuda(q), 24)
    c = ctx.join(cuda(q), cuda(p), 24)
    for x, y in ((a, b), (a, c)):
        assert (x[0] == y[0]).all() and (x[1] == y[1]).all()


def test_host_buffers_and_queries_equal_to_data(ctx):
    import torch
    p = gen.make_points("uniform", 12000, 3, seed=68)
    with ctx.index(torch.from_numpy(p), 9) as ix:   # host points
        ids, dist = ix.query(torch.from_numpy(p), 9)  # host queries and outputs
        assert ids.device.type == "cpu"
        assert_same((ids, dist), oracle.bf_rs(p, p, 9))
        assert (ids[:, 0].numpy() == np.arange(len(p))).all()


def test_errors_leave_the_index_usable(ctx):
    from paper_1810_04758_b300 import KnnJoinError
    p = gen.make_points("uniform", 500, 2, seed=69)
    q = gen.make_points("uniform", 50, 2, seed=70)
    ix = ctx.index(cuda(p), 8)
    with pytest.raises(KnnJoinError):
        ix.query(cuda(q), 501)                     # K > n
    with pytest.raises(KnnJoinError):
        ix.query(cuda(q[:0]), 4)                   # no queries
    bad = q.copy()
    bad[7, 1] = np.nan
    with pytest.raises(KnnJoinError):
        ix.query(cuda(bad), 4)
    with pytest.raises(ValueError):
        ix.query(cuda(np.zeros((5, 3), np.float32)), 4)
    assert_same(ix.query(cuda(q), 8), oracle.bf_rs(q, p, 8))
    ix.close()
    ix.close()                                     # second close: no-op
    with pytest.raises(ValueError):
        ix.query(cuda(q), 8)


def test_indexes_on_two_threads(ctx):
    import torch
    sets = [gen.make_points("uniform", 20000, d, seed=71 + d) for d in (2, 4)]
    qs = [gen.make_points("uniform", 8000, d, seed=81 + d) for d in (2, 4)]
    ixs = [ctx.index(cuda(p), 16) for p in sets]
    torch.cuda.synchronize()
    out = [None, None]

    def work(i):
        res = None
        for _ in range(3):
            res = ixs[i].query(torch.from_numpy(qs[i]), 16)   # host buffers: no torch stream involved
        out[i] = res

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i in range(2):
        assert_same(out[i], oracle.bf_rs(qs[i], sets[i], 16))
        ixs[i].close()


def test_context_close_frees_live_indexes():
    from paper_1810_04758_b300 import Context
    p = gen.make_points("uniform", 3000, 2, seed=90)
    c = Context(device=0)
    ix = c.index(cuda(p), 4)
    ids, _ = ix.query(cuda(p[:10]), 4)
    assert (ids[:, 0].cpu().numpy() == np.arange(10)).all()
    c.close()      # frees the index too
    ix.close()     # no-op after the context is gone


@pytest.mark.parametrize("d,K,Kq", [(1, 8, 30), (8, 16, 4), (3, 200, 256)])
def test_dimensions_and_k_other_than_the_index(ctx, d, K, Kq):
    # the index's search distance is chosen for K; queries may ask for more
    # or fewer neighbours (up to 256 and n)
    p = gen.make_points("uniform", 9000, d, seed=75 + d)
    q = gen.make_points("uniform", 2000, d, seed=85 + d)
    with ctx.index(cuda(p), K) as ix:
        assert_same(ix.query(cuda(q), Kq), oracle.bf_rs(q, p, Kq))


def test_index_of_skewed_data_with_outlier_queries(ctx):
    # exponential data (density skew: the mega-tile walk) queried by points
    # spread far beyond the data's box
    p = gen.make_points("expo", 40000, 3, seed=77)
    q = (4.0 * gen.make_points("uniform", 3000, 3, seed=78).astype(np.float64) - 1.0).astype(np.float32)
    with ctx.index(cuda(p), 32) as ix:
        assert_same(ix.query(cuda(q), 32), oracle.bf_rs(q, p, 32))
