"""Virtual shards on one GPU: a self-join split into row ranges
(shard_rows + knnjoin_self_join_rows, as each GPU of a multi-GPU split would
run it) must reassemble to the whole join and to the oracle, bit for bit,
with device or host outputs, chunked output and the paper's policy."""
import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = {"plain": Context(device=0), "chunked": Context(device=0, out_chunk_mb=1),
         "policy": Context(device=0, policy=1)}
    yield c
    for v in c.values():
        v.close()


def reassemble(ctx, t, K, world):
    from paper_1810_04758_b300 import shard_rows
    parts = [ctx.self_join_rows(t, K, *shard_rows(t.shape[0], world, r)) for r in range(world)]
    return (np.concatenate([p[0].cpu().numpy() for p in parts]),
            np.concatenate([p[1].cpu().numpy() for p in parts]))


@pytest.mark.parametrize("kind,d,n,K", [("uniform", 2, 30000, 16), ("expo", 4, 20000, 32),
                                        ("uniform", 6, 12000, 24), ("clustered2d", 2, 25000, 8)])
@pytest.mark.parametrize("world", [2, 3, 8])
def test_shards_reassemble(ctxs, kind, d, n, K, world):
    import torch
    p = gen.make_points(kind, n, d, seed=30 + d)
    got = reassemble(ctxs["plain"], torch.from_numpy(p).cuda(), K, world)
    want = oracle.bf(p, K)
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])


@pytest.mark.parametrize("mode", ["chunked", "policy", "host"])
def test_shards_with_other_paths(ctxs, mode):
    import torch
    p = gen.make_points("uniform", 20000, 3, seed=34)
    t = torch.from_numpy(p)  # host points and outputs (chunked output needs host outputs)
    if mode == "policy":
        t = t.cuda()
    c = ctxs["plain" if mode == "host" else mode]
    got = reassemble(c, t, 32, 3)
    want = oracle.bf(p, 32)
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
    if mode == "chunked":
        assert c.stats()["chunks"] > 1


def test_single_row_shard_and_errors(ctxs):
    import torch
    from paper_1810_04758_b300 import KnnJoinError
    p = gen.make_points("uniform", 5000, 2, seed=35)
    t = torch.from_numpy(p).cuda()
    ids, dist = ctxs["plain"].self_join_rows(t, 6, 4321, 4322)
    want = oracle.bf_rows(p, 6, [4321])
    np.testing.assert_array_equal(ids.cpu().numpy(), want[0])
    np.testing.assert_array_equal(dist.cpu().numpy(), want[1])
    for b, e in ((5, 5), (-1, 10), (10, 5001), (7, 3)):
        with pytest.raises(KnnJoinError):
            ctxs["plain"].self_join_rows(t, 6, b, e)


def spatially_sorted(kind, n, d, seed):
    """Points in the order of their first coordinate: equal row ranges are
    then regions of very different density (on exponential data)."""
    p = gen.make_points(kind, n, d, seed=seed)
    return p[np.argsort(p[:, 0], kind="stable")]


@pytest.mark.parametrize("kind,d,n,K", [("expo", 2, 40000, 16), ("expo", 4, 25000, 32),
                                        ("uniform", 6, 15000, 24), ("clustered2d", 2, 30000, 8)])
@pytest.mark.parametrize("world", [1, 3, 8])
def test_cost_balanced_shards_reassemble(ctxs, kind, d, n, K, world):
    import torch
    from paper_1810_04758_b300 import gather_shards
    p = spatially_sorted(kind, n, d, seed=40 + d)
    t = torch.from_numpy(p).cuda()
    c = ctxs["plain"]
    bounds, costs = c.shard_bounds(t, K, world)
    assert bounds[0] == 0 and bounds[-1] == n and (np.diff(bounds) >= 0).all()
    # the cut balances the cost model to within one query's cost
    assert costs.max() <= costs.mean() * 1.02
    # every rank computes the same bounds (deterministic index)
    b2, _ = c.shard_bounds(t, K, world)
    np.testing.assert_array_equal(bounds, b2)
    parts = []
    for r in range(world):
        if bounds[r + 1] > bounds[r]:
            rows, ids, dist = c.self_join_range(t, K, int(bounds[r]), int(bounds[r + 1]))
            parts.append((rows.cpu().numpy(), ids.cpu().numpy(), dist.cpu().numpy()))
    gi, gd = gather_shards(n, K, parts)
    wi, wd = oracle.bf(p, K)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_array_equal(gd, wd)


def test_cost_balanced_shards_balance_the_work(ctxs):
    # on spatially sorted skewed data the cost model must predict the work:
    # the candidates each shard evaluates stay within 15% of an even share
    import torch
    p = spatially_sorted("expo", 400000, 3, seed=44)
    t = torch.from_numpy(p).cuda()
    c = ctxs["plain"]
    world = 4
    bounds, costs = c.shard_bounds(t, 32, world)
    assert costs.max() <= costs.mean() * 1.02
    cand = []
    for r in range(world):
        c.self_join_range(t, 32, int(bounds[r]), int(bounds[r + 1]))
        cand.append(c.stats()["candidates"])
    assert max(cand) <= 1.15 * sum(cand) / world


def test_cost_balanced_shard_errors(ctxs):
    import torch
    from paper_1810_04758_b300 import KnnJoinError
    p = gen.make_points("uniform", 5000, 2, seed=45)
    t = torch.from_numpy(p).cuda()
    for b, e in ((5, 5), (-1, 10), (10, 5001)):
        with pytest.raises(KnnJoinError):
            ctxs["plain"].self_join_range(t, 6, b, e)
    with pytest.raises(KnnJoinError):
        ctxs["plain"].shard_bounds(t, 6, 0)
    with pytest.raises(KnnJoinError):  # the paper's policy re-sorts per epoch: not supported
        ctxs["policy"].shard_bounds(t, 6, 2)
