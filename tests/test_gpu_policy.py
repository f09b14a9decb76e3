"""The paper's GPU-Only policy (knnjoin_config.policy = 1): one global eps,
a query fails when fewer than K neighbours lie within eps, failed queries
are redone on a grid re-indexed with eps += eps_min / 2.  Only the schedule
differs from the default policy: rows must equal the oracle's.  The policy
itself is tested with the tail strategy off; the tail strategy (Sec. 5.4:
the last few queries in one pass over the whole grid) is tested beside it,
under both policies."""
import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = Context(device=0, policy=1, tail_queries=-1)
    yield c
    c.close()


def run(ctx, p, K):
    import torch
    ids, dist = ctx.self_join(torch.from_numpy(p).cuda(), K)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("kind,d,n,K", [
    ("uniform", 2, 30000, 32), ("uniform", 4, 20000, 32), ("uniform", 6, 20000, 32),
    ("expo", 2, 30000, 64), ("expo", 4, 20000, 64), ("expo", 6, 12000, 32), ("clustered2d", 2, 40000, 32),
])
def test_paper_policy_matches_oracle(ctx, kind, d, n, K):
    p = gen.make_points(kind, n, d, seed=71)
    gi, gd = run(ctx, p, K)
    st = ctx.stats()
    wi, wd = oracle.bf(p, K)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_array_equal(gd, wd)
    assert st["passes"] >= 1 and st["pass_queries"][0] == n


def test_paper_policy_reindexes_on_skewed_data(ctx):
    # exponential data: sparse queries fail at eps_min and need wider grids
    p = gen.make_points("expo", 30000, 3, seed=72)
    gi, gd = run(ctx, p, 32)
    st = ctx.stats()
    assert st["passes"] >= 3
    q = st["pass_queries"]
    assert all(q[i + 1] < q[i] for i in range(len(q) - 1))
    wi, wd = oracle.bf(p, 32)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_array_equal(gd, wd)


def test_paper_policy_r_x_s(ctx):
    import torch
    q = gen.make_points("expo", 8000, 2, seed=73)
    p = gen.make_points("expo", 20000, 2, seed=74)
    gi, gd = ctx.join(torch.from_numpy(q).cuda(), torch.from_numpy(p).cuda(), 16)
    wi, wd = oracle.bf_rs(q, p, 16)
    np.testing.assert_array_equal(gi.cpu().numpy(), wi)
    np.testing.assert_array_equal(gd.cpu().numpy(), wd)


@pytest.mark.parametrize("kind,d,n,K", [("expo", 3, 30000, 32), ("expo", 6, 12000, 32),
                                        ("clustered2d", 2, 40000, 16)])
def test_tail_strategy_paper_policy(kind, d, n, K):
    import torch
    from paper_1810_04758_b300 import Context
    p = gen.make_points(kind, n, d, seed=75)
    t = torch.from_numpy(p).cuda()
    with Context(device=0, policy=1, tail_queries=-1) as off, Context(device=0, policy=1) as on:
        io, do = off.self_join(t, K)
        so = off.stats()
        it, dt = on.self_join(t, K)
        st = on.stats()
    torch.cuda.synchronize()
    assert torch.equal(io, it) and torch.equal(do, dt)
    assert st["passes"] <= so["passes"]
    wi, wd = oracle.bf(p, K)
    np.testing.assert_array_equal(it.cpu().numpy(), wi)
    np.testing.assert_array_equal(dt.cpu().numpy(), wd)


@pytest.mark.parametrize("policy", [0, 1])
def test_tail_strategy_forced(policy):
    # every query left after the first epoch / second pass goes to the whole grid
    import torch
    from paper_1810_04758_b300 import Context
    p = gen.make_points("expo", 25000, 4, seed=76)
    t = torch.from_numpy(p).cuda()
    with Context(device=0, policy=policy, tail_queries=1 << 30) as c:
        ids, dist = c.self_join(t, 64)
        st = c.stats()
    torch.cuda.synchronize()
    assert st["passes"] <= (2 if policy == 1 else 3)
    wi, wd = oracle.bf(p, 64)
    np.testing.assert_array_equal(ids.cpu().numpy(), wi)
    np.testing.assert_array_equal(dist.cpu().numpy(), wd)


def _with_far_points(p, far):
    return np.ascontiguousarray(np.concatenate([p, np.asarray(far, np.float32)]).astype(np.float32))


@pytest.mark.parametrize("K", [8, 40])
def test_brute_force_tail(K):
    """Far outliers stay uncertified through the ring passes; when few are
    left, the tail takes every (query, point) pair at once (exact FP32 K-th
    by radix select, band, exact re-score): the last pass evaluates exactly
    queries x (n - 1) pairs, and the rows equal the oracle's."""
    import torch
    from paper_1810_04758_b300 import Context
    far = [[40.0, 40.0], [-35.0, 50.0], [60.0, -20.0], [-45.0, -45.0], [55.0, 55.0], [40.5, 40.0]]
    p = _with_far_points(gen.make_points("uniform", 30000, 2, seed=31), far)
    with Context(device=0) as c:
        ids, dist = c.self_join(torch.from_numpy(p).cuda(), K)
        st = c.stats()
    torch.cuda.synchronize()
    wi, wd = oracle.bf(p, K)
    np.testing.assert_array_equal(ids.cpu().numpy(), wi)
    np.testing.assert_array_equal(dist.cpu().numpy(), wd)
    last = st["passes"] - 1
    assert last >= 2 and st["pass_queries"][last] >= 1
    assert st["pass_candidates"][last] == st["pass_queries"][last] * (len(p) - 1)


def test_brute_force_tail_r_x_s_and_shards():
    """The same tail for far R x S queries (nothing excluded) and for a
    cost-balanced shard of a self-join (rows by sorted position)."""
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import Context
    data = gen.make_points("expo", 40000, 3, seed=32)
    q = _with_far_points(gen.make_points("uniform", 500, 3, seed=33) * 0.2,
                         [[5.0, 5.0, 5.0], [-4.0, 3.0, 9.0], [7.0, -6.0, 1.0]])
    with Context(device=0) as c:
        ids, dist = c.join(torch.from_numpy(q).cuda(), torch.from_numpy(data).cuda(), 16)
        torch.cuda.synchronize()
        wi, wd = oracle.bf_rs(q, data, 16)
        np.testing.assert_array_equal(ids.cpu().numpy(), wi)
        np.testing.assert_array_equal(dist.cpu().numpy(), wd)
        p = _with_far_points(gen.make_points("uniform", 20000, 3, seed=34), [[9.0, 9.0, 9.0], [-8.0, 1.0, 2.0]])
        t = torch.from_numpy(p).cuda()
        bounds, _ = c.shard_bounds(t, 8, 3)
        got = [c.self_join_range(t, 8, int(bounds[i]), int(bounds[i + 1])) for i in range(3)]
        torch.cuda.synchronize()
    rows = np.concatenate([r.cpu().numpy() for r, _, _ in got])
    gi = np.concatenate([i.cpu().numpy() for _, i, _ in got])
    gd = np.concatenate([d.cpu().numpy() for _, _, d in got])
    order = np.argsort(rows)
    wi, wd = oracle.bf(p, 8)
    np.testing.assert_array_equal(rows[order], np.arange(len(p)))
    np.testing.assert_array_equal(gi[order], wi)
    np.testing.assert_array_equal(gd[order], wd)


def test_brute_force_tail_band_overflow_falls_back():
    """A far R x S query whose K nearest tie with hundreds of data points
    (300 copies of one site) overflows the tail's band: it takes a
    whole-grid scan pass after the brute force (and the general kernel), and
    its row still equals the oracle's."""
    import torch
    from paper_1810_04758_b300 import Context
    data = _with_far_points(gen.make_points("uniform", 20000, 2, seed=35), [[3.0, 3.0]] * 300)
    q = _with_far_points(gen.make_points("uniform", 200, 2, seed=36), [[9.0, 11.0]])
    with Context(device=0) as c:
        ids, dist = c.join(torch.from_numpy(q).cuda(), torch.from_numpy(data).cuda(), 8)
        st = c.stats()
    torch.cuda.synchronize()
    wi, wd = oracle.bf_rs(q, data, 8)
    np.testing.assert_array_equal(ids.cpu().numpy(), wi)
    np.testing.assert_array_equal(dist.cpu().numpy(), wd)
    # a brute-force pass (every pair of its queries), then a pass after it
    n = len(data)
    bf = [i for i in range(2, st["passes"]) if st["pass_queries"][i] > 0 and
          st["pass_candidates"][i] == st["pass_queries"][i] * n]
    assert bf and bf[0] + 1 < st["passes"], (st["passes"], st["pass_queries"], st["pass_candidates"])
