"""The paper's GPU-Only policy (knnjoin_config.policy = 1): one global eps,
a query fails when fewer than K neighbours lie within eps, failed queries
are redone on a grid re-indexed with eps += eps_min / 2.  Only the schedule
differs from the default policy: rows must equal the oracle's."""
import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = Context(device=0, policy=1)
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
