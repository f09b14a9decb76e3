"""Chunked output (knnjoin_config.out_chunk_mb): results bound for host
memory are computed in chunks of query rows, each copied out before the
next.  Rows must equal the oracle's, whatever the chunking."""
import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = Context(device=0, out_chunk_mb=1)
    yield c
    c.close()


@pytest.mark.parametrize("kind,d,n,K", [("uniform", 3, 50000, 16), ("expo", 2, 40000, 32), ("uniform", 6, 20000, 32)])
def test_chunked_self_join_matches_oracle(ctx, kind, d, n, K):
    import torch
    p = gen.make_points(kind, n, d, seed=81)
    ids, dist = ctx.self_join(torch.from_numpy(p), K)  # host in, host out
    st = ctx.stats()
    rows = (1 << 20) // (K * 12)
    assert st["chunks"] == -(-n // rows) and st["chunks"] > 1
    wi, wd = oracle.bf(p, K)
    np.testing.assert_array_equal(ids.numpy(), wi)
    np.testing.assert_array_equal(dist.numpy(), wd)


def test_chunked_r_x_s_matches_oracle(ctx):
    import torch
    q = gen.make_points("uniform", 30000, 4, seed=82)
    p = gen.make_points("uniform", 20000, 4, seed=83)
    ids, dist = ctx.join(torch.from_numpy(q), torch.from_numpy(p), 16)
    assert ctx.stats()["chunks"] > 1
    wi, wd = oracle.bf_rs(q, p, 16)
    np.testing.assert_array_equal(ids.numpy(), wi)
    np.testing.assert_array_equal(dist.numpy(), wd)


def test_device_outputs_are_not_chunked(ctx):
    import torch
    p = gen.make_points("uniform", 50000, 3, seed=84)
    ids, dist = ctx.self_join(torch.from_numpy(p).cuda(), 16)
    assert ctx.stats()["chunks"] == 1
