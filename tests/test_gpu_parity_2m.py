"""Parity at the benchmark sizes (n = 2,000,000), in the configuration the
benchmark times.

The oracle cannot brute-force 2M x 2M pairs in seconds, so each run is
checked (a) on sampled rows, one by one, against the oracle's brute force
over all 2M points (ids bit-exact, distances identical), and (b) on every
row by properties that hold at any size: ascending distances, no self, no
repeated id, ids in range, and the prefix property between K and K/2.
"""
import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = Context(device=0)
    yield c
    c.close()


def sample_rows(n, count, seed):
    key = gen.stream_key(seed, "rows", n)
    r = (gen.raw_u64(key, count) % np.uint64(n)).astype(np.int64)
    return np.unique(np.concatenate([r, [0, n - 1]]))


@pytest.mark.parametrize("name", ["unif2d_2m", "unif4d_2m", "unif6d_2m",
                                  "expo2d_2m", "expo4d_2m", "expo6d_2m"])
def test_2m_sampled_rows_and_invariants(ctx, name):
    import torch
    p, K = gen.config_points(name)
    n = len(p)
    t = torch.from_numpy(p).cuda()
    ids, dist = ctx.self_join(t, K)
    half, _ = ctx.self_join(t, K // 2)
    torch.cuda.synchronize()
    ids, dist, half = ids.cpu().numpy(), dist.cpu().numpy(), half.cpu().numpy()
    rows = sample_rows(n, 300, seed=hash(name) % 1000)
    wi, wd = oracle.bf_rows(p, K, rows)
    np.testing.assert_array_equal(ids[rows], wi)
    np.testing.assert_array_equal(dist[rows], wd)
    assert (ids >= 0).all() and (ids < n).all()
    assert (ids != np.arange(n, dtype=np.int32)[:, None]).all()
    s = np.sort(ids, axis=1)
    assert (s[:, 1:] != s[:, :-1]).all()
    assert (np.diff(dist, axis=1) >= 0).all()
    np.testing.assert_array_equal(half, ids[:, :K // 2])
