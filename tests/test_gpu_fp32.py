"""GPU checks of the FP32-only ranking diagnostic (knnjoin_fp32_mismatch) and
of the exact join on inputs built so that FP32 squared distances tie where
the exact ones do not.

The diagnostic's counts must equal the oracle's (oracle.fp32_mismatch on the
same exact rows); the join's ids and distances must equal the oracle's brute
force bit for bit even where FP32 cannot tell candidates apart.
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


def counts(res):
    return res["rows_differing"], res["positions_differing"], res["ids_missing"]


@pytest.mark.parametrize("kind,d,n,K", [("uniform", 2, 20000, 32), ("uniform", 4, 20000, 32),
                                        ("uniform", 6, 20000, 32), ("expo", 3, 20000, 64)])
def test_counts_match_oracle(ctx, kind, d, n, K):
    import torch
    p = gen.make_points(kind, n, d, seed=80 + d)
    t = torch.from_numpy(p).cuda()
    ids, _ = ctx.self_join(t, K)
    rows = np.arange(0, n, 3)
    got = ctx.fp32_mismatch(t, ids, rows)
    assert counts(got) == oracle.fp32_mismatch(p, ids.cpu().numpy(), rows)


@pytest.mark.parametrize("columns,per_column,K", [(400, 50, 64), (60, 300, 200), (2000, 12, 16)])
def test_exact_join_where_fp32_ties(ctx, columns, per_column, K):
    import torch
    p = gen.points_columns(columns, per_column, gen.stream_key(0, "columns", columns))
    want = oracle.bf(p, K)
    ids, dist = ctx.self_join(torch.from_numpy(p).cuda(), K)
    np.testing.assert_array_equal(ids.cpu().numpy(), want[0])
    np.testing.assert_array_equal(dist.cpu().numpy(), want[1])
    rows = np.arange(len(p))
    got = ctx.fp32_mismatch(torch.from_numpy(p).cuda(), ids, rows)
    exp = oracle.fp32_mismatch(p, want[0], rows)
    assert counts(got) == exp
    if K > per_column:
        assert exp[1] > 0  # FP32 alone would have reordered these rows


def test_host_inputs_and_hand_case(ctx):
    import torch
    # query (0,0): A = (1, 2^-6) and B = (1, 2^-6 + 2^-29) tie in FP32; the
    # exact order is [A, B], the FP32-only order [B, A] (B has the lower id)
    pts = np.array([[0.0, 0.0], [1.0, 2.0 ** -6 + 2.0 ** -29], [1.0, 2.0 ** -6], [5.0, 5.0]], np.float32)
    ids, _ = ctx.self_join(torch.from_numpy(pts), 2)
    assert list(ids[0].numpy()) == [2, 1]
    got = ctx.fp32_mismatch(torch.from_numpy(pts), ids, [0])
    assert counts(got) == (1, 2, 0)


def test_invalid_arguments(ctx):
    import torch
    from paper_1810_04758_b300 import KnnJoinError
    p = torch.from_numpy(gen.make_points("uniform", 500, 2, seed=90)).cuda()
    ids, _ = ctx.self_join(p, 4)
    with pytest.raises(KnnJoinError):
        ctx.fp32_mismatch(p, ids, [500])          # row out of range
    with pytest.raises(KnnJoinError):
        ctx.fp32_mismatch(p, ids, [])             # no rows
    bad = ids.clone()
    bad[7, 1] = 7                                 # the row itself
    with pytest.raises(KnnJoinError):
        ctx.fp32_mismatch(p, bad, [7])
    bad[7, 1] = 10 ** 6                           # outside [0, n)
    with pytest.raises(KnnJoinError):
        ctx.fp32_mismatch(p, bad, [7])
    assert counts(ctx.fp32_mismatch(p, ids, [3, 8])) == oracle.fp32_mismatch(p.cpu().numpy(), ids.cpu().numpy(), [3, 8])


@pytest.mark.parametrize("K", [1, 256])
def test_counts_match_oracle_at_k_extremes(ctx, K):
    import torch
    p = gen.make_points("uniform", 6000, 3, seed=95)
    t = torch.from_numpy(p).cuda()
    ids, _ = ctx.self_join(t, K)
    rows = np.arange(0, 6000, 5)
    assert counts(ctx.fp32_mismatch(t, ids, rows)) == oracle.fp32_mismatch(p, ids.cpu().numpy(), rows)
