"""Parity at the benchmark sizes (n = 2,000,000), in the configuration the
benchmark times (each join's cell-width multiplier autotuned first).

Every row is compared: the SHA-256 of the GPU's whole ids array (int32) and
whole distance array (float64 bits) must equal the digests of the oracle's
exact grid join on the same points (tests/golden/digests_2m.json, written by
oracle/digests.py, which calls only the oracle).  On a mismatch the per-block
digests name the differing row blocks, and rows of the first such block are
compared one by one against the oracle to show what differs.  Beside that,
sampled rows (a fixed SplitMix64 stream, so a failure replays) are checked
against the oracle's brute force over all 2M points, and every row against
properties that hold at any size: ascending distances, no self, no repeated
id, ids in range, and the prefix property between K and K/2.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "digests_2m.json")
NAMES = ["unif2d_2m", "unif4d_2m", "unif6d_2m", "expo2d_2m", "expo4d_2m", "expo6d_2m"]


@pytest.fixture(scope="module")
def ctx():
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = Context(device=0)
    yield c
    c.close()


def sample_rows(n, count, name):
    key = gen.stream_key(0, "parity-rows:" + name, n)
    r = (gen.raw_u64(key, count) % np.uint64(n)).astype(np.int64)
    return np.unique(np.concatenate([r, [0, n - 1]]))


def block_digests(ids, dist, rows_per_block):
    ids = np.ascontiguousarray(ids, dtype="<i4")
    dist = np.ascontiguousarray(dist, dtype="<f8")
    out = []
    for r0 in range(0, ids.shape[0], rows_per_block):
        r1 = r0 + rows_per_block
        out.append([hashlib.sha256(ids[r0:r1].tobytes()).hexdigest()[:16],
                    hashlib.sha256(dist[r0:r1].tobytes()).hexdigest()[:16]])
    return out


@pytest.mark.parametrize("name", NAMES)
def test_2m_every_row_sampled_rows_and_invariants(ctx, name):
    import torch
    golden = json.load(open(GOLDEN))[name]
    p, K = gen.config_points(name)
    n = len(p)
    t = torch.from_numpy(p).cuda()
    ctx.autotune(t, K)  # the launch configuration the benchmark times
    ids, dist = ctx.self_join(t, K)
    half, _ = ctx.self_join(t, K // 2)
    torch.cuda.synchronize()
    ids, dist, half = ids.cpu().numpy(), dist.cpu().numpy(), half.cpu().numpy()

    # every row: whole-array digests against the oracle's
    gi = hashlib.sha256(np.ascontiguousarray(ids, dtype="<i4").tobytes()).hexdigest()
    gd = hashlib.sha256(np.ascontiguousarray(dist, dtype="<f8").tobytes()).hexdigest()
    if (gi, gd) != (golden["ids_sha256"], golden["dist_sha256"]):
        rpb = golden["rows_per_block"]
        got = block_digests(ids, dist, rpb)
        bad = [b for b, (g, w) in enumerate(zip(got, golden["blocks"])) if g != w]
        b0 = bad[0]
        rows = np.arange(b0 * rpb, min(n, (b0 + 1) * rpb), max(1, rpb // 512), dtype=np.int64)
        wi, wd = oracle.grid_rows(p, K, rows)[:2]
        wrong = rows[(ids[rows] != wi).any(axis=1) | (dist[rows] != wd).any(axis=1)]
        pytest.fail(f"{name}: output differs from the oracle in row blocks {bad} of {rpb} rows; "
                    f"{len(wrong)} of {len(rows)} sampled rows of block {b0} differ, e.g. {wrong[:5]}")

    # sampled rows against brute force over all n points
    rows = sample_rows(n, 300, name)
    wi, wd = oracle.bf_rows(p, K, rows)
    np.testing.assert_array_equal(ids[rows], wi)
    np.testing.assert_array_equal(dist[rows], wd)

    # properties of every row
    assert (ids >= 0).all() and (ids < n).all()
    assert (ids != np.arange(n, dtype=np.int32)[:, None]).all()
    s = np.sort(ids, axis=1)
    assert (s[:, 1:] != s[:, :-1]).all()
    assert (np.diff(dist, axis=1) >= 0).all()
    np.testing.assert_array_equal(half, ids[:, :K // 2])
