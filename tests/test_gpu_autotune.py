"""Cell-width autotuning (knnjoin_autotune) and its JSON cache.

The multiplier only changes speed: joins at any multiplier, tuned or not,
must give identical results, equal to the oracle's."""
import json

import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu
CANDIDATES = [1.0, 1.0625, 1.125, 1.1875, 1.25, 1.3125, 1.4, 1.5, 1.625]


def test_autotune_cache_and_identical_results(tmp_path):
    import torch
    from paper_1810_04758_b300 import build, Context
    build.build()
    path = str(tmp_path / "tune.json")
    p = gen.make_points("expo", 60000, 3, seed=61)
    t = torch.from_numpy(p).cuda()
    K = 16
    with Context(device=0, tune_cache_path=path) as ctx:
        best = ctx.autotune(t, K)
        assert any(abs(best - c) < 1e-6 for c in CANDIDATES)
        ids, dist = ctx.self_join(t, K)
        assert abs(ctx.stats()["width_mult"] - best) < 1e-6
        ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    with open(path) as f:
        entries = json.load(f)["entries"]
    assert [(e["d"], e["K"], e["nlog2"]) for e in entries] == [(3, K, 15)]
    assert abs(entries[0]["width_mult"] - best) < 1e-6
    # a new context reads the cache; a fixed multiplier overrides it
    with Context(device=0, tune_cache_path=path) as ctx:
        ctx.self_join(t, K)
        assert abs(ctx.stats()["width_mult"] - best) < 1e-6
    want = oracle.bf(p, K)
    np.testing.assert_array_equal(ids, want[0])
    np.testing.assert_array_equal(dist, want[1])
    for wm in (1.0, 1.625):
        with Context(device=0, width_mult=wm, tune_cache_path=path) as ctx:
            gi, gd = ctx.self_join(t, K)
            assert abs(ctx.stats()["width_mult"] - wm) < 1e-6
            np.testing.assert_array_equal(gi.cpu().numpy(), ids)
            np.testing.assert_array_equal(gd.cpu().numpy(), dist)
