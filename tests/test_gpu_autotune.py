"""Autotuning (knnjoin_autotune: cell-width multiplier, then candidate
buffer size) and its JSON cache.

Both only change speed: joins at any multiplier or buffer size, tuned or
not, must give identical results, equal to the oracle's."""
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
    assert entries[0]["buffer"] in (2, 4)  # 64 or 128 entries for K = 16
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


def test_tuned_buffer_sizes_give_identical_results(tmp_path):
    # a cache that asks for the larger buffer (128 entries, 8 queries per
    # work item) for one class: rows identical to the default buffer's
    import torch
    from paper_1810_04758_b300 import build, Context
    build.build()
    p = gen.make_points("uniform", 50000, 4, seed=62)
    t = torch.from_numpy(p).cuda()
    K = 24
    path = str(tmp_path / "tune.json")
    with open(path, "w") as f:
        json.dump({"knnjoin_tune": 1, "entries": [{"d": 4, "K": K, "nlog2": 15, "width_mult": 1.125,
                                                   "buffer": 4}]}, f)
    with Context(device=0) as c0, Context(device=0, tune_cache_path=path) as c1:
        i0, d0 = c0.self_join(t, K)
        assert c0.stats()["buffer_entries"] == 64
        i1, d1 = c1.self_join(t, K)
        assert c1.stats()["buffer_entries"] == 128
    torch.cuda.synchronize()
    assert torch.equal(i0, i1) and torch.equal(d0, d1)
    want = oracle.bf(p, K)
    np.testing.assert_array_equal(i1.cpu().numpy(), want[0])
