"""Batched joins scanned together (knnjoin_config.batch_union), through the C ABI.

Every join of the batch runs its own pass loop; the scan of each pass is one
launch per group of joins with the same d and buffer size, over the union of
their work items, dense first across joins (the paper's Sec. 4.5 work queue
across joins).  Scheduling changes, results must not:

* a mixed batch (d 2/3/4/6, K 4..64, uniform and exponential) equals the
  oracle's brute force and the worker-pool batch, bit for bit;
* more joins of one group than one launch holds (S2_MULTI_JOBS = 64) are
  split over several launches and stay exact;
* host output buffers work;
* a join that fails part-way (a NaN coordinate, found on the device) leaves
  the batch without stalling the others: the call returns its status, the
  other joins' rows are exact, and the context stays usable.
"""
import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kj():
    import paper_1810_04758_b300 as m
    from paper_1810_04758_b300 import build
    build.build()
    m.load_library()
    return m


def mixed_jobs(count, seed, n_lo=500, n_hi=30000):
    jobs = gen.batched_jobs(count, seed=seed, n_lo=n_lo, n_hi=n_hi)
    return [(gen.batched_points(j, seed=seed), j["K"]) for j in jobs]


def test_union_batch_equals_oracle_and_pool(kj):
    import torch
    jobs = mixed_jobs(40, seed=11)
    dev = [torch.from_numpy(p).cuda() for p, _ in jobs]
    Ks = [K for _, K in jobs]
    with kj.Context(0, batch_union=True) as cu, kj.Context(0, workers=6) as cp:
        outs_u = cu.self_join_batch(dev, Ks)
        outs_p = cp.self_join_batch(dev, Ks)
        torch.cuda.synchronize()
        for (p, K), (iu, du), (ip, dp) in zip(jobs, outs_u, outs_p):
            assert torch.equal(iu, ip) and torch.equal(du, dp)
            wi, wd = oracle.bf(p, K)
            np.testing.assert_array_equal(iu.cpu().numpy(), wi)
            np.testing.assert_array_equal(du.cpu().numpy(), wd)
        # a second batch on the same context reuses its pipelines
        outs_2 = cu.self_join_batch(dev[:7], Ks[:7])
        torch.cuda.synchronize()
        for (i2, d2), (iu, du) in zip(outs_2, outs_u[:7]):
            assert torch.equal(i2, iu) and torch.equal(d2, du)


def test_union_batch_more_joins_than_one_launch(kj):
    import torch
    # 80 joins of one group (d = 3, K = 16): two launches of the union kernel
    pts = [gen.make_points("uniform" if j % 2 else "expo", 800 + 37 * j, 3, seed=100 + j) for j in range(80)]
    dev = [torch.from_numpy(p).cuda() for p in pts]
    with kj.Context(0, batch_union=True) as cu:
        outs = cu.self_join_batch(dev, [16] * len(dev))
        torch.cuda.synchronize()
    for p, (ids, dist) in zip(pts, outs):
        wi, wd = oracle.bf(p, 16)
        np.testing.assert_array_equal(ids.cpu().numpy(), wi)
        np.testing.assert_array_equal(dist.cpu().numpy(), wd)


def test_union_batch_host_buffers(kj):
    import torch
    jobs = mixed_jobs(12, seed=12, n_hi=8000)
    host = [torch.from_numpy(p) for p, _ in jobs]
    outs_in = [(torch.empty((len(p), K), dtype=torch.int32).pin_memory(),
                torch.empty((len(p), K), dtype=torch.float64)) for p, K in jobs]
    with kj.Context(0, batch_union=True) as cu:
        outs = cu.self_join_batch(host, [K for _, K in jobs], outs_in)
        torch.cuda.synchronize()
    for (p, K), (ids, dist) in zip(jobs, outs):
        wi, wd = oracle.bf(p, K)
        np.testing.assert_array_equal(ids.numpy(), wi)
        np.testing.assert_array_equal(dist.numpy(), wd)


def test_union_batch_failing_join_leaves(kj):
    import torch
    jobs = mixed_jobs(9, seed=13, n_hi=6000)
    bad = gen.make_points("uniform", 3000, 2, seed=14)
    bad[1234, 1] = np.nan  # found by the join's first kernel, after it joined the batch
    pts = [p for p, _ in jobs[:4]] + [bad] + [p for p, _ in jobs[4:]]
    Ks = [K for _, K in jobs[:4]] + [8] + [K for _, K in jobs[4:]]
    dev = [torch.from_numpy(p).cuda() for p in pts]
    with kj.Context(0, batch_union=True) as cu:
        outs = [(torch.full((len(p), K), -1, dtype=torch.int32, device="cuda"),
                 torch.full((len(p), K), -1.0, dtype=torch.float64, device="cuda")) for p, K in zip(pts, Ks)]
        with pytest.raises(kj.KnnJoinError) as e:
            cu.self_join_batch(dev, Ks, outs)
        assert e.value.status == kj.KNN_ERR_INVALID
        assert "job 4" in str(e.value)
        torch.cuda.synchronize()
        for j, (p, K) in enumerate(zip(pts, Ks)):
            if j == 4:
                continue
            wi, wd = oracle.bf(p, K)
            np.testing.assert_array_equal(outs[j][0].cpu().numpy(), wi)
            np.testing.assert_array_equal(outs[j][1].cpu().numpy(), wd)
        # the context is still usable
        ids, dist = cu.self_join(dev[0], Ks[0])
        torch.cuda.synchronize()
        wi, _ = oracle.bf(pts[0], Ks[0])
        np.testing.assert_array_equal(ids.cpu().numpy(), wi)
