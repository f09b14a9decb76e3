"""Multi-rank plumbing on CPU (gloo, world size 2).

bench.py runs replicas by default (each rank the whole workload, the job's
time the slowest rank's): two gloo ranks report different times; both must
see the maximum, and one rank alone must see its own.  A join split by row
ranges (shard_rows, knnjoin_self_join_rows on each GPU) must reassemble to
the whole join: two gloo ranks compute their shards with the oracle and the
gathered rows must equal the oracle's full self-join.  Cost-balanced shards
(knnjoin_shard_bounds / knnjoin_self_join_range) hold scattered original
rows; their gather (gather_shards) is tested the same way.
"""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v = bench.max_over_ranks(10.0 + 7.5 * rank, "cpu", world)
        dist.barrier()
        q.put((rank, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 17.5, 1: 17.5}


def test_max_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, "cpu", 1) == 3.25


def _shard_rank(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import knn_inputs as gen
    import oracle
    from paper_1810_04758_b300 import shard_rows
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = gen.make_points("uniform", 3001, 3, seed=5)
        b, e = shard_rows(len(p), world, rank)
        ids, dist_ = oracle.bf_rows(p, 7, np.arange(b, e), threads=1)
        parts = [None] * world
        dist.all_gather_object(parts, (b, e, ids, dist_))
        if rank == 0:
            parts.sort(key=lambda t: t[0])
            got_i = np.concatenate([t[2] for t in parts])
            got_d = np.concatenate([t[3] for t in parts])
            want_i, want_d = oracle.bf(p, 7, threads=1)
            q.put(bool(np.array_equal(got_i, want_i) and np.array_equal(got_d, want_d)
                       and parts[0][0] == 0 and parts[-1][1] == len(p)))
    finally:
        dist.destroy_process_group()


def test_row_shards_reassemble_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True


@pytest.mark.parametrize("n,world", [(10, 1), (10, 3), (2_000_000, 8), (7, 7)])
def test_shard_rows_cover_disjointly(n, world):
    sys.path.insert(0, ROOT)
    from paper_1810_04758_b300 import shard_rows
    r = [shard_rows(n, world, k) for k in range(world)]
    assert r[0][0] == 0 and r[-1][1] == n
    assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
    sizes = [e - b for b, e in r]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def _scattered_shard_rank(rank, world, port, q):
    # a cost-balanced shard holds the rows of a range of the index's key
    # order: scattered original rows.  Here the order is the points' first
    # coordinate; each rank computes its range with the oracle, the ranks
    # exchange (rows, ids, dist) and rank 0 reassembles with gather_shards.
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import knn_inputs as gen
    import oracle
    from paper_1810_04758_b300 import gather_shards
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = gen.make_points("expo", 2501, 2, seed=6)
        order = np.argsort(p[:, 0], kind="stable")
        cut = [0, 1700, len(p)]  # uneven ranges, as a cost-balanced cut may be
        rows = order[cut[rank]:cut[rank + 1]]
        ids, dist_ = oracle.bf_rows(p, 5, rows, threads=1)
        parts = [None] * world
        dist.all_gather_object(parts, (rows, ids, dist_))
        if rank == 0:
            gi, gd = gather_shards(len(p), 5, parts)
            wi, wd = oracle.bf(p, 5, threads=1)
            q.put(bool(np.array_equal(gi, wi) and np.array_equal(gd, wd)))
    finally:
        dist.destroy_process_group()


def test_scattered_row_shards_gather_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 33500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_scattered_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True


def test_gather_shards_rejects_gaps_and_overlaps():
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_1810_04758_b300 import gather_shards
    i = np.zeros((2, 1), np.int32)
    d = np.zeros((2, 1), np.float64)
    with pytest.raises(ValueError):
        gather_shards(3, 1, [(np.array([0, 1]), i, d)])  # row 2 missing
    with pytest.raises(ValueError):
        gather_shards(2, 1, [(np.array([0, 1]), i, d), (np.array([1]), i[:1], d[:1])])  # row 1 twice
