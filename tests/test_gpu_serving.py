"""Batched and served joins (worker pool, footprint admission), through the C ABI.

* a batch of uneven jobs equals the same jobs run one by one, and the oracle;
* served jobs submitted while others run give the same results as alone
  (continuous batching changes scheduling, never results);
* cancellation, a full queue, invalid submissions and an allocator hook that
  starts failing (host-side fault injection) return statuses and leave the
  context usable.
"""
import ctypes
import time

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


def mixed_jobs(count, seed, n_hi=30000):
    jobs = gen.batched_jobs(count, seed=seed, n_lo=500, n_hi=n_hi)
    return [(gen.batched_points(j, seed=seed), j["K"]) for j in jobs]


def test_batch_equals_single_and_oracle(kj):
    import torch
    jobs = mixed_jobs(24, seed=3)
    with kj.Context(0, workers=6) as ctx:
        dev = [torch.from_numpy(p).cuda() for p, _ in jobs]
        outs = ctx.self_join_batch(dev, [K for _, K in jobs])
        torch.cuda.synchronize()
        for (p, K), t, (ids, dist) in zip(jobs, dev, outs):
            si, sd = ctx.self_join(t, K)
            assert torch.equal(ids, si) and torch.equal(dist, sd)
            wi, wd = oracle.bf(p, K)
            np.testing.assert_array_equal(ids.cpu().numpy(), wi)
            np.testing.assert_array_equal(dist.cpu().numpy(), wd)


@pytest.mark.parametrize("large_first", [False, True])
def test_served_results_same_alone_and_in_mix(kj, large_first):
    import torch
    jobs = mixed_jobs(30, seed=5)
    if large_first:
        # two joins of >= 2^25 output entries, which go to high-priority streams
        jobs.insert(3, (gen.make_points("uniform", 600000, 3, seed=6), 64))
        jobs.insert(20, (gen.make_points("expo", 550000, 4, seed=7), 64))
    with kj.Context(0, workers=4) as alone:
        ref = []
        for p, K in jobs:
            ids, dist = alone.self_join(torch.from_numpy(p).cuda(), K)
            ref.append((ids.cpu(), dist.cpu()))
    with kj.Context(0, workers=8, large_first=large_first) as ctx:
        pending = []
        for k, (p, K) in enumerate(jobs):
            t = torch.from_numpy(p).cuda() if k % 2 else torch.from_numpy(p)  # device and host inputs
            jid, ids, dist = ctx.submit(t, K)
            pending.append((jid, t, ids, dist, k))
            if k % 7 == 3:
                time.sleep(0.002)  # arrivals while others run
        done = {}
        deadline = time.time() + 120
        while len(done) < len(pending) and time.time() < deadline:
            for jid, t, ids, dist, k in pending:
                if jid in done:
                    continue
                st = ctx.poll(jid)
                if st != kj.KNN_ERR_NOT_READY:
                    assert st == kj.KNN_OK, ctx.last_error()
                    done[jid] = (ids, dist, k)
            time.sleep(0.001)
        assert len(done) == len(pending)
        torch.cuda.synchronize()
        for ids, dist, k in done.values():
            assert torch.equal(ids.cpu(), ref[k][0]) and torch.equal(dist.cpu(), ref[k][1])


def test_cancel_queue_full_and_invalid(kj):
    import torch
    p = torch.from_numpy(gen.make_points("uniform", 200000, 3, seed=1)).cuda()
    # one worker and a tiny budget: jobs wait in the queue
    with kj.Context(0, workers=1, max_jobs=3, hbm_budget_bytes=1) as ctx:
        ids = []
        full = False
        for _ in range(10):
            try:
                jid, a, b = ctx.submit(p, 16)
            except kj.KnnJoinError as e:
                assert e.status == kj.KNN_ERR_QUEUE_FULL
                full = True
                break
            ids.append((jid, a, b))
        assert full and len(ids) >= 3
        last = ids[-1][0]
        assert ctx.cancel(last) == kj.KNN_OK
        for jid, _, _ in ids:
            while True:
                st = ctx.poll(jid)
                if st != kj.KNN_ERR_NOT_READY:
                    break
                time.sleep(0.002)
            assert st == (kj.KNN_ERR_CANCELLED if jid == last else kj.KNN_OK)
        with pytest.raises(kj.KnnJoinError) as e:
            ctx.submit(p, 0)
        assert e.value.status == kj.KNN_ERR_INVALID
        assert ctx.poll(123456) == kj.KNN_ERR_INVALID
        # still usable
        ids2, _ = ctx.self_join(p[:5000].contiguous(), 4)
        assert ids2.shape == (5000, 4)


ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def test_allocator_hook_failure_is_reported(kj):
    """torch's caching allocator backs the library's scratch through the
    hooks; after a set number of allocations the hook returns NULL."""
    import torch
    state = {"left": 10 ** 9, "live": {}}

    def alloc(nbytes, user):
        if state["left"] <= 0:
            return None
        state["left"] -= 1
        ptr = torch.cuda.caching_allocator_alloc(nbytes, 0)
        state["live"][ptr] = nbytes
        return ptr

    def free(ptr, user):
        state["live"].pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    a_cb, f_cb = ALLOC(alloc), FREE(free)
    cfg = kj.KnnjoinConfig()
    cfg.device = 0
    cfg.stream = torch.cuda.current_stream().cuda_stream
    cfg.alloc = ctypes.cast(a_cb, ctypes.c_void_p)
    cfg.free = ctypes.cast(f_cb, ctypes.c_void_p)
    ctx = kj.knnjoin_create(cfg)
    try:
        p = gen.make_points("uniform", 30000, 2, seed=9)
        t = torch.from_numpy(p).cuda()
        ids = torch.empty((30000, 8), dtype=torch.int32, device="cuda")
        dist = torch.empty((30000, 8), dtype=torch.float64, device="cuda")
        kj.knnjoin_self_join(ctx, t.data_ptr(), 30000, 2, 8, ids.data_ptr(), dist.data_ptr())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), oracle.bf(p, 8)[0])
        assert state["live"], "scratch came from the hook"
        # a bigger join needs new buffers: make the hook fail
        big = torch.from_numpy(gen.make_points("uniform", 120000, 2, seed=9)).cuda()
        ids2 = torch.empty((120000, 8), dtype=torch.int32, device="cuda")
        dist2 = torch.empty((120000, 8), dtype=torch.float64, device="cuda")
        state["left"] = 0
        with pytest.raises(kj.KnnJoinError) as e:
            kj.knnjoin_self_join(ctx, big.data_ptr(), 120000, 2, 8, ids2.data_ptr(), dist2.data_ptr())
        assert e.value.status == kj.KNN_ERR_NOMEM
        state["left"] = 10 ** 9
        kj.knnjoin_self_join(ctx, big.data_ptr(), 120000, 2, 8, ids2.data_ptr(), dist2.data_ptr())
        torch.cuda.synchronize()
        assert (ids2.cpu().numpy()[:, 0] != np.arange(120000)).all()
    finally:
        kj.knnjoin_destroy(ctx)
        torch.cuda.synchronize()
    assert not state["live"], "every hook allocation was freed"


def test_allocator_hook_misaligned_pointer_is_rejected(kj):
    """A hook pointer that is not 16-byte aligned (scratch is read with
    16-byte vector loads) is handed back to the free hook and the call fails
    with KNN_ERR_INVALID before any kernel touches it; an aligned hook then
    works on the same context."""
    import torch
    state = {"shift": 4, "live": {}, "freed_bad": 0}

    def alloc(nbytes, user):
        base = torch.cuda.caching_allocator_alloc(nbytes + 256, 0)
        ptr = base + state["shift"]
        state["live"][ptr] = base
        return ptr

    def free(ptr, user):
        if ptr % 16:
            state["freed_bad"] += 1
        torch.cuda.caching_allocator_delete(state["live"].pop(ptr))

    a_cb, f_cb = ALLOC(alloc), FREE(free)
    cfg = kj.KnnjoinConfig()
    cfg.device = 0
    cfg.stream = torch.cuda.current_stream().cuda_stream
    cfg.alloc = ctypes.cast(a_cb, ctypes.c_void_p)
    cfg.free = ctypes.cast(f_cb, ctypes.c_void_p)
    ctx = kj.knnjoin_create(cfg)
    try:
        p = gen.make_points("uniform", 5000, 3, seed=19)
        t = torch.from_numpy(p).cuda()
        ids = torch.empty((5000, 8), dtype=torch.int32, device="cuda")
        dist = torch.empty((5000, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(kj.KnnJoinError) as e:
            kj.knnjoin_self_join(ctx, t.data_ptr(), 5000, 3, 8, ids.data_ptr(), dist.data_ptr())
        assert e.value.status == kj.KNN_ERR_INVALID
        assert "aligned" in str(e.value)
        assert state["freed_bad"] >= 1
        state["shift"] = 0
        kj.knnjoin_self_join(ctx, t.data_ptr(), 5000, 3, 8, ids.data_ptr(), dist.data_ptr())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), oracle.bf(p, 8)[0])
    finally:
        kj.knnjoin_destroy(ctx)
        torch.cuda.synchronize()
    assert not state["live"]
