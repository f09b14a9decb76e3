"""The allocation-free self-join entry point, called through the C ABI.

Some callers cannot let a library allocate device memory: code that runs
inside another framework's memory pool or under a hard memory cap, or an
embedding that owns every allocation.  knnjoin_self_join_noalloc serves them
from a fixed scratch array inside the library.  These tests check that two
calls in a row give exactly the results of the ordinary knnjoin_self_join
(ids equal, distances equal -- the exactness every parity test here uses),
over several d and K (including the K > 32 buffers), that sizes beyond the
limit and buffers in the wrong place are refused with a clear status, and
that an input too spread out for the array fails cleanly and leaves the
next call correct.  The file is collected last, and passes alone or after
the other tests.
"""
import numpy as np
import pytest

import knn_inputs as gen

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build

    build.build()
    kj.load_library()
    return kj


def _noalloc(kj, t, K):
    import torch

    n, d = t.shape
    ids = torch.full((n, K), -7, dtype=torch.int32, device=t.device)
    dist = torch.full((n, K), -7.0, dtype=torch.float64, device=t.device)
    stream = torch.cuda.current_stream().cuda_stream
    kj.knnjoin_self_join_noalloc(t.data_ptr(), n, d, K, ids.data_ptr(), dist.data_ptr(), stream)
    torch.cuda.synchronize()
    return ids, dist


CASES = [("uniform", 40000, 3, 16, 21), ("expo", 65536, 2, 32, 22), ("uniform", 20000, 6, 64, 23),
         ("expo", 30000, 4, 128, 24)]


def test_noalloc_matches_self_join_twice():
    import torch

    kj = _lib()
    with kj.Context(device=0) as ctx:
        for dist_name, n, d, K, seed in CASES:
            t = torch.from_numpy(gen.make_points(dist_name, n, d, seed=seed)).cuda()
            want_ids, want_dist = ctx.self_join(t, K)
            torch.cuda.synchronize()
            for _ in range(2):  # the second call starts from the first one's scratch contents
                ids, dist = _noalloc(kj, t, K)
                assert torch.equal(ids, want_ids), (dist_name, n, d, K)
                assert torch.equal(dist, want_dist), (dist_name, n, d, K)


def test_noalloc_rejects_too_many_points():
    import torch

    kj = _lib()
    n = kj.KNN_NOALLOC_MAX_POINTS + 1
    t = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    ids = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    dist = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(kj.KnnJoinError) as e:
        kj.knnjoin_self_join_noalloc(t.data_ptr(), n, 2, 4, ids.data_ptr(), dist.data_ptr(), 0)
    assert e.value.status == kj.KNN_ERR_INVALID
    assert "limit" in str(e.value)


def test_noalloc_rejects_host_buffers():
    import torch

    kj = _lib()
    n, d, K = 1000, 2, 4
    p = torch.from_numpy(gen.make_points("uniform", n, d, seed=25))
    dev = p.cuda()
    ids_d = torch.empty((n, K), dtype=torch.int32, device="cuda")
    dist_d = torch.empty((n, K), dtype=torch.float64, device="cuda")
    ids_h = torch.empty((n, K), dtype=torch.int32).pin_memory()
    dist_h = torch.empty((n, K), dtype=torch.float64)
    for pts, ids, dist in [(p, ids_d, dist_d), (dev, ids_h, dist_d), (dev, ids_d, dist_h)]:
        with pytest.raises(kj.KnnJoinError) as e:
            kj.knnjoin_self_join_noalloc(pts.data_ptr(), n, d, K, ids.data_ptr(), dist.data_ptr(), 0)
        assert e.value.status == kj.KNN_ERR_INVALID
    # the entry point still works after the refusals
    ids, dist = _noalloc(kj, dev, K)
    with kj.Context(device=0) as ctx:
        want_ids, want_dist = ctx.self_join(dev, K)
    assert torch.equal(ids, want_ids) and torch.equal(dist, want_dist)


def test_noalloc_spread_out_input():
    """Coordinates on a geometric scale (each point a random power of 1.9 times
    a uniform value) need cell tables on many grid levels: the call returns the
    exact result, or a clean KNN_ERR_NOMEM after which the next call is exact."""
    import torch

    kj = _lib()
    rng = np.random.default_rng(26)
    n, d, K = 60000, 3, 8
    u = gen.make_points("uniform", n, d, seed=27).astype(np.float64)
    scale = 1.9 ** rng.integers(-40, 1, size=(n, 1))
    t = torch.from_numpy((u * scale).astype(np.float32)).cuda()
    with kj.Context(device=0) as ctx:
        want_ids, want_dist = ctx.self_join(t, K)
        torch.cuda.synchronize()
        try:
            ids, dist = _noalloc(kj, t, K)
            assert torch.equal(ids, want_ids) and torch.equal(dist, want_dist)
        except kj.KnnJoinError as e:
            assert e.status == kj.KNN_ERR_NOMEM, str(e)
            assert "fixed scratch array exhausted" in str(e)
        small = torch.from_numpy(gen.make_points("uniform", 5000, 2, seed=28)).cuda()
        ids, dist = _noalloc(kj, small, 8)
        w_ids, w_dist = ctx.self_join(small, 8)
        assert torch.equal(ids, w_ids) and torch.equal(dist, w_dist)
