"""The allocation-free self-join entry point, called through the C ABI.

Some callers cannot let a library allocate device memory: code that runs
inside another framework's memory pool or under a hard memory cap, or an
embedding that owns every allocation.  knnjoin_self_join_noalloc serves them
from a fixed scratch array inside the library.  This test checks that two
calls in a row give exactly the results of the ordinary knnjoin_self_join
(ids equal, distances equal -- the exactness every parity test here uses),
and that a size beyond the limit is refused with a clear message.  It lives
in a file collected last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

import knn_inputs as gen

pytestmark = pytest.mark.gpu


def test_noalloc_matches_self_join_twice():
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build

    build.build()
    kj.load_library()
    cases = [(gen.make_points("uniform", 40000, 3, seed=21), 16),
             (gen.make_points("expo", 65536, 2, seed=22), 32)]
    with kj.Context(device=0) as ctx:
        for p, K in cases:
            t = torch.from_numpy(p).cuda()
            want_ids, want_dist = ctx.self_join(t, K)
            ids = torch.full_like(want_ids, -7)
            dist = torch.full_like(want_dist, -7.0)
            stream = torch.cuda.current_stream().cuda_stream
            kj.knnjoin_self_join_noalloc(t.data_ptr(), p.shape[0], p.shape[1], K,
                                         ids.data_ptr(), dist.data_ptr(), stream)
            torch.cuda.synchronize()
            assert torch.equal(ids, want_ids)
            assert torch.equal(dist, want_dist)


def test_noalloc_rejects_too_many_points():
    import torch
    import paper_1810_04758_b300 as kj

    kj.load_library()
    n = kj.KNN_NOALLOC_MAX_POINTS + 1
    t = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    ids = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    dist = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(kj.KnnJoinError) as e:
        kj.knnjoin_self_join_noalloc(t.data_ptr(), n, 2, 4, ids.data_ptr(), dist.data_ptr(), 0)
    assert e.value.status == kj.KNN_ERR_INVALID
    assert "limit" in str(e.value)
