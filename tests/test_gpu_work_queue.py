"""The density-ordered work queue (step a6) against the paper's Fig. 4.

Fig. 4 (Sec. 4.5) shows the work queue of |D| = 100 points: C holds, for
each point, the number of points in its grid cell, sorted non-increasing,
and the GPU takes queries from the dense end.  tests/golden/fig4_workqueue.json
stores the positions the figure prints (1-32 in a cell of 32 points, 33-52
in a cell of 20, 95-100 single points) and a fill for the positions it does
not print.  The points here are built so that their cells have exactly
those sizes (each cell's points are copies of one site, sites far apart),
and the queue the library builds must be that C.  The paper's GPU-Only
policy is used: one grid of cell side eps, as in the paper's GPU kernel, so
that every query starts in its own level-0 cell.
"""
import json
import os

import numpy as np
import pytest

import knn_inputs as gen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fig4_workqueue.json")


def fig4_cells():
    g = json.load(open(GOLDEN))
    printed = {int(k): v for k, v in g["printed_positions"].items()}
    sizes = [32, 20] + list(g["fill_cells"]) + [1] * 6
    assert sum(sizes) == g["n_points"]
    C = np.concatenate([np.full(s, s) for s in sizes])
    for pos, c in printed.items():  # the fill agrees with every printed position
        assert C[pos - 1] == c
    return sizes, C


def test_work_queue_matches_fig4():
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build
    build.build()
    sizes, want = fig4_cells()
    # one site per cell, sites spread over [0, 100) in a shuffled order
    order = np.argsort(gen.raw_u64(gen.stream_key(0, "fig4", 0), len(sizes)), kind="stable")
    sites = (order.astype(np.float64) * 7.0 + 1.0).astype(np.float32)
    pts = np.concatenate([np.stack([np.full(s, sites[c]), np.full(s, sites[c] * 0.5)], axis=1)
                          for c, s in enumerate(sizes)]).astype(np.float32)
    perm = np.argsort(gen.raw_u64(gen.stream_key(0, "fig4", 1), len(pts)), kind="stable")
    pts = np.ascontiguousarray(pts[perm])
    t = torch.from_numpy(pts).cuda()
    with kj.Context(device=0, policy=1) as ctx:
        got = kj.knnjoin_work_queue(ctx.ctx, t.data_ptr(), len(pts), 2, 1)
    assert len(got) == len(pts)
    np.testing.assert_array_equal(got, want)
    assert (np.diff(got) <= 0).all()  # densest first


def test_work_queue_is_dense_first_on_skewed_data():
    import torch
    import paper_1810_04758_b300 as kj
    p = gen.make_points("expo", 20000, 2, seed=91)
    t = torch.from_numpy(p).cuda()
    with kj.Context(device=0) as ctx:
        got = kj.knnjoin_work_queue(ctx.ctx, t.data_ptr(), len(p), 2, 8)
    assert len(got) == len(p)
    assert (np.diff(got) <= 0).all()
    assert got.sum() >= len(p)  # every query in a cell of at least itself
