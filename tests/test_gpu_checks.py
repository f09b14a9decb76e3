"""The checked build (-DKNN_CHECKS): every guarded index in the scan kernels
is tested on the device; a failed test is reported as KNN_ERR_CUDA with the
failing sites.  A run of the self-join, R x S, the paper's policy and chunked
output on the checked library must pass every check and match the oracle.
The checked library is loaded in a child process (one library per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import knn_inputs as gen
import oracle
import paper_1810_04758_b300 as kj
from paper_1810_04758_b300 import build
kj.load_library(build.build_checked())

def same(got, want):
    assert np.array_equal(got[0].cpu().numpy(), want[0])
    assert np.array_equal(got[1].cpu().numpy(), want[1])

with kj.Context(device=0) as ctx:
    for kind, d, n, K in [("uniform", 2, 30000, 32), ("expo", 4, 20000, 64), ("uniform", 6, 15000, 16),
                          ("clustered2d", 2, 30000, 8)]:
        p = gen.make_points(kind, n, d, seed=91)
        same(ctx.self_join(torch.from_numpy(p).cuda(), K), oracle.bf(p, K))
    core = (0.5 + 1e-3 * gen.make_points("uniform", 20000, 2, seed=92).astype(np.float64)).astype(np.float32)
    p = np.concatenate([core, gen.make_points("uniform", 8000, 2, seed=93)])
    same(ctx.self_join(torch.from_numpy(p).cuda(), 16), oracle.bf(p, 16))
    q = gen.make_points("expo", 8000, 3, seed=94)
    p = gen.make_points("expo", 12000, 3, seed=95)
    same(ctx.join(torch.from_numpy(q).cuda(), torch.from_numpy(p).cuda(), 24), oracle.bf_rs(q, p, 24))
with kj.Context(device=0, policy=1) as ctx:
    p = gen.make_points("expo", 20000, 2, seed=96)
    same(ctx.self_join(torch.from_numpy(p).cuda(), 32), oracle.bf(p, 32))
with kj.Context(device=0, out_chunk_mb=1) as ctx:
    p = gen.make_points("uniform", 40000, 3, seed=97)
    same(ctx.self_join(torch.from_numpy(p), 16), oracle.bf(p, 16))
print("checked ok")
'''


def test_checked_build_passes_every_check():
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCRIPT], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
