"""Seeded sweep of GPU parity cases: sizes, dimensions, K, distributions
(including far outliers, which end in the brute-force tail), scales and the
API variants (self-join, R x S, the paper's policy, chunked output, host
pointers, the tail forced after the second pass, cost-balanced shards), each
compared bit for bit with the oracle's brute force.  The case list is drawn
once from a fixed SplitMix64 stream."""
import numpy as np
import pytest

import knn_inputs as gen
import oracle

pytestmark = pytest.mark.gpu

KINDS = ["uniform", "expo", "clustered2d", "lattice", "duplicates", "scaled", "outliers"]
MODES = ["self", "self", "rxs", "policy", "chunked", "host", "tail", "shards"]


def draw_cases(count=96):
    u = gen.uniform_f64(gen.stream_key(0, "gpu_sweep"), 8 * count).reshape(count, 8)
    cases = []
    for i in range(count):
        kind = KINDS[int(u[i, 0] * len(KINDS))]
        d = 2 if kind == "clustered2d" else 1 + int(u[i, 1] * 8)
        n = int(np.exp(np.log(300) + u[i, 2] * (np.log(25000) - np.log(300))))
        K = max(1, min(n - 1, 256, int(np.exp(u[i, 3] * np.log(200)))))
        mode = MODES[int(u[i, 4] * len(MODES))]
        scale = [1.0, 1e-30, 1e30, -3.5, 1e6][int(u[i, 5] * 5)]
        cases.append((i, kind, d, n, K, mode, scale))
    return cases


def make(kind, n, d, scale, seed):
    if kind == "lattice":
        m = max(2, int(round(n ** (1.0 / d))) + 1)
        r = gen.raw_u64(gen.stream_key(seed, "sweep_lattice", n * 10 + d), n * d) % np.uint64(m)
        p = r.astype(np.float64).reshape(n, d)
    elif kind == "duplicates":
        sites = max(2, n // 7)
        base = gen.make_points("uniform", sites, d, seed=seed).astype(np.float64)
        pick = gen.raw_u64(gen.stream_key(seed, "sweep_dup", n), n) % np.uint64(sites)
        p = base[pick.astype(np.int64)]
    elif kind == "outliers":
        p = gen.make_points("uniform", n, d, seed=seed).astype(np.float64)
        k = max(1, n // 500)
        p[:k] = (gen.uniform_f64(gen.stream_key(seed, "sweep_far", n), k * d).reshape(k, d) - 0.5) * 200.0
    elif kind == "scaled":
        p = gen.make_points("expo", n, d, seed=seed).astype(np.float64) * 1e3 - 7.0
    else:
        p = gen.make_points(kind, n, d, seed=seed).astype(np.float64)
    return (p * scale).astype(np.float32)


@pytest.fixture(scope="module")
def ctxs():
    from paper_1810_04758_b300 import build, Context
    build.build()
    c = {"self": Context(device=0), "policy": Context(device=0, policy=1),
         "chunked": Context(device=0, out_chunk_mb=1), "tail": Context(device=0, tail_queries=1 << 30)}
    yield c
    for v in c.values():
        v.close()


@pytest.mark.parametrize("case", draw_cases(), ids=lambda c: f"{c[0]}-{c[1]}-d{c[2]}-n{c[3]}-K{c[4]}-{c[5]}")
def test_sweep(ctxs, case):
    import torch
    i, kind, d, n, K, mode, scale = case
    p = make(kind, n, d, scale, seed=100 + i)
    if mode == "rxs":
        q = make(kind, max(1, n // 2), d, scale, seed=500 + i)
        Kr = min(K, n)
        ids, dist = ctxs["self"].join(torch.from_numpy(q).cuda(), torch.from_numpy(p).cuda(), Kr)
        want = oracle.bf_rs(q, p, Kr)
    elif mode == "shards":
        t = torch.from_numpy(p).cuda()
        b, _ = ctxs["self"].shard_bounds(t, K, 3)
        parts = [ctxs["self"].self_join_range(t, K, int(b[j]), int(b[j + 1])) for j in range(3) if b[j + 1] > b[j]]
        rows = np.concatenate([r.cpu().numpy() for r, _, _ in parts])
        order = np.argsort(rows)
        np.testing.assert_array_equal(rows[order], np.arange(n))
        ids = torch.from_numpy(np.concatenate([x.cpu().numpy() for _, x, _ in parts])[order])
        dist = torch.from_numpy(np.concatenate([x.cpu().numpy() for _, _, x in parts])[order])
        want = oracle.bf(p, K)
    else:
        c = ctxs[mode if mode in ("policy", "chunked", "tail") else "self"]
        t = torch.from_numpy(p)
        if mode not in ("chunked", "host"):
            t = t.cuda()
        ids, dist = c.self_join(t, K)
        want = oracle.bf(p, K)
    np.testing.assert_array_equal(ids.cpu().numpy(), want[0])
    np.testing.assert_array_equal(dist.cpu().numpy(), want[1])
