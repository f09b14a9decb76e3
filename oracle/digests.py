"""Digests of the oracle's full results on the 2M-point workloads -- TEST INFRASTRUCTURE.

Runs the oracle's exact grid join (oracle/knn_oracle.c, oracle_grid: the
same total order as the brute force, pinned against it) on each named
2,000,000-point workload and stores, per workload, the SHA-256 of the whole
ids array (int32, little-endian, row-major [n][K]) and of the whole
distance array (float64 bit patterns, row-major [n][K]), plus the same
digests per block of ROWS_PER_BLOCK rows, so that a mismatch can be located
without the arrays.  Output: tests/golden/digests_2m.json.  Calls only the
oracle and the input generators.

    python -m oracle.digests [names...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

import knn_inputs as gen
import oracle

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                   "digests_2m.json")
ROWS_PER_BLOCK = 1 << 17


def array_digests(ids: np.ndarray, dist: np.ndarray) -> dict:
    """Whole-array and per-block SHA-256 of ids (int32 LE) and dist (float64 LE)."""
    ids = np.ascontiguousarray(ids, dtype="<i4")
    dist = np.ascontiguousarray(dist, dtype="<f8")
    n = ids.shape[0]
    blocks = []
    for r0 in range(0, n, ROWS_PER_BLOCK):
        r1 = min(n, r0 + ROWS_PER_BLOCK)
        blocks.append([hashlib.sha256(ids[r0:r1].tobytes()).hexdigest()[:16],
                       hashlib.sha256(dist[r0:r1].tobytes()).hexdigest()[:16]])
    return dict(ids_sha256=hashlib.sha256(ids.tobytes()).hexdigest(),
                dist_sha256=hashlib.sha256(dist.tobytes()).hexdigest(),
                rows_per_block=ROWS_PER_BLOCK, blocks=blocks)


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        p, K = gen.config_points(name)
        t = time.time()
        ids, dist, _ = oracle.grid(p, K)
        entry = dict(n=int(p.shape[0]), d=int(p.shape[1]), K=int(K), **array_digests(ids, dist),
                     oracle_seconds=round(time.time() - t, 2), threads=os.cpu_count())
        data[name] = entry
        data["_about"] = ("SHA-256 of the oracle grid join's full ids (int32 LE) and distances "
                          "(float64 LE) on the 2M-point workloads, whole and per block of rows; "
                          "written by oracle/digests.py")
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(name, entry["ids_sha256"][:16], entry["dist_sha256"][:16], entry["oracle_seconds"], "s",
              flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or [k for k in gen.CONFIGS if k.endswith("_2m")])
