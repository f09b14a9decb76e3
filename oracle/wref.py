"""Reference-schedule work counts W_ref for the roofline -- TEST/BENCH INFRASTRUCTURE.

Runs the oracle's grid join (width from the Sec. 4.4 selection with
multiplier 1, ring of 3^n cells, wider retry) on each named 2M-point
workload and stores, per workload, the number of candidate distance
evaluations and its pass profile in tests/golden/wref_2m.json.  Calls only
the oracle and the input generators.

    python -m oracle.wref [names...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import knn_inputs as gen
import oracle

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                   "wref_2m.json")


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        p, K = gen.config_points(name)
        t = time.time()
        _, _, st = oracle.grid(p, K)
        data[name] = dict(n=int(p.shape[0]), d=int(p.shape[1]), K=int(K),
                          candidates=st["candidates"], passes=st["passes"],
                          pass_queries=st["pass_queries"], pass_candidates=st["pass_candidates"],
                          eps_min=st["eps_min"], eps_mean=st["eps_mean"], width=st["width"],
                          oracle_seconds=round(time.time() - t, 2), threads=os.cpu_count())
        data["_about"] = ("W_ref: candidate distance evaluations of the oracle's grid join "
                          "(oracle/knn_oracle.c, oracle_grid, width multiplier 1), written by "
                          "oracle/wref.py")
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(name, data[name], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or [k for k in gen.CONFIGS if k.endswith("_2m")])
