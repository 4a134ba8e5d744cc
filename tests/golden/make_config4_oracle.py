"""Write config4_oracle.json: the FP64 oracle's (y0, z0) for every instance
of the 4096-instance Black-Scholes batch (seed 13560: strike ~ U[70, 130],
sigma ~ U[.1, .5], T ~ U[.25, 2], r ~ U[0, .05], Nx in {2^10..2^14},
N in {32, 64, 128, 256}, k ~ U{1..6}, L = 16), beside the closed-form price
(Black-Scholes, Section 5 Example 3 without dividend).  Rows are in the order
of workloads.config4().  Calls only the oracle; about 20 minutes on 8 host
threads (instances are solved in parallel, one host thread each).

    python tests/golden/make_config4_oracle.py
"""
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

COUNT, SEED = 4096, 13560


def _num(v):
    return v if math.isfinite(v) else repr(v)


def _one(i):
    from oracle import oracle as O
    from paper_1909_13560_gb300 import workloads as W
    p = W.config4(count=COUNT, seed=SEED)[i]
    r = O.solve(p, threads=1)
    u, z = O.exact(p, 0.0, p["x0"])
    return [_num(r["y0"]), _num(r["z0"]), u, z, r["status"]]


def main():
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    # spawn: the workers load their own copy of the oracle library
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        rows = pool.map(_one, range(COUNT), chunksize=8)
    out = {"workload": "config4", "count": COUNT, "seed": SEED,
           "columns": ["y0", "z0", "exact_y0", "exact_z0", "status"], "rows": rows}
    with open(os.path.join(HERE, "config4_oracle.json"), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))
    print(f"{COUNT} instances in {time.perf_counter() - t0:.0f} s")


if __name__ == "__main__":
    main()
