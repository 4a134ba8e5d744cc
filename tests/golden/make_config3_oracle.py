"""Write config3_oracle.json: the FP64 oracle's (y0, z0) for the lending/
borrowing call at full size (Nx = 2^20, N = 1024, L = 16; r = .04, R = .06,
mu = .06, sigma = .2, T = .5, strike 100) for k = 2 and the configuration's
k = 4, beside the closed-form price and z at t = 0 (Black-Scholes at the rate
r - (R - r), Section 5 Example 3 with the borrowing term).  Calls only the
oracle.  About 16 minutes on 8 host threads.

    python tests/golden/make_config3_oracle.py
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1909_13560_gb300 import workloads as W  # noqa: E402

KS = (2, 4)


def _num(v):
    # JSON has no NaN or infinity: a non-finite oracle value is stored as text
    return v if math.isfinite(v) else repr(v)


def main():
    out = {"workload": "config3", "Nx": 1 << 20, "N": 1024, "L": 16, "rows": []}
    threads = os.cpu_count() or 1
    for k in KS:
        p = W.config3(k=k)
        t0 = time.perf_counter()
        r = O.solve(p, threads=threads)
        u, z = O.exact(p, 0.0, p["x0"])
        out["rows"].append({"k": k, "y0": _num(r["y0"]), "z0": _num(r["z0"]), "exact_y0": u,
                            "exact_z0": z, "picard_iters_max": r["picard_iters_max"],
                            "status": r["status"]})
        print(k, r["y0"], r["z0"], f"{time.perf_counter() - t0:.0f} s", flush=True)
    with open(os.path.join(HERE, "config3_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
