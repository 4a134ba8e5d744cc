"""Write config2_oracle.json: the FP64 oracle's (y0, z0) for the benchmark
workload (Black-Scholes call, Nx = 65536, N = 256, L = 16, k = 1..6), for the
scheme's variants on the same workload (K_z != K_y, the E[y dW]/dt z form,
the one-step start-up; VARIANTS below) and the closed-form price and z at
t = 0.  Calls only the oracle.

    python tests/golden/make_config2_oracle.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1909_13560_gb300 import workloads as W  # noqa: E402


# name -> problem fields changed from config2(k)
VARIANTS = {
    "ky1_kz2": dict(k=1, kz=2),
    "ky2_kz3": dict(k=2, kz=3),
    "ky2_kz1": dict(k=2, kz=1),
    "k1_zform": dict(k=1, zform=1),
    "k2_onestep_S8": dict(k=2, init_mode="ONESTEP", init_substeps=8),
    "k3_onestep_S8": dict(k=3, init_mode="ONESTEP", init_substeps=8),
}


def variant_problem(name):
    v = dict(VARIANTS[name])
    p = W.config2(k=v.pop("k"))
    p.update(v)
    return p


def main():
    out = {"workload": "config2", "rows": [], "variants": []}
    for k in range(1, 7):
        p = W.config2(k=k)
        r = O.solve(p, threads=os.cpu_count() or 1)
        u, z = O.exact(p, 0.0, p["x0"])
        out["rows"].append({"k": k, "y0": r["y0"], "z0": r["z0"], "exact_y0": u,
                            "exact_z0": z, "picard_iters_max": r["picard_iters_max"]})
        print(k, r["y0"], r["z0"], flush=True)
    for name in VARIANTS:
        p = variant_problem(name)
        r = O.solve(p, threads=os.cpu_count() or 1)
        u, z = O.exact(p, 0.0, p["x0"])
        out["variants"].append({"name": name, "fields": VARIANTS[name], "y0": r["y0"],
                                "z0": r["z0"], "exact_y0": u, "exact_z0": z,
                                "picard_iters_max": r["picard_iters_max"]})
        print(name, r["y0"], r["z0"], flush=True)
    with open(os.path.join(HERE, "config2_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
