"""Batched solves (one persistent launch for many uneven problems) against
single solves and the oracle."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_13560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)
TOL32 = 2e-7


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_13560_gb300 import bsde
    bsde.load()
    return bsde


def _mixed(count=42, seed=7):
    """Uneven problems: the config4 recipe at smaller sizes, plus
    lending/borrowing calls, the paper's two nonlinear examples and the
    linear sin problem (all five drivers)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = i % 6
        k = int(rng.integers(1, 7))
        N = int(8 << int(rng.integers(0, 3)))
        k = min(k, N)
        Nx = int(rng.integers(200, 3000))
        if kind <= 1:
            out.append(W.call_problem(strike=float(rng.uniform(70, 130)),
                                      sigma=float(rng.uniform(0.1, 0.5)),
                                      T=float(rng.uniform(0.25, 2.0)),
                                      r=float(rng.uniform(0.0, 0.05)), Nx=Nx, N=N, k=k, L=16))
        elif kind == 2:
            out.append(W.call_problem(strike=100.0, sigma=0.2, T=0.5, r=0.04, R=0.06, mu=0.06,
                                      Nx=Nx, N=N, k=k, L=16, driver="LB"))
        elif kind == 3:
            out.append(W.ex1_problem(Nx=Nx, N=N, k=k, L=12, x_lim=8.0))
        elif kind == 4:
            out.append(W.ex2_problem(Nx=Nx, N=N, k=k, L=12, x_lim=8.0))
        else:
            out.append(W.sin_problem(Nx=Nx, N=N, k=k, L=8))
    return out


def test_batch_equals_single_solves(B):
    probs = _mixed()
    bs = B.BatchSolver(probs)
    res = bs.solve()
    bs.close()
    for p, r in zip(probs, res):
        s = B.solve(p, "fp32c")
        assert r["y0"] == s["y0"] and r["z0"] == s["z0"], (p["driver"], p["Nx"], p["N"], p["k"])
        assert r["status"] == s["status"]


def test_batch_alone_equals_in_the_mix(B):
    probs = _mixed(count=30, seed=11)
    mix = B.BatchSolver(probs)
    res = mix.solve()
    mix.close()
    for i in (0, 7, 19, 29):
        one = B.BatchSolver([probs[i]])
        r1 = one.solve()[0]
        one.close()
        assert r1["y0"] == res[i]["y0"] and r1["z0"] == res[i]["z0"]


@pytest.mark.parametrize("cluster,groups,flat", [(1, 4, 0), (4, 4, 0), (8, 2, 0), (2, 6, 0),
                                                 (1, 1, 1), (4, 1, 1), (2, 4, 1)])
def test_batch_configs_agree_with_oracle(B, cluster, groups, flat):
    probs = _mixed(count=12, seed=3)
    bs = B.BatchSolver(probs)
    bs.set_config(cluster, groups, flat)
    assert bs.config() == {"cluster": cluster, "target_groups": groups, "flat_tiles": flat}
    res = bs.solve()
    bs.close()
    for p, r in zip(probs, res):
        ref = O.solve(p, threads=THREADS, want_level=True)
        scale = max(1.0, float(np.max(np.abs(ref["y"]))))
        zscale = max(1.0, float(np.max(np.abs(ref["z"]))))
        assert abs(r["y0"] - ref["y0"]) <= TOL32 * scale, (p["driver"], r["y0"], ref["y0"])
        assert abs(r["z0"] - ref["z0"]) <= TOL32 * zscale, (p["driver"], r["z0"], ref["z0"])


def test_batch_autotune_picks_a_valid_config(B):
    probs = _mixed(count=20, seed=5)
    bs = B.BatchSolver(probs)
    before = bs.solve()
    best = bs.autotune()
    assert best["cluster"] in (1, 2, 4, 8)
    assert (best["target_groups"], best["flat_tiles"]) in ((2, 0), (4, 0), (6, 0), (1, 1))
    assert bs.config() == best
    after = bs.solve()
    bs.close()
    for a, b in zip(before, after):
        assert abs(a["y0"] - b["y0"]) <= 1e-6 * max(1.0, abs(a["y0"]))


@pytest.mark.parametrize("groups", [1, 4, 6])
def test_batch_flat_tiles_equal_grouped_tiles_bitwise(B, groups):
    """Flat step tiles (one point per thread, its groups in turn) and grouped
    ones (groups of threads per point, partial sums folded in shared memory)
    with the same group split run the same pairs in the same order of
    operations: bitwise equal results, whatever the cluster size."""
    probs = _mixed(count=20, seed=13)
    bs = B.BatchSolver(probs)
    bs.set_config(2, groups, 0)
    a = bs.solve()
    bs.set_config(4, groups, 1)
    b = bs.solve()
    bs.close()
    for x, y in zip(a, b):
        assert x["y0"] == y["y0"] and x["z0"] == y["z0"] and x["status"] == y["status"]


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_batch_cluster_sizes_equal_bitwise(B, cluster):
    """The CTAs of a cluster share an instance's level phases; a cluster size
    changes which SM computes which tile, never a result: bitwise equal to
    1-CTA clusters at the same group split."""
    probs = _mixed(count=20, seed=29)
    bs = B.BatchSolver(probs)
    bs.set_config(1, 1, 1)
    a = bs.solve()
    bs.set_config(cluster, 1, 1)
    b = bs.solve()
    b2 = bs.solve()
    bs.close()
    for x, y, y2 in zip(a, b, b2):
        assert x["y0"] == y["y0"] and x["z0"] == y["z0"] and x["status"] == y["status"]
        assert y["y0"] == y2["y0"] and y["z0"] == y2["z0"]


def test_batch_rejects_fp64_problems(B):
    with pytest.raises(B.BsdeError) as ei:
        B.bsde_batch_workspace_bytes([W.sin_problem()], "fp64")
    assert ei.value.code == B.BSDE_EINVAL


def _stored_config4():
    import json
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "config4_oracle.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return [[float(v) for v in r[:4]] for r in json.load(fh)["rows"]]


def test_config4_sample_against_oracle(B):
    """The first 64 instances of the 4096-instance Black-Scholes batch (seed
    13560) in one persistent launch.  Where the scheme converges on an
    instance's grid (the FP64 oracle's y0 and z0 within 1% of the closed
    form, the bench's criterion) the batch's y0 and z0 agree with the oracle
    within the FP32C tolerance.  Where it diverges (k >= 3 on grids far finer
    than the Gauss-Hermite node spacing) the instance is counted and left
    out, as the bench leaves it out of its value; such solves are covered by
    the first-levels parity of single solves, which the batch equals bit for
    bit (test_batch_equals_single_solves).  The live oracle also reproduces
    the values stored for the bench's gate."""
    probs = W.config4(count=64)
    bs = B.BatchSolver(probs)
    res = bs.solve()
    bs.close()
    stored = _stored_config4()
    conv = div = 0
    worst = 0.0
    for i, (p, r) in enumerate(zip(probs, res)):
        ref = O.solve(p, threads=THREADS, want_level=True)
        u, z = O.exact(p, 0.0, p["x0"])
        ok = (np.isfinite(ref["y0"]) and abs(ref["y0"] - u) <= 1e-2 * max(1.0, abs(u))
              and abs(ref["z0"] - z) <= 1e-2 * max(1.0, abs(z)))
        if stored is not None:
            # written on another host: its libm may differ from this one's by an ulp
            assert abs(stored[i][2] - u) <= 1e-13 * max(1.0, abs(u))
            if ok:
                assert abs(stored[i][0] - ref["y0"]) <= 1e-10 * max(1.0, abs(ref["y0"]))
        if not ok:
            div += 1
            continue
        conv += 1
        scale = max(1.0, float(np.max(np.abs(ref["y"]))))
        zscale = max(1.0, float(np.max(np.abs(ref["z"]))))
        ey, ez = abs(r["y0"] - ref["y0"]) / scale, abs(r["z0"] - ref["z0"]) / zscale
        worst = max(worst, ey, ez)
        assert ey <= TOL32 and ez <= TOL32, (i, p["Nx"], p["N"], p["k"], r["y0"], ref["y0"])
    print(f"config4 sample: {conv} converging instances within {worst:.2e} of the oracle, "
          f"{div} diverging on their grids")
    assert conv >= 32
