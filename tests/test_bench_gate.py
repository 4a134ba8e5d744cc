"""The benchmark's accuracy gate and the stored FP64 oracle values it reads
(CPU only).

A solve counts towards the benchmark's value only when the scheme converges
on its grid (the stored oracle within 1% of the closed form) and the solve
agrees with the stored oracle within its precision's tolerance.  These tests
pin the gate's decisions on constructed cases and the stored files'
contents: which configurations the oracle says converge, and that each
stored closed-form value is the closed form.
"""
import json
import math
import os

import pytest

import bench
from paper_1909_13560_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_gate_counts_a_solve_that_matches_a_converged_oracle():
    g = bench.gate(6.1205154, 11.1246292, 6.12051547, 11.12462915, 6.1206541, 11.1246292, "fp32c")
    assert g["scheme_converges"] and g["within_tol"] and g["counted"]


def test_gate_rejects_a_solve_outside_the_precision_tolerance():
    # 1e-5 off the oracle: fine for an accuracy test, not for parity in FP32C
    g = bench.gate(6.12052547, 11.1246292, 6.12051547, 11.1246292, 6.1206541, 11.1246292, "fp32c")
    assert g["scheme_converges"] and not g["within_tol"] and not g["counted"]
    # the FP64 tolerance is tighter still
    g = bench.gate(6.12051547 + 1e-10, 11.1246292, 6.12051547, 11.1246292, 6.1206541,
                   11.1246292, "fp64")
    assert not g["within_tol"]


def test_gate_rejects_agreement_with_a_diverged_oracle():
    # both runs follow the same growth: agreement, but no price
    y, z = -8.878994155823492e+58, 2.3512543600937575e+62
    g = bench.gate(y, z, y, z, 6.1206541, 11.1246292, "fp32c")
    assert g["within_tol"] and not g["scheme_converges"] and not g["counted"]


def test_gate_rejects_non_finite_results():
    g = bench.gate(float("nan"), float("nan"), 6.12051547, 11.1246292, 6.1206541, 11.1246292,
                   "fp32c")
    assert not g["within_tol"] and not g["counted"]
    g = bench.gate(1.0, 1.0, float("nan"), 1.0, 1.0, 1.0, "fp32c")
    assert not g["scheme_converges"]


def test_gate_z_matters_too():
    # config2 k = 3: y within 1e-4 of the price but z 16% off it
    g = bench.gate(9.414539756, 10.0625213, 9.414539756, 10.0625213, 9.413403384, 11.974126514,
                   "fp32c")
    assert not g["scheme_converges"]


def test_stored_config3_values():
    gold = bench._golden("config3")
    assert set(gold) == {2, 4}
    u, z = bench._closed_form_call(W.config3(k=2))
    for k in (2, 4):
        # the stored closed form is Black-Scholes at r - (R - r) (reading 13)
        assert gold[k]["exact_y0"] == pytest.approx(u, rel=1e-12)
        assert gold[k]["exact_z0"] == pytest.approx(z, rel=1e-12)
    assert bench.gate(gold[2]["y0"], gold[2]["z0"], gold[2]["y0"], gold[2]["z0"],
                      gold[2]["exact_y0"], gold[2]["exact_z0"], "fp64")["counted"]
    assert not bench.gate(gold[4]["y0"], gold[4]["z0"], gold[4]["y0"], gold[4]["z0"],
                          gold[4]["exact_y0"], gold[4]["exact_z0"], "fp64")["scheme_converges"]


def test_stored_config2_values_converge_for_k_up_to_2():
    gold = bench._golden("config2")
    conv = {k: bench.gate(g["y0"], g["z0"], g["y0"], g["z0"], g["exact_y0"], g["exact_z0"],
                          "fp64")["scheme_converges"] for k, g in gold.items()}
    assert conv == {1: True, 2: True, 3: False, 4: False, 5: False, 6: False}


def test_stored_config4_values_match_the_instances():
    rows = bench._golden4()
    probs = W.config4()
    assert rows is not None and len(rows) == len(probs) == 4096
    with open(os.path.join(GOLDEN, "config4_oracle.json")) as fh:
        meta = json.load(fh)
    assert meta["seed"] == 13560 and meta["columns"][:4] == ["y0", "z0", "exact_y0", "exact_z0"]
    # the stored closed form is the instance's Black-Scholes price (sampled)
    for i in range(0, 4096, 257):
        p = probs[i]
        u, _ = bench._closed_form_call(p)
        assert rows[i][2] == pytest.approx(u, rel=1e-10, abs=1e-12)
    conv = sum(1 for y, z, u, zz in rows
               if math.isfinite(y) and abs(y - u) <= 1e-2 * max(1.0, abs(u))
               and abs(z - zz) <= 1e-2 * max(1.0, abs(zz)))
    assert conv == 3185


def test_roofline_flop_counts():
    # the method's count: 42 flop per node with compensated sums (30 plain),
    # 3 per step j, 6 per Picard iteration
    assert bench.flops_per_gp_step_method(2, 16, True, 4) == 42 * 32 + 6 + 24
    assert bench.flops_per_gp_step_method(4, 16, False, 5) == 30 * 64 + 12 + 30
    # the narrower count: 23 per node, 2L + 4k + 12 per point
    assert bench.flops_per_gp_step(2, 16) == 23 * 32 + 32 + 8 + 12
    # the 2-D tensor-product passes, per point and level
    fp = bench.flops_per_gp_step_tp(6, 8, "fp64")
    assert fp == {"x2": 6 * 8 * 66.0, "x1": 6 * 8 * 60.0 + 6 * 27.0 + 80.0}
    f32 = bench.flops_per_gp_step_tp(6, 8, "fp32c")
    assert f32["x2"] == 6 * 4 * 195.0 and f32["x1"] == 6 * 4 * 193.0 + 80.0


@pytest.mark.parametrize("kernel", ["k_step32f_config3", "k_step32f_config2", "k_step32_config2",
                                    "k2_tp1_32", "k2_tp2_32", "k2_tp1", "k2_tp2", "k2_step32p"])
def test_roofline_traffic_entries(kernel):
    """Every kernel whose DRAM traffic the bench line reports has an entry in
    the committed traffic table, positive, with the profile summary it came
    from."""
    t = bench._traffic(kernel)
    assert t is not None and t > 0
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "profiles", "dram_traffic.json")) as fh:
        entry = json.load(fh)[kernel]
    assert entry["workload"]
    refs = [w for w in entry["note"].replace(",", " ").replace(")", " ").split()
            if w.endswith(".md")]
    assert refs and all(os.path.exists(os.path.join(root, "profiles", r)) for r in refs)
    assert bench._traffic("no_such_kernel") is None
