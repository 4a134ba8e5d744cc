"""Parity of the scheme's variants on the CUDA path (through the C ABI) with
the FP64 CPU oracle:

  * K_z != K_y (Eq. 16; K = max(K_y, K_z) levels per step), in particular
    the balanced choice K_z = K_y + 1 the paper suggests after Eq. 17;
  * the E[y^{n+1} DeltaW_1] / dt form of the z line's first term (the
    quantity Eq. 20 replaces by E[z^{n+1}], Eq. 12 with l = 1);
  * the one-step start-up of Section 3.1 step 2 (the 1-step scheme from t_N
    with step dt / S).

Tolerances are those of the main parity tests: FP64 1e-12, FP32C 2e-7,
relative to max(1, max |level value|).  Where the z form is unstable
(K_z >= 2, a root of modulus > 1) only a short horizon is compared.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_13560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)
TOL = {"fp64": 1e-12, "fp32c": 2e-7}


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_13560_gb300 import bsde
    bsde.load()
    return bsde


def _with(p, **kw):
    q = dict(p)
    q.update(kw)
    return q


def _cmp(got, ref, tol, what):
    scale = max(1.0, float(np.max(np.abs(ref["y"]))))
    zscale = max(1.0, float(np.max(np.abs(ref["z"]))))
    ey = float(np.max(np.abs(got["y"] - ref["y"])))
    ez = float(np.max(np.abs(got["z"] - ref["z"])))
    e0y = abs(got["y0"] - ref["y0"])
    e0z = abs(got["z0"] - ref["z0"])
    msg = f"{what}: max|dy|={ey:.3e} max|dz|={ez:.3e} |dy0|={e0y:.3e} |dz0|={e0z:.3e}"
    print(msg)
    assert ey <= tol * scale and e0y <= tol * scale, msg
    assert ez <= tol * zscale and e0z <= tol * zscale, msg
    assert got["levels_done"] == ref["levels_done"], msg
    assert got["picard_iters_max"] <= ref["picard_iters_max"] + 2, msg


KYKZ = {
    "sin_1_2": _with(W.sin_problem(Nx=1001, N=32, k=1), kz=2),
    "sin_2_3": _with(W.sin_problem(Nx=1001, N=32, k=2), kz=3),
    "sin_3_2": _with(W.sin_problem(Nx=1001, N=32, k=3), kz=2),
    "bs_3_4": _with(W.call_problem(Nx=2049, N=64, k=3), kz=4),
    "bs_5_6": _with(W.call_problem(Nx=2049, N=64, k=5), kz=6),
    "lb_2_3": _with(W.config3(Nx=2049, N=64, k=2), kz=3),
    "ex2_4_1": _with(W.ex2_problem(Nx=1025, N=32, k=4, L=16), kz=1),
    "ragged_1_4": _with(W.sin_problem(Nx=1037, N=20, k=1, L=7), kz=4),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("name", list(KYKZ))
def test_ky_kz_parity(B, name, prec):
    p = KYKZ[name]
    ref = O.solve(p, threads=THREADS, want_level=True)
    got = B.solve(p, prec, want_level=True)
    _cmp(got, ref, TOL[prec], f"{prec} {name}")


ZFORM = {
    "sin_k1": _with(W.sin_problem(Nx=1001, N=32, k=1), zform=1),
    "bs_k1": _with(W.call_problem(Nx=2049, N=64, k=1), zform=1),
    "ex2_k1": _with(W.ex2_problem(Nx=1025, N=32, k=1, L=16), zform=1),
    "ex1_2_1": _with(W.ex1_problem(Nx=1025, N=32, k=2, L=16), kz=1, zform=1),
    "sin_k2_short": _with(W.sin_problem(Nx=1001, N=4, k=2, T=0.1), zform=1),
    "ragged_k1_L7": _with(W.sin_problem(Nx=1037, N=20, k=1, L=7), zform=1),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("name", list(ZFORM))
def test_zform_parity(B, name, prec):
    p = ZFORM[name]
    ref = O.solve(p, threads=THREADS, want_level=True)
    got = B.solve(p, prec, want_level=True)
    _cmp(got, ref, TOL[prec], f"{prec} {name}")


ONESTEP = {
    "ex1_k2_S1": _with(W.ex1_problem(Nx=1025, N=16, k=2, L=16), init_mode="ONESTEP",
                       init_substeps=1),
    "ex1_k3_S4": _with(W.ex1_problem(Nx=1025, N=16, k=3, L=16), init_mode="ONESTEP",
                       init_substeps=4),
    "ex2_k4_S3": _with(W.ex2_problem(Nx=1025, N=32, k=4, L=16), init_mode="ONESTEP",
                       init_substeps=3),
    "bs_smooth_k6_S2": _with(W.call_problem(Nx=2049, N=64, k=6), init_mode="ONESTEP",
                             init_substeps=2),
    "sin_2_3_S5": _with(W.sin_problem(Nx=1037, N=20, k=2, L=7), kz=3, init_mode="ONESTEP",
                        init_substeps=5),
    "sin_k1_noop": _with(W.sin_problem(Nx=1001, N=16, k=1), init_mode="ONESTEP",
                         init_substeps=7),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("name", list(ONESTEP))
def test_onestep_parity(B, name, prec):
    p = ONESTEP[name]
    ref = O.solve(p, threads=THREADS, want_level=True)
    got = B.solve(p, prec, want_level=True)
    _cmp(got, ref, TOL[prec], f"{prec} {name}")


def test_onestep_launch_count(B):
    p = ONESTEP["ex1_k3_S4"]
    s = B.Solver(p, "fp64")
    K, S, N = 3, 4, p["N"]
    main = 1 + 2 * K + 2 * (N - K + 1) + 2
    startup = 3 + 2 * (K - 1) * S + (K - 1)
    assert s.launches == main + startup
    s.close()


def test_onestep_caller_levels_skip_the_startup(B):
    """With caller levels the start-up is not run: the result equals that of
    a closed-form-start plan given the same levels, and differs from the
    start-up's own."""
    p = ONESTEP["ex1_k3_S4"]
    iy, iz = O.init_levels(p)
    a = B.solve(p, "fp64", init=(iy, iz))
    b = B.solve(_with(p, init_mode="EXACT"), "fp64", init=(iy, iz))
    c = B.solve(p, "fp64")
    assert a["y0"] == b["y0"] and a["z0"] == b["z0"]
    assert a["z0"] != c["z0"]


def test_variants_in_a_batch_equal_single_solves(B):
    probs = [KYKZ["bs_3_4"], KYKZ["ex2_4_1"], ZFORM["bs_k1"], ZFORM["ex1_2_1"],
             W.call_problem(Nx=1500, N=32, k=2)]
    bs = B.BatchSolver(probs)
    res = bs.solve()
    bs.close()
    for p, r in zip(probs, res):
        s = B.solve(p, "fp32c")
        assert r["y0"] == s["y0"] and r["z0"] == s["z0"], p
        assert r["levels_done"] == s["levels_done"]


def test_batch_rejects_the_startup(B):
    with pytest.raises(B.BsdeError):
        B.BatchSolver([ONESTEP["ex1_k3_S4"]])


@pytest.mark.parametrize("name,fields", [("ky1_kz2", dict(k=1, kz=2)),
                                         ("k1_zform", dict(k=1, zform=1)),
                                         ("k2_onestep_S8", dict(k=2, init_mode="ONESTEP",
                                                                init_substeps=8))])
def test_config2_full_size_variants(B, name, fields):
    """The benchmark workload (Nx = 65536, N = 256, L = 16) with the variants
    the benchmark times: whole level 0 against the oracle in both
    precisions."""
    f = dict(fields)
    p = W.config2(k=f.pop("k"))
    p.update(f)
    ref = O.solve(p, threads=THREADS, want_level=True)
    for prec in ("fp64", "fp32c"):
        got = B.solve(p, prec, want_level=True)
        _cmp(got, ref, TOL[prec], f"config2 {name} {prec}")
