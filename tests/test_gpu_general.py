"""Parity of the general forward path on the CUDA side (through the C ABI)
with the oracle: affine forward coefficients advanced by one Euler step per
node and point, the short-rate driver f = -x y, the Vasicek bond and the
price-space call, with both z forms, the one-step start-up and caller
levels.  Tolerances as for the main parity tests: 1e-12 relative (FP64),
2e-7 relative (FP32C)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_13560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)
TOL = 1e-12


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


def _cmp(got, ref, what, tol=TOL):
    scale = max(1.0, float(np.max(np.abs(ref["y"]))))
    zscale = max(1.0, float(np.max(np.abs(ref["z"]))))
    ey = float(np.max(np.abs(got["y"] - ref["y"])))
    ez = float(np.max(np.abs(got["z"] - ref["z"])))
    msg = (f"{what}: max|dy|={ey:.3e} max|dz|={ez:.3e} |dy0|={abs(got['y0'] - ref['y0']):.3e} "
           f"|dz0|={abs(got['z0'] - ref['z0']):.3e}")
    print(msg)
    assert ey <= tol * scale and ez <= tol * zscale, msg
    assert abs(got["y0"] - ref["y0"]) <= tol * scale and abs(got["z0"] - ref["z0"]) <= tol * zscale
    assert got["picard_iters_max"] <= ref["picard_iters_max"] + 2


CASES = {
    "vasicek_k1_ydw": _with(W.vasicek_problem(Nx=1537, N=32, k=1), zform=1),
    "vasicek_k3_kz1_ydw": _with(W.vasicek_problem(Nx=1537, N=32, k=3), kz=1, zform=1),
    "vasicek_k4_ez": W.vasicek_problem(Nx=1025, N=24, k=4),
    "vasicek_onestep": _with(W.vasicek_problem(Nx=1025, N=16, k=3), kz=1, zform=1,
                             init_mode="ONESTEP", init_substeps=4),
    "gbm_call_k3": W.gbm_call_problem(Nx=2049, N=32, k=3),
    "gbm_call_k2_nosmooth": W.gbm_call_problem(Nx=1501, N=24, k=2, smoothing=0),
    "affine_sin_ragged": _with(W.sin_problem(Nx=1037, N=20, k=2, L=7), forward="AFFINE",
                               a_x=0.1, a_1=-0.2, b_x=0.9, b_1=0.05),
    "short_rate_const_fwd": _with(W.sin_problem(Nx=801, N=12, k=3, L=8), driver="SHORT_RATE"),
}


@pytest.mark.parametrize("prec,tol", [("fp64", TOL), ("fp32c", 2e-7)])
@pytest.mark.parametrize("name", list(CASES))
def test_general_forward_parity(B, name, prec, tol):
    p = CASES[name]
    ref = O.solve(p, threads=THREADS, want_level=True)
    got = B.solve(p, prec, want_level=True)
    _cmp(got, ref, f"{name} {prec}", tol)


def test_zero_slopes_match_the_constant_kernel(B):
    """The general kernel with zero slopes and the constant-shift kernel solve
    the same scheme (their arithmetic differs, their results agree to
    rounding)."""
    p = W.call_problem(Nx=1025, N=16, k=3)
    a = B.solve(p, "fp64", want_level=True)
    b = B.solve(_with(p, forward="AFFINE", a_1=0.0, b_1=0.0), "fp64", want_level=True)
    scale = max(1.0, float(np.max(np.abs(a["y"]))))
    assert float(np.max(np.abs(a["y"] - b["y"]))) <= TOL * scale


def test_general_forward_with_caller_levels(B):
    p = _with(W.vasicek_problem(Nx=1025, N=16, k=2), kz=1, zform=1)
    iy, iz = O.init_levels(p)
    iy = iy * (1.0 + 0.01 * np.linspace(-1, 1, p["Nx"]))
    ref = O.solve(p, iy, iz, threads=THREADS, want_level=True)
    got = B.solve(p, "fp64", init=(iy, iz), want_level=True)
    _cmp(got, ref, "vasicek caller levels")


def test_general_forward_fp32c_caller_levels(B):
    p = _with(W.vasicek_problem(Nx=1025, N=16, k=2), kz=1, zform=1)
    iy, iz = O.init_levels(p)
    iy = iy * (1.0 + 0.01 * np.linspace(-1, 1, p["Nx"]))
    ref = O.solve(p, iy, iz, threads=THREADS, want_level=True)
    got = B.solve(p, "fp32c", init=(iy, iz), want_level=True)
    _cmp(got, ref, "vasicek caller levels fp32c", 2e-7)
