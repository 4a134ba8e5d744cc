"""Pins of the oracle's general forward path: the forward process advanced
from the grid point by one Euler step, X = x + a(x) j dt + b(x) DeltaW with
a, b affine in x (the general Markovian X of Section 1), an x-dependent
driver (f = -x y, the short-rate discount), and two closed forms:

* the Vasicek zero-coupon bond (dX = kappa (theta - X) dt + sigma dW, g = 1)
  and the Black-Scholes call in the price itself (dS = mu S dt + sigma S dW)
  against their PDEs by finite differences;
* the scheme converges to them at the Euler rate: for Vasicek only with the
  E[y^{n+1} DeltaW_1] / dt z form (K_z = 1), while Eq. 20's E[z^{n+1}]
  leaves a z error of the size of z itself whatever N is -- the identity
  E[y DeltaW] = dt E[z] behind it holds for constant coefficients only;
* zero slopes reproduce the constant-coefficient scheme bit for bit.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_13560_gb300 import workloads as W

THREADS = max(1, os.cpu_count() or 1)


def _fit(e):
    return [math.log2(a / b) for a, b in zip(e, e[1:])]


def test_zero_slopes_reproduce_the_constant_scheme():
    p = W.call_problem(Nx=1025, N=16, k=3)
    q = dict(p, forward="AFFINE", a_1=0.0, b_1=0.0)
    a = O.solve(p, threads=THREADS, want_level=True)
    b = O.solve(q, threads=THREADS, want_level=True)
    assert np.array_equal(a["y"], b["y"]) and np.array_equal(a["z"], b["z"])


def _pde_residual(p, t, x, h=1e-4):
    u = lambda tt, xx: O.exact(p, tt, xx)[0]
    ut = (u(t + h, x) - u(t - h, x)) / (2 * h)
    hx = h * max(1.0, abs(x))
    ux = (u(t, x + hx) - u(t, x - hx)) / (2 * hx)
    uxx = (u(t, x + hx) - 2 * u(t, x) + u(t, x - hx)) / hx ** 2
    a = p["a_x"] + p.get("a_1", 0.0) * x
    b = p["b_x"] + p.get("b_1", 0.0) * x
    z = O.exact(p, t, x)[1]
    assert z == pytest.approx(b * ux, rel=1e-5, abs=1e-9)
    return ut + a * ux + 0.5 * b * b * uxx + O.driver(p, t, u(t, x), z, x)


def test_vasicek_bond_solves_its_pde():
    p = W.vasicek_problem()
    for t, x in [(0.3, 0.01), (1.2, 0.05), (1.9, 0.035)]:
        assert abs(_pde_residual(p, t, x)) < 1e-6


def test_price_space_call_solves_its_pde():
    p = W.gbm_call_problem()
    for t, x in [(0.2, 90.0), (0.6, 104.0), (0.9, 120.0)]:
        assert abs(_pde_residual(p, t, x)) < 2e-4


def _vasicek_errors(**kw):
    p0 = W.vasicek_problem()
    u, z = O.exact(p0, 0.0, p0["x0"])
    ey, ez = [], []
    for N in (16, 32, 64, 128):
        p = W.vasicek_problem(N=N, k=kw.get("k", 1), Nx=4097)
        p.update(kw)
        r = O.solve(p, threads=THREADS)
        ey.append(abs(r["y0"] - u))
        ez.append(abs(r["z0"] - z))
    return ey, ez, z


@pytest.mark.parametrize("kw", [dict(k=1, zform=1), dict(k=2, kz=1, zform=1)])
def test_vasicek_converges_at_the_euler_rate_with_the_ydw_z_form(kw):
    ey, ez, _ = _vasicek_errors(**kw)
    assert min(_fit(ey)) >= 0.8, ey
    assert ez[-1] < 1e-4 and ez[-1] < ez[0]


def test_vasicek_z_is_inconsistent_with_the_ez_form():
    ey, ez, z = _vasicek_errors(k=2)
    assert min(_fit(ey)) >= 0.8  # y does not see z (f = -x y)
    assert min(ez) > 0.5 * abs(z)  # z misses the drift's slope: no convergence


def test_price_space_call_converges_to_black_scholes():
    p0 = W.gbm_call_problem()
    u, z = O.exact(p0, 0.0, p0["x0"])
    ey, ez = [], []
    for N in (16, 32, 64, 128):
        r = O.solve(W.gbm_call_problem(N=N, k=3, Nx=4097), threads=THREADS)
        ey.append(abs(r["y0"] - u))
        ez.append(abs(r["z0"] - z))
    assert min(_fit(ey)) >= 0.8 and min(_fit(ez)) >= 0.8, (ey, ez)


def test_price_space_cell_average():
    """The smoothed level N: averages over [x - dx/2, x + dx/2] of the payoff
    and of b(s) 1{s > K}, against a fine midpoint rule."""
    p = W.gbm_call_problem(Nx=41, N=8, k=1, smoothing=1)
    iy, iz = O.init_levels(p)
    dx = (p["x_max"] - p["x_min"]) / (p["Nx"] - 1)
    x = p["x_min"] + dx * np.arange(p["Nx"])
    s = (np.arange(2_000_000) + 0.5) / 2_000_000 - 0.5  # the jump at K costs ~1/n
    for i in range(p["Nx"]):
        ss = x[i] + dx * s
        assert iy[0, i] == pytest.approx(np.mean(np.maximum(ss - p["strike"], 0.0)), abs=1e-6)
        assert iz[0, i] == pytest.approx(np.mean(p["b_1"] * ss * (ss > p["strike"])), abs=1e-5)


def test_short_rate_driver_reads_the_forward_state():
    p = W.vasicek_problem()
    assert O.driver(p, 0.3, 2.0, 0.5, x=0.04) == pytest.approx(-0.08)
