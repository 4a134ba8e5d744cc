"""Pins of the FP64 CPU oracle against things other than itself.

Each test fixes one part of the oracle with an independent fact: a value the
paper prints, a closed form, an exact rational derivation, a library routine
or an invariant of the mathematics.  A plausible slip anywhere in the oracle
(a dropped term, a wrong sign or index, a swapped operand) fails at least one
of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_13560_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
THREADS = max(1, min(8, os.cpu_count() or 1))


# --------------------------------------------------------------------------
# Multistep coefficients (Tables 1 and 2) from the not-a-knot spline (Eq. 8-15)
# --------------------------------------------------------------------------

def _solve_exact(A, b):
    n = len(b)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def _spline_pieces(K, v):
    """Coefficients (a, b, c, d) per unit interval of the interpolant of the
    values v_0..v_K at t = 0..K used to integrate the driver in time: linear
    for K = 1, the parabola for K = 2 (the three-point not-a-knot spline),
    the not-a-knot cubic spline for K >= 3 (Eq. 15: interpolation plus C^1
    and C^2 continuity at the interior knots, plus continuity of the third
    derivative at the first and last interior knots)."""
    nunk = 4 * K
    rows, rhs = [], []

    def eq(coefs, val):
        row = [Fraction(0)] * nunk
        for idx, cval in coefs:
            row[idx] += Fraction(cval)
        rows.append(row)
        rhs.append(Fraction(val))

    for q in range(K):
        a, b, c, d = 4 * q, 4 * q + 1, 4 * q + 2, 4 * q + 3
        eq([(a, 1)], v[q])
        eq([(a, 1), (b, 1), (c, 1), (d, 1)], v[q + 1])
    for q in range(K - 1):
        eq([(4 * q + 1, 1), (4 * q + 2, 2), (4 * q + 3, 3), (4 * q + 5, -1)], 0)
        eq([(4 * q + 2, 2), (4 * q + 3, 6), (4 * q + 6, -2)], 0)
    if K == 1:
        eq([(2, 1)], 0)
        eq([(3, 1)], 0)
    elif K == 2:
        eq([(3, 1), (7, -1)], 0)
        eq([(3, 1)], 0)
    else:
        eq([(3, 1), (7, -1)], 0)
        eq([(4 * (K - 2) + 3, 1), (4 * (K - 1) + 3, -1)], 0)
    x = _solve_exact(rows, rhs)
    return [tuple(x[4 * q:4 * q + 4]) for q in range(K)]


def _gamma_exact(K):
    gy, gz = [], []
    for j in range(K + 1):
        v = [Fraction(int(i == j)) for i in range(K + 1)]
        pieces = _spline_pieces(K, v)
        integ = [a + b / 2 + c / 3 + d / 4 for (a, b, c, d) in pieces]
        gy.append(sum(integ) / K)   # (1/K) * integral over [0, K]: Table 1
        gz.append(integ[0])         # integral over [0, 1]: Table 2
    return gy, gz


@pytest.mark.parametrize("K", range(1, 7))
def test_gamma_tables_equal_spline_integrals(K):
    gy, gz = _gamma_exact(K)
    oy, oz = O.gamma(K)
    for j in range(K + 1):
        assert oy[j] == pytest.approx(float(gy[j]), abs=1e-16)
        assert oz[j] == pytest.approx(float(gz[j]), abs=1e-16)
    assert sum(gy) == 1 and sum(gz) == 1


def test_gamma_rejects_out_of_table():
    with pytest.raises(ValueError):
        O.gamma(7)
    with pytest.raises(ValueError):
        O.gamma(0)


# --------------------------------------------------------------------------
# Gauss-Hermite rule (Eq. 21)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("L", [1, 2, 3, 4, 8, 16, 31, 32, 64])
def test_gauss_hermite_matches_numpy(L):
    a, w = O.gauss_hermite(L)
    ra, rw = np.polynomial.hermite.hermgauss(L)
    assert np.max(np.abs(a - ra)) <= 1e-13 * max(1.0, np.abs(ra).max())
    assert np.max(np.abs(w - rw) / rw) <= 2e-12
    assert np.sum(w) == pytest.approx(math.sqrt(math.pi), rel=1e-14)


@pytest.mark.parametrize("L", [2, 5, 8, 16, 32])
def test_gauss_hermite_exact_to_degree_2L_minus_1(L):
    a, w = O.gauss_hermite(L)
    for p in range(2 * L):
        exact = 0.0 if p % 2 else math.gamma((p + 1) / 2)
        got = float(np.sum(w * a ** p))
        assert got == pytest.approx(exact, rel=1e-12, abs=1e-12 * math.gamma((p + 2) / 2))
    # and not exact one degree higher (the rule has exactly L nodes)
    p = 2 * L
    assert abs(float(np.sum(w * a ** p)) - math.gamma((p + 1) / 2)) > 1e-8


# --------------------------------------------------------------------------
# Spatial spline (natural cubic spline, Section 3.3) and clamping (Section 3.2)
# --------------------------------------------------------------------------

def test_spline_matches_scipy_natural_cubic_spline():
    from scipy.interpolate import CubicSpline
    rng = np.random.default_rng(7)
    n, x_min, x_max = 257, -3.0, 5.0
    x = np.linspace(x_min, x_max, n)
    v = np.sin(1.7 * x) + 0.3 * x ** 2 + rng.normal(0, 0.01, n)
    dx = (x_max - x_min) / (n - 1)
    M = O.spline(v, dx)
    cs = CubicSpline(x, v, bc_type="natural")
    assert np.max(np.abs(M - cs(x, 2))) <= 1e-9 * np.abs(M).max()
    for X in rng.uniform(x_min, x_max, 200):
        assert O.interp(v, M, x_min, dx, X) == pytest.approx(float(cs(X)), abs=1e-12)


def test_spline_clamps_outside_domain():
    v = np.array([3.0, -1.0, 2.0, 5.0, 4.0])
    M = O.spline(v, 0.5)
    assert O.interp(v, M, 1.0, 0.5, 0.2) == 3.0
    assert O.interp(v, M, 1.0, 0.5, 1.0) == 3.0
    assert O.interp(v, M, 1.0, 0.5, 3.0) == 4.0
    assert O.interp(v, M, 1.0, 0.5, 9.0) == 4.0
    # nodes are reproduced
    for i in range(5):
        assert O.interp(v, M, 1.0, 0.5, 1.0 + 0.5 * i) == pytest.approx(v[i], abs=1e-15)


def test_spline_reproduces_linear_data():
    x = np.linspace(-2, 2, 101)
    v = 3.0 * x - 1.0
    dx = 0.04
    M = O.spline(v, dx)
    for X in np.linspace(-2, 2, 333):
        assert O.interp(v, M, -2.0, dx, X) == pytest.approx(3 * X - 1, abs=1e-13)


def test_spline_fourth_order_on_sin():
    errs = []
    for n in (101, 201, 401):
        x = np.linspace(-4, 4, n)
        dx = 8.0 / (n - 1)
        v = np.sin(x)
        M = O.spline(v, dx)
        X = np.linspace(-1, 1, 97) + 0.3 * dx   # interior, off the nodes
        errs.append(max(abs(O.interp(v, M, -4.0, dx, t) - math.sin(t)) for t in X))
    for e0, e1 in zip(errs, errs[1:]):
        assert 12.0 < e0 / e1 < 20.0


# --------------------------------------------------------------------------
# Drivers and closed forms
# --------------------------------------------------------------------------

def test_black_scholes_closed_form_matches_paper_example3():
    # Example 3 (Eq. 30-31): T = .33, K = S0 = 100, r = .03, mu = .05,
    # delta = .04, sigma = .2, printed solution (y_0, z_0) = (4.3671, 10.0950).
    p = W.call_problem(T=0.33, r=0.03, mu=0.05, delta=0.04, sigma=0.2, Nx=5, N=4, k=1)
    u, z = O.exact(p, 0.0, math.log(100.0))
    assert round(u, 4) == 4.3671
    assert round(z, 4) == 10.0950


def test_lending_borrowing_call_reduces_to_black_scholes():
    # For a call y - z/sigma = -K e^{-r tau} N(d2) < 0, so min(.) is active and
    # the driver is linear with rate r - s(R - r): check f on that solution.
    p = W.config3(Nx=5, N=4, k=1)
    for x in (4.2, 4.6, 5.0):
        for t in (0.0, 0.25):
            u, z = O.exact(p, t, x)
            assert u - z / p["sigma"] < 0
            reff = p["r"] - p["lb_sign"] * (p["R"] - p["r"])
            f = O.driver(p, t, u, z)
            assert f == pytest.approx(-(reff * u + (p["mu"] - reff) * z / p["sigma"]), rel=1e-14)


@pytest.mark.parametrize("make", [W.sin_problem, W.ex1_problem, W.ex2_problem])
def test_closed_forms_solve_the_pde(make):
    """u_t + a u_x + b^2/2 u_xx + f(t, u, b u_x) = 0 (Eq. 5 with the forward
    drift) by central differences of the oracle's closed form."""
    p = make()
    h = 1e-4
    for t in (0.1, 0.5, 0.9):
        for x in (-1.3, 0.0, 0.7):
            u = lambda tt, xx: O.exact(p, tt, xx)[0]
            ut = (u(t + h, x) - u(t - h, x)) / (2 * h)
            ux = (u(t, x + h) - u(t, x - h)) / (2 * h)
            uxx = (u(t, x + h) - 2 * u(t, x) + u(t, x - h)) / h ** 2
            z = O.exact(p, t, x)[1]
            assert z == pytest.approx(p["b_x"] * ux, abs=1e-7)
            res = ut + p["a_x"] * ux + 0.5 * p["b_x"] ** 2 * uxx + O.driver(p, t, u(t, x), z)
            assert abs(res) < 1e-5


def test_log_price_call_cell_average():
    """Kreiss smoothing read as cell averages (Section 5, Example 3): level N
    holds the averages over [x - dx/2, x + dx/2] of the payoff (e^x - K)^+ and
    of b_X g' = sigma e^x 1{x > ln K}, against a fine midpoint rule; without
    smoothing it holds the point values."""
    p = W.call_problem(Nx=41, N=8, k=1, L=8, smoothing=1)
    iy, iz = O.init_levels(p)
    dx = (p["x_max"] - p["x_min"]) / (p["Nx"] - 1)
    x = p["x_min"] + dx * np.arange(p["Nx"])
    s = (np.arange(2_000_000) + 0.5) / 2_000_000 - 0.5  # the jump at ln K costs ~1/n
    for i in range(p["Nx"]):
        xs = x[i] + dx * s
        ey = np.exp(xs)
        assert iy[0, i] == pytest.approx(np.mean(np.maximum(ey - p["strike"], 0.0)), abs=2e-6)
        assert iz[0, i] == pytest.approx(np.mean(p["sigma"] * ey * (xs > math.log(p["strike"]))),
                                         abs=2e-5)
    py, pz = O.init_levels(dict(p, smoothing=0))
    assert np.allclose(py[0], np.maximum(np.exp(x) - p["strike"], 0.0), rtol=0, atol=1e-12)
    off_kink = np.abs(x - math.log(p["strike"])) > 1e-9  # g' is undefined at the strike
    assert np.allclose(pz[0][off_kink],
                       (p["sigma"] * np.exp(x) * (x > math.log(p["strike"])))[off_kink],
                       rtol=0, atol=1e-12)


def test_call_closed_form_solves_the_pde_in_log_price():
    p = W.call_problem(T=1.0, r=0.03, mu=0.05, delta=0.01, sigma=0.2, Nx=5, N=4, k=1)
    h = 1e-4
    for t in (0.2, 0.6):
        for x in (4.4, 4.6, 4.8):
            u = lambda tt, xx: O.exact(p, tt, xx)[0]
            ut = (u(t + h, x) - u(t - h, x)) / (2 * h)
            ux = (u(t, x + h) - u(t, x - h)) / (2 * h)
            uxx = (u(t, x + h) - 2 * u(t, x) + u(t, x - h)) / h ** 2
            z = O.exact(p, t, x)[1]
            res = ut + p["a_x"] * ux + 0.5 * p["b_x"] ** 2 * uxx + O.driver(p, t, u(t, x), z)
            assert abs(res) < 1e-5


# --------------------------------------------------------------------------
# The backward loop (Eq. 20) against printed values, closed forms, invariants
# --------------------------------------------------------------------------

def _paper_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "paper_tables.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            ex, K, N, M, ye, ze = line.split()
            rows.append((ex, int(K), int(N), int(M), float(ye), float(ze)))
    return rows


@pytest.mark.parametrize("row", _paper_rows(), ids=lambda r: f"{r[0]}-K{r[1]}-N{r[2]}-M{r[3]}")
def test_oracle_reproduces_paper_tables(row):
    ex, K, N, M, ye, ze = row
    if ex == "ex1":
        p, exact = W.ex1_problem(Nx=M + 1, N=N, k=K, L=32), (0.5, 0.25)
    else:
        p, exact = W.ex2_problem(Nx=M + 1, N=N, k=K, L=32), (math.log(3.0), 1.0 / 3.0)
    r = O.solve(p, threads=THREADS)
    # the paper prints three significant digits
    assert abs(r["y0"] - exact[0]) == pytest.approx(ye, rel=0.02)
    assert abs(r["z0"] - exact[1]) == pytest.approx(ze, rel=0.02)


def test_config1_close_to_closed_form():
    r = O.solve(W.config1(), threads=THREADS)
    assert abs(r["y0"]) < 1e-4 and abs(r["z0"] - 1.0) < 2e-4
    assert r["status"] == 0 and r["picard_iters_max"] <= 30


def _fit(errs):
    return [math.log2(a / b) for a, b in zip(errs, errs[1:])]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_time_order_z_dependent_driver(k):
    """Theorems 2.1-2.2, Remark 2.3: with f depending on z both orders are
    min(k, 3) for K_y = K_z = k (the sin problem)."""
    ey, ez = [], []
    for N in (16, 32, 64, 128):
        r = O.solve(W.sin_problem(Nx=3201, N=N, k=k, L=16), threads=THREADS)
        ey.append(abs(r["y0"]))
        ez.append(abs(r["z0"] - 1.0))
    want = min(k, 3)
    assert min(_fit(ey)[1:]) >= want - 0.3
    assert min(_fit(ez)[1:]) >= want - 0.3


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_time_order_z_free_driver(k):
    """Remark 2.3: with f independent of z the y order reaches min(k+1, 4),
    the z order min(k, 3) (Example 1 before the spatial error floor)."""
    ey, ez = [], []
    for N in (16, 32, 64):
        r = O.solve(W.ex1_problem(Nx=6401, N=N, k=k, L=32), threads=THREADS)
        ey.append(abs(r["y0"] - 0.5))
        ez.append(abs(r["z0"] - 0.25))
    assert min(_fit(ey)) >= min(k + 1, 4) - 0.3
    assert min(_fit(ez)) >= min(k, 3) - 0.3


def _grid(p):
    dx = (p["x_max"] - p["x_min"]) / (p["Nx"] - 1)
    return p["x_min"] + dx * np.arange(p["Nx"]), dx


def _zero_driver(p):
    return dict(p, driver="BS", r=0.0, mu=0.0, delta=0.0, sigma=1.0)


def test_heat_semigroup_is_exact_in_time():
    """f = 0, X = W, g = sin: u = exp(-(T-t)/2) sin x, z = u_x.  With f = 0 the
    time integration is exact, so only interpolation/quadrature error is left."""
    # domain +-12: the clamped boundary is 8 standard deviations of W_T away
    p = _zero_driver(W.sin_problem(Nx=2401, N=32, k=3, L=16, x_lim=12.0))
    x, dx = _grid(p)
    dt = p["T"] / p["N"]
    iy = np.array([np.exp(-(m * dt) / 2) * np.sin(x) for m in range(p["k"])])
    iz = np.array([np.exp(-(m * dt) / 2) * np.cos(x) for m in range(p["k"])])
    r = O.solve(p, iy, iz, threads=THREADS, want_level=True)
    inner = np.abs(x) < 4
    assert np.max(np.abs(r["y"][inner] - np.exp(-0.5) * np.sin(x[inner]))) < 1e-9
    assert np.max(np.abs(r["z"][inner] - np.exp(-0.5) * np.cos(x[inner]))) < 1e-9


def test_linear_terminal_with_drift_is_exact():
    """f = 0, dX = a dt + b dW, g = x: u = x + a (T-t), z = b, reproduced to
    rounding wherever no node leaves the domain."""
    a, b = 0.37, 0.8
    # domain +-12: no GH node chain from |x| < 3 reaches the clamped boundary
    p = _zero_driver(W.sin_problem(Nx=1201, N=16, k=4, L=8, x_lim=12.0))
    p.update(a_x=a, b_x=b)
    x, dx = _grid(p)
    dt = p["T"] / p["N"]
    iy = np.array([x + a * m * dt for m in range(p["k"])])
    iz = np.full((p["k"], p["Nx"]), b)
    r = O.solve(p, iy, iz, threads=THREADS, want_level=True)
    inner = np.abs(x) < 3
    assert np.max(np.abs(r["y"][inner] - (x[inner] + a * p["T"]))) < 1e-12
    assert np.max(np.abs(r["z"][inner] - b)) < 1e-12


def test_quadratic_terminal_with_drift_is_exact():
    """f = 0, dX = a dt + b dW, g = x^2: u = (x + a tau)^2 + b^2 tau,
    z = 2 b (x + a tau).  Cubic splines are exact on quadratics away from the
    natural end conditions, GH is exact on polynomials, f = 0 is exact in time."""
    a, b = -0.25, 0.6
    p = _zero_driver(W.sin_problem(Nx=2401, N=16, k=3, L=8, x_lim=12.0))
    p.update(a_x=a, b_x=b)
    x, dx = _grid(p)
    dt = p["T"] / p["N"]
    tau = np.array([m * dt for m in range(p["k"])])[:, None]
    iy = (x[None, :] + a * tau) ** 2 + b * b * tau
    iz = 2 * b * (x[None, :] + a * tau)
    r = O.solve(p, iy, iz, threads=THREADS, want_level=True)
    inner = np.abs(x) < 3
    T = p["T"]
    assert np.max(np.abs(r["y"][inner] - ((x[inner] + a * T) ** 2 + b * b * T))) < 1e-10
    assert np.max(np.abs(r["z"][inner] - 2 * b * (x[inner] + a * T))) < 1e-10


def _scalar_recurrence(f, c_levels, k, N, dt, tol, pmax):
    gy, _ = _gamma_exact(k)
    gy = [float(g) for g in gy]
    y = {N - m: c_levels[m] for m in range(k)}
    for n in range(N - k, -1, -1):
        A = y[n + k] + k * dt * sum(gy[j] * f((n + j) * dt, y[n + j]) for j in range(1, k + 1))
        v = y[n + 1]
        for _ in range(pmax):
            v1 = A + k * dt * gy[0] * f(n * dt, v)
            done = abs(v1 - v) <= tol
            v = v1
            if done:
                break
        y[n] = v
    return y[0]


@pytest.mark.parametrize("k", [1, 2, 3, 5, 6])
def test_space_independent_data_reduce_to_scalar_multistep(k):
    """Constant levels and a driver without z: every node carries the same
    value, so Eq. 20 collapses to the scalar recurrence
    y^n = y^{n+k} + k dt sum_j gamma_j f(y^{n+j}) + k dt gamma_0 f(y^n),
    with z identically zero."""
    p = W.ex1_problem(Nx=33, N=20, k=k, L=6, x_lim=4.0)
    dt = p["T"] / p["N"]
    c = [0.3 + 0.05 * m for m in range(k)]
    iy = np.array([[c[m]] * p["Nx"] for m in range(k)])
    iz = np.zeros((k, p["Nx"]))
    r = O.solve(p, iy, iz, want_level=True)
    f = lambda t, y: -y ** 3 + 2.5 * y ** 2 - 1.5 * y
    want = _scalar_recurrence(f, c, k, p["N"], dt, p["picard_tol"], p["picard_max"])
    assert np.max(np.abs(r["y"] - want)) < 1e-14
    assert np.max(np.abs(r["z"])) < 1e-15


def test_stein_identity_of_the_expectations():
    """E[y(X) dW] = j dt E[z] for z = b u_x (Gaussian integration by parts):
    the two estimates of Eq. 21 agree to interpolation/quadrature accuracy."""
    p = W.sin_problem(Nx=1601, N=32, k=4, L=16)
    x, dx = _grid(p)
    dt = p["T"] / p["N"]
    n = 10
    ly = np.array([np.sin(x + (n + j) * dt) for j in range(1, p["k"] + 1)])
    lz = np.array([np.cos(x + (n + j) * dt) for j in range(1, p["k"] + 1)])
    idx = np.arange(400, 1201, 50)
    e = O.expectations(p, n, ly, lz, idx)
    for j in range(1, p["k"] + 1):
        ez, eyw = e[:, j - 1, 0], e[:, j - 1, 4]
        assert np.max(np.abs(eyw - j * dt * ez)) < 1e-10
        # and E[y] is the heat semigroup applied to sin(x + t): exp(-j dt/2) sin
        ey = e[:, j - 1, 3]
        assert np.max(np.abs(ey - np.exp(-j * dt / 2) * np.sin(x[idx] + (n + j) * dt))) < 1e-10


def test_price_independent_of_mu():
    """The call price does not depend on mu (it enters the forward drift and
    the driver and cancels): two mu values give the same y0 to discretisation
    accuracy."""
    base = W.call_problem(Nx=2049, N=64, k=3, L=16)
    p2 = W.call_problem(Nx=2049, N=64, k=3, L=16, mu=0.10)
    r1 = O.solve(base, threads=THREADS)
    r2 = O.solve(p2, threads=THREADS)
    exact = O.exact(base, 0.0, base["x0"])
    # a mistake in how mu enters (drift or driver alone) moves y0 by O(1e-1)
    assert abs(r1["y0"] - r2["y0"]) < 1e-4
    assert abs(r1["y0"] - exact[0]) < 1e-4 and abs(r2["y0"] - exact[0]) < 1e-4


def test_invalid_problems_rejected():
    for bad in (dict(k=7), dict(k=5, N=4), dict(Nx=3), dict(L=0)):
        p = W.sin_problem()
        p.update(bad)
        with pytest.raises(ValueError):
            O.solve(p)


def test_partial_levels_sample():
    """levels=m stops after m backward levels; the readout is of that level."""
    p = W.sin_problem(N=16, k=2)
    full = O.solve(p)
    part = O.solve(p, levels=3)
    assert part["levels_done"] == 3 and full["levels_done"] == 15
    assert part["y0"] != full["y0"]
