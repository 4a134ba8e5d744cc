"""Two more pins of the FP64 oracle.

* The Picard fixed point for a linear driver (the scheme's implicit y-step,
  Eq. 20 first line) has a closed form: with space-independent data and the
  Black-Scholes driver f = -r y - theta z the step is a scalar division.
* Brute force at 50 significant digits on tiny inputs: the whole scheme of
  Eq. 20-21 (Gauss-Hermite nodes as roots of H_L, natural cubic spline by a
  dense solve, the expectations and both equations of Eq. 20 with the exact
  implicit step) written out again with mpmath and compared with the oracle's
  level 0.  Only the rounding of the oracle (and its Picard stopping rule)
  may differ.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_13560_gb300 import workloads as W
from test_oracle_pins import _gamma_exact


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_picard_fixed_point_of_a_linear_driver(k):
    p = W.call_problem(Nx=33, N=20, k=k, L=6)
    dt = p["T"] / p["N"]
    r = p["r"]
    c = [0.7 + 0.11 * m for m in range(k)]  # level N - m
    iy = np.array([[c[m]] * p["Nx"] for m in range(k)])
    iz = np.zeros((k, p["Nx"]))
    got = O.solve(p, iy, iz, want_level=True)
    gy, _ = _gamma_exact(k)
    gy = [float(g) for g in gy]
    y = {p["N"] - m: c[m] for m in range(k)}
    for n in range(p["N"] - k, -1, -1):
        A = y[n + k] + k * dt * sum(gy[j] * (-r * y[n + j]) for j in range(1, k + 1))
        y[n] = A / (1.0 + k * dt * gy[0] * r)  # y = A + k dt g0 (-r y), solved
    assert np.max(np.abs(got["y"] - y[0])) < 1e-13
    assert np.max(np.abs(got["z"])) < 1e-13


def _mp_scheme(k, Nx, N, L, x_lim, T, mp, kz=None, zform=0, start=None, stop=0,
               return_all=False, general=None):
    """Eq. 20-21 for f = y/2 - z, g = sin(x + T), X = W, at mp precision, with
    K_y = k and K_z = kz (default k; Eq. 16: K = max(K_y, K_z) levels), the
    z line's first term E[z^{n+1}] or (zform) E[y^{n+1} DeltaW_1] / dt, and
    the K initial levels from `start` ({level: (ys, zs)}) or the closed form.
    Runs levels N-K down to `stop`; returns level `stop` (y, z) at the grid
    points, or every level ({level: (ys, zs)}) with return_all.
    general = (a0, a1, b0, b1): the forward process advanced by one Euler step,
    X = x + (a0 + a1 x) j dt + (b0 + b1 x) DeltaW, with the short-rate driver
    f = -X y (implicit step y = A / (1 + k dt gy_0 x))."""
    kz = k if kz is None else kz
    K = max(k, kz)
    dt = mp.mpf(T) / N
    xs = [mp.mpf(-x_lim) + 2 * mp.mpf(x_lim) * i / (Nx - 1) for i in range(Nx)]
    dx = xs[1] - xs[0]
    # Gauss-Hermite: roots of the physicists' H_L, weights
    # 2^(L-1) L! sqrt(pi) / (L^2 H_{L-1}(a)^2)
    def herm(n, x):
        h0, h1 = mp.mpf(1), 2 * x
        if n == 0:
            return h0
        for m in range(1, n):
            h0, h1 = h1, 2 * x * h1 - 2 * m * h0
        return h1
    coef = [mp.mpf(0)] * (L + 1)  # H_L coefficients, highest first
    hc = [[mp.mpf(1)], [mp.mpf(2), mp.mpf(0)]]
    for m in range(1, L):
        a, b = hc[-1], hc[-2]
        nxt = [2 * v for v in a] + [mp.mpf(0)]
        bb = [mp.mpf(0)] * (len(nxt) - len(b)) + b
        hc.append([u - 2 * m * v for u, v in zip(nxt, bb)])
    nodes = sorted(mp.re(z) for z in mp.polyroots(hc[L], maxsteps=200, extraprec=200))
    wts = [2 ** (L - 1) * mp.factorial(L) * mp.sqrt(mp.pi) / (L * L * herm(L - 1, a) ** 2)
           for a in nodes]
    gy, _ = _gamma_exact(k)
    _, gz = _gamma_exact(kz)
    gy = [mp.mpf(g.numerator) / g.denominator for g in gy]
    gz = [mp.mpf(g.numerator) / g.denominator for g in gz]

    def second_derivs(v):
        # natural spline: M_0 = M_{Nx-1} = 0, M_{i-1} + 4 M_i + M_{i+1} = 6 (v_{i-1} - 2 v_i + v_{i+1}) / dx^2
        n = Nx - 2
        A = mp.matrix(n, n)
        rhs = mp.matrix(n, 1)
        for i in range(n):
            A[i, i] = 4
            if i > 0:
                A[i, i - 1] = 1
            if i < n - 1:
                A[i, i + 1] = 1
            rhs[i] = 6 * (v[i] - 2 * v[i + 1] + v[i + 2]) / dx ** 2
        sol = mp.lu_solve(A, rhs)
        return [mp.mpf(0)] + [sol[i] for i in range(n)] + [mp.mpf(0)]

    def interp(v, M, X):
        if X <= xs[0]:
            return v[0]
        if X >= xs[-1]:
            return v[-1]
        s = (X - xs[0]) / dx
        c = min(int(mp.floor(s)), Nx - 2)
        th = s - c
        om = 1 - th
        return (om * v[c] + th * v[c + 1]
                + dx ** 2 / 6 * ((om ** 3 - om) * M[c] + (th ** 3 - th) * M[c + 1]))

    lev = {}
    for m in range(K):
        t = (N - m) * dt
        if start is not None:
            lev[N - m] = start[N - m]
        else:
            lev[N - m] = ([mp.sin(x + t) for x in xs], [mp.cos(x + t) for x in xs])
    spl = {m: (second_derivs(lev[m][0]), second_derivs(lev[m][1])) for m in lev}
    rpi = 1 / mp.sqrt(mp.pi)
    for n in range(N - K, stop - 1, -1):
        ys, zs = [], []
        for x in xs:
            Ez, EFdW, EF, Ey, EyW1 = {}, {}, {}, mp.mpf(0), mp.mpf(0)
            for j in range(1, K + 1):
                vy, vz = lev[n + j]
                My, Mz = spl[n + j]
                ez = efdw = ef = mp.mpf(0)
                for a, w in zip(nodes, wts):
                    dW = mp.sqrt(2 * j * dt) * a
                    if general is None:
                        X = x + dW
                    else:
                        a0, a1, b0, b1 = general
                        X = x + (a0 + a1 * x) * j * dt + (b0 + b1 * x) * dW
                    yh = interp(vy, My, X)
                    zh = interp(vz, Mz, X)
                    F = yh / 2 - zh if general is None else -X * yh
                    ez += w * rpi * zh
                    efdw += w * rpi * F * dW
                    ef += w * rpi * F
                    if j == k:
                        Ey += w * rpi * yh
                    if j == 1:
                        EyW1 += w * rpi * yh * dW
                Ez[j], EFdW[j], EF[j] = ez, efdw, ef
            first = EyW1 / dt if zform else Ez[1]
            z = (first + sum(gz[j] * (EFdW[j] - Ez[j]) for j in range(1, kz + 1))) / gz[0]
            Ay = Ey + k * dt * sum(gy[j] * EF[j] for j in range(1, k + 1))
            if general is None:
                # y = Ay + k dt gy_0 (y/2 - z): the fixed point, exactly
                y = (Ay - k * dt * gy[0] * z) / (1 - k * dt * gy[0] / 2)
            else:
                # y = Ay + k dt gy_0 (-x y)
                y = Ay / (1 + k * dt * gy[0] * x)
            ys.append(y)
            zs.append(z)
        lev[n] = (ys, zs)
        spl[n] = (second_derivs(ys), second_derivs(zs))
    return lev if return_all else lev[stop]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_oracle_against_50_digit_scheme(k):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    Nx, N, L, x_lim, T = 17, 6, 4, 3.0, 1.0
    p = W.sin_problem(Nx=Nx, N=N, k=k, L=L, x_lim=x_lim, T=T)
    got = O.solve(p, want_level=True)
    ys, zs = _mp_scheme(k, Nx, N, L, x_lim, T, mp)
    ey = max(abs(float(a) - b) for a, b in zip(ys, got["y"]))
    ez = max(abs(float(a) - b) for a, b in zip(zs, got["z"]))
    # the oracle's Picard iteration stops once |dy| <= 1e-12 (contraction
    # k dt gy_0 / 2 < 0.15 here), and FP64 rounding is ~1e-15
    assert ey < 1e-12 and ez < 1e-12, (ey, ez)


@pytest.mark.parametrize("k,kz,zform", [(1, 2, 0), (2, 3, 0), (3, 1, 0), (1, 1, 1),
                                        (2, 2, 1), (1, 2, 1)])
def test_variants_against_50_digit_scheme(k, kz, zform):
    """K_z != K_y (Eq. 16) and the E[y DeltaW_1] / dt z form, brute force."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    Nx, N, L, x_lim, T = 17, 6, 4, 3.0, 1.0
    p = W.sin_problem(Nx=Nx, N=N, k=k, L=L, x_lim=x_lim, T=T)
    p.update(kz=kz, zform=zform)
    got = O.solve(p, want_level=True)
    ys, zs = _mp_scheme(k, Nx, N, L, x_lim, T, mp, kz=kz, zform=zform)
    ey = max(abs(float(a) - b) for a, b in zip(ys, got["y"]))
    ez = max(abs(float(a) - b) for a, b in zip(zs, got["z"]))
    assert ey < 1e-12 and ez < 1e-12, (ey, ez)


@pytest.mark.parametrize("k,kz,S", [(2, 2, 2), (3, 3, 1), (1, 3, 2)])
def test_onestep_startup_against_50_digit_scheme(k, kz, S):
    """Section 3.1 step 2: levels N-1..N-K+1 from the 1-step scheme with step
    dt / S, then the K-step loop; at 50 digits the start-up is the same
    scheme run on the finer time grid t = n' T / (N S)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    Nx, N, L, x_lim, T = 17, 6, 4, 3.0, 1.0
    K = max(k, kz)
    p = W.sin_problem(Nx=Nx, N=N, k=k, L=L, x_lim=x_lim, T=T)
    p.update(kz=kz, init_mode="ONESTEP", init_substeps=S)
    got = O.solve(p, want_level=True)
    fine = _mp_scheme(1, Nx, N * S, L, x_lim, T, mp, stop=N * S - (K - 1) * S,
                      return_all=True)
    start = {N - m: fine[(N - m) * S] for m in range(K)}
    ys, zs = _mp_scheme(k, Nx, N, L, x_lim, T, mp, kz=kz, start=start)
    ey = max(abs(float(a) - b) for a, b in zip(ys, got["y"]))
    ez = max(abs(float(a) - b) for a, b in zip(zs, got["z"]))
    assert ey < 1e-12 and ez < 1e-12, (ey, ez)


@pytest.mark.parametrize("k,kz,zform", [(1, 1, 1), (2, 1, 1), (2, 2, 0)])
def test_general_forward_against_50_digit_scheme(k, kz, zform):
    """The general forward path (affine a, b by one Euler step, the short-rate
    driver f = -x y), brute force, from the same smooth initial levels."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    Nx, N, L, x_lim, T = 17, 6, 4, 3.0, 1.0
    a0, a1, b0, b1 = "0.05", "-0.3", "0.2", "0.04"
    p = W.sin_problem(Nx=Nx, N=N, k=k, L=L, x_lim=x_lim, T=T)
    # Picard to rounding (the contraction k dt gy_0 |x| reaches 0.25 here, so
    # the default stop at |dy| <= 1e-12 would leave a few 1e-12)
    p.update(kz=kz, zform=zform, driver="SHORT_RATE", forward="AFFINE", a_x=float(a0),
             a_1=float(a1), b_x=float(b0), b_1=float(b1), picard_tol=1e-15)
    K = max(k, kz)
    xs = np.linspace(-x_lim, x_lim, Nx)
    dt = T / N
    iy = np.array([1.0 + 0.1 * np.sin(xs + (N - m) * dt) for m in range(K)])
    iz = np.array([0.05 * np.cos(xs - (N - m) * dt) for m in range(K)])
    got = O.solve(p, iy, iz, want_level=True)
    xm = [mp.mpf(-x_lim) + 2 * mp.mpf(x_lim) * i / (Nx - 1) for i in range(Nx)]
    start = {}
    for m in range(K):
        # the same doubles the oracle received
        start[N - m] = ([mp.mpf(float(v)) for v in iy[m]], [mp.mpf(float(v)) for v in iz[m]])
    ys, zs = _mp_scheme(k, Nx, N, L, x_lim, T, mp, kz=kz, zform=zform, start=start,
                        general=tuple(mp.mpf(v) for v in (a0, a1, b0, b1)))
    ey = max(abs(float(a) - b) for a, b in zip(ys, got["y"]))
    ez = max(abs(float(a) - b) for a, b in zip(zs, got["z"]))
    assert ey < 1e-12 and ez < 1e-12, (ey, ez)
