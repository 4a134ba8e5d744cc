"""Seeded synthetic workloads: problem parameters and closed-form input data.

These generators describe *what* is solved (drivers, terminal conditions,
domains, grid sizes, seeded parameter draws, the exact initial levels as host
input); they contain none of the scheme's arithmetic.  Both the CUDA path and the CPU oracle consume the same
dicts.  No dataset is involved anywhere: the paper's examples are analytic
BSDEs (Section 5) and every workload here is defined by closed-form data.

Problem dict keys
-----------------
driver      "LIN_SIN" | "BS" | "LB" | "EX1" | "EX2"
terminal    "SIN" | "CALL_LOG" | "LOGISTIC" | "LNSIN"
T, x_min, x_max, x0        time horizon, uniform grid [x_min, x_max], readout point
a_x, b_x    forward process dX = a_x dt + b_x dW (X = W: 0, 1;
            log price, Eq. 33: mu - sigma^2/2, sigma)
r, mu, sigma, R, delta, lb_sign, strike   driver / payoff parameters
Nx, N, k, L                 grid points, time steps, steps of the scheme, GH nodes
picard_tol, picard_max, smoothing
"""
from __future__ import annotations

import math

import numpy as np


def sin_problem(Nx: int = 2001, N: int = 64, k: int = 2, L: int = 8,
                x_lim: float = 8.0, T: float = 1.0) -> dict:
    """1-D linear BSDE f = y/2 - z, g(x) = sin(x + T), X = W; exact
    y = sin(W_t + t), z = cos(W_t + t), so (y_0, z_0) = (0, 1)."""
    return dict(driver="LIN_SIN", terminal="SIN", T=T, x_min=-x_lim, x_max=x_lim,
                x0=0.0, a_x=0.0, b_x=1.0, Nx=Nx, N=N, k=k, L=L,
                picard_tol=1e-12, picard_max=30, smoothing=0)


def call_problem(S0: float = 100.0, strike: float = 100.0, r: float = 0.03,
                 mu: float = 0.05, sigma: float = 0.2, T: float = 1.0,
                 delta: float = 0.0, Nx: int = 65536, N: int = 256, k: int = 6,
                 L: int = 16, width_sd: float = 6.0, smoothing: int = 1,
                 driver: str = "BS", R: float = 0.0, lb_sign: float = 1.0) -> dict:
    """European call as a linear (BS) or lending/borrowing-rate (LB) BSDE in
    log price X = ln S (Eq. 30, Eq. 33); grid ln S0 +- width_sd*sigma*sqrt(T)."""
    x0 = math.log(S0)
    half = width_sd * sigma * math.sqrt(T)
    return dict(driver=driver, terminal="CALL_LOG", T=T, x_min=x0 - half,
                x_max=x0 + half, x0=x0, a_x=mu - 0.5 * sigma * sigma, b_x=sigma,
                r=r, mu=mu, sigma=sigma, R=R, delta=delta, lb_sign=lb_sign,
                strike=strike, Nx=Nx, N=N, k=k, L=L, picard_tol=1e-12,
                picard_max=30, smoothing=smoothing)


def ex1_problem(Nx: int = 4097, N: int = 128, k: int = 3, L: int = 32,
                x_lim: float = 16.0) -> dict:
    """Example 1 (Eq. 22-23): exact (y_0, z_0) = (1/2, 1/4)."""
    return dict(driver="EX1", terminal="LOGISTIC", T=1.0, x_min=-x_lim, x_max=x_lim,
                x0=0.0, a_x=0.0, b_x=1.0, Nx=Nx, N=N, k=k, L=L,
                picard_tol=1e-12, picard_max=30, smoothing=0)


def ex2_problem(Nx: int = 4097, N: int = 128, k: int = 3, L: int = 32,
                x_lim: float = 16.0) -> dict:
    """Example 2 (Eq. 24-25): exact (y_0, z_0) = (ln 3, 1/3)."""
    return dict(driver="EX2", terminal="LNSIN", T=1.0, x_min=-x_lim, x_max=x_lim,
                x0=0.0, a_x=0.0, b_x=1.0, Nx=Nx, N=N, k=k, L=L,
                picard_tol=1e-12, picard_max=30, smoothing=0)


# --- the five benchmark configurations -------------------------------------

def config1() -> dict:
    """sin driver, x in [-8, 8], Nx = 2001, N = 64, k = 2, L = 8, FP64."""
    return sin_problem()


def config2(k: int = 6) -> dict:
    """Black-Scholes call in log price, S0 = K = 100, r = .03, mu = .05,
    sigma = .2, T = 1, domain +-6 sigma sqrt(T), Nx = 65536, N = 256, L = 16."""
    return call_problem(k=k)


def config3(Nx: int = 1 << 20, N: int = 1024, k: int = 4) -> dict:
    """Call with different lending/borrowing rates r = .04, R = .06,
    mu = .06, sigma = .2, T = .5, K = 100, Nx = 2^20, N = 1024, k = 4, L = 16."""
    return call_problem(r=0.04, R=0.06, mu=0.06, sigma=0.2, T=0.5, Nx=Nx, N=N,
                        k=k, driver="LB", lb_sign=1.0)


def config4(count: int = 4096, seed: int = 13560) -> list:
    """Batch of Black-Scholes calls: K ~ U[70,130], sigma ~ U[.1,.5],
    T ~ U[.25,2], r ~ U[0,.05], Nx in {2^10..2^14}, N in {32,64,128,256},
    k ~ U{1..6}, L = 16, S0 = 100, mu = .05."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(call_problem(
            strike=float(rng.uniform(70, 130)), sigma=float(rng.uniform(0.1, 0.5)),
            T=float(rng.uniform(0.25, 2.0)), r=float(rng.uniform(0.0, 0.05)),
            Nx=int(1 << int(rng.integers(10, 15))),
            N=int(32 << int(rng.integers(0, 4))),
            k=int(rng.integers(1, 7)), L=16))
    return out


def config5_arrivals(rate: float = 2000.0, duration: float = 10.0,
                     seed: int = 1909) -> list:
    """Poisson arrivals of pricing solves: 70% Black-Scholes (Nx = 2^12,
    N = 64, k = 3), 30% lending/borrowing calls (Nx = 2^16, N = 256, k = 4),
    L = 16, parameters drawn as in config4.  Returns (t_arrival, problem)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        strike = float(rng.uniform(70, 130))
        sigma = float(rng.uniform(0.1, 0.5))
        T = float(rng.uniform(0.25, 2.0))
        r = float(rng.uniform(0.0, 0.05))
        if rng.uniform() < 0.7:
            p = call_problem(strike=strike, sigma=sigma, T=T, r=r, Nx=1 << 12, N=64,
                             k=3, L=16)
        else:
            p = call_problem(strike=strike, sigma=sigma, T=T, r=r, R=r + 0.02,
                             mu=0.06, Nx=1 << 16, N=256, k=4, L=16, driver="LB")
        out.append((t, p))
    return out


def levels_K(p: dict) -> int:
    """K = max(K_y, K_z) (Eq. 16): initial levels, and levels read per step."""
    return max(int(p["k"]), int(p.get("kz", 0)) or int(p["k"]))


def gp_steps(p: dict) -> int:
    """Grid-point time steps of one solve: Nx * (N - K + 1) levels computed
    (the one-step start-up, when asked for, is not counted)."""
    return int(p["Nx"]) * (int(p["N"]) - levels_K(p) + 1)


def initial_levels(p: dict):
    """Host arrays (K, Nx) of the K initial levels N, N-1, ..., N-K+1 from the
    closed-form solution of the problem (the exact start), with the level-N
    call payoff replaced by its cell average when smoothing is on.  This is
    input data for callers that pass their own levels through host memory."""
    from scipy.special import ndtr
    k, Nx, N = levels_K(p), int(p["Nx"]), int(p["N"])
    dx = (p["x_max"] - p["x_min"]) / (Nx - 1)
    x = p["x_min"] + dx * np.arange(Nx)
    dt = p["T"] / N
    ys, zs = np.zeros((k, Nx)), np.zeros((k, Nx))
    for m in range(k):
        t = (N - m) * dt
        term = p["terminal"]
        if term == "SIN":
            u, ux = np.sin(x + t), np.cos(x + t)
        elif term == "LOGISTIC":
            e = np.exp(x + t)
            u, ux = e / (e + 1), e / (e + 1) ** 2
        elif term == "LNSIN":
            e = math.exp(t * t)
            u, ux = np.log(np.sin(x) + 3) * e, e * np.cos(x) / (np.sin(x) + 3)
        elif term == "ONE":
            u, ux = vasicek_bond(p, t, x)
        elif term == "CALL_PRICE":
            u, ux = price_call(p, t, x, smooth=(m == 0 and bool(p.get("smoothing", 0))))
        else:
            K = p["strike"]
            if m == 0 and p.get("smoothing", 0):
                a, b, kap = x - dx / 2, x + dx / 2, math.log(K)
                ea = np.exp(a) * np.expm1(b - a) / dx
                d = np.clip(b - kap, 0.0, None)
                mid = K * (np.expm1(d) - d) / dx
                u = np.where(b <= kap, 0.0, np.where(a >= kap, ea - K, mid))
                ux = np.where(b <= kap, 0.0, np.where(a >= kap, ea, K * np.expm1(d) / dx))
            else:
                r, dl = p.get("r", 0.0), p.get("delta", 0.0)
                if p["driver"] == "LB":
                    r, dl = r - p.get("lb_sign", 1.0) * (p["R"] - r), 0.0
                S, tau, sig = np.exp(x), p["T"] - t, p["sigma"]
                if tau <= 0:
                    u, ux = np.maximum(S - K, 0.0), np.where(S > K, S, 0.0)
                else:
                    sq = sig * math.sqrt(tau)
                    d1 = (np.log(S / K) + (r - dl + 0.5 * sig * sig) * tau) / sq
                    a = S * math.exp(-dl * tau) * ndtr(d1)
                    u, ux = a - K * math.exp(-r * tau) * ndtr(d1 - sq), a
        bx = p["b_x"] + (p.get("b_1", 0.0) * x if p.get("forward", "CONST") == "AFFINE" else 0.0)
        ys[m], zs[m] = u, bx * ux
        if term == "CALL_PRICE" and m == 0 and p.get("smoothing", 0):
            zs[m] = price_call_z_average(p, x)
    return ys, zs


def vasicek_bond(p: dict, t: float, x):
    """Zero-coupon bond price A(tau) exp(-B(tau) x) and its x-derivative under
    dX = kappa (theta - X) dt + sigma dW (kappa = -a_1, theta = a_x / kappa,
    sigma = b_x)."""
    tau = p["T"] - t
    x = np.asarray(x, dtype=np.float64)
    if tau <= 0:
        return np.ones_like(x), np.zeros_like(x)
    kap = -p["a_1"]
    th, sg = p["a_x"] / kap, p["b_x"]
    B = -math.expm1(-kap * tau) / kap
    lnA = (th - sg * sg / (2 * kap * kap)) * (B - tau) - sg * sg * B * B / (4 * kap)
    u = np.exp(lnA - B * x)
    return u, -B * u


def price_call(p: dict, t: float, x, smooth: bool = False):
    """Black-Scholes call in the price x = S (volatility b_1) and its
    x-derivative; with smooth, the level-N cell averages of the payoff over
    [x - dx/2, x + dx/2]."""
    from scipy.special import ndtr
    x = np.asarray(x, dtype=np.float64)
    K, tau, sg = p["strike"], p["T"] - t, p["b_1"]
    r, dl = p.get("r", 0.0), p.get("delta", 0.0)
    if smooth:
        dx = (p["x_max"] - p["x_min"]) / (int(p["Nx"]) - 1)
        a, b = x - dx / 2, x + dx / 2
        lo = np.maximum(a, K)
        u = np.where(b <= K, 0.0, 0.5 * ((b - K) ** 2 - (lo - K) ** 2) / dx)
        return u, np.zeros_like(x)
    if tau <= 0:
        return np.maximum(x - K, 0.0), (x > K).astype(np.float64)
    sq = sg * math.sqrt(tau)
    with np.errstate(divide="ignore"):
        d1 = (np.log(np.maximum(x, 1e-300) / K) + (r - dl + 0.5 * sg * sg) * tau) / sq
    u = x * math.exp(-dl * tau) * ndtr(d1) - K * math.exp(-r * tau) * ndtr(d1 - sq)
    return np.where(x > 0, u, 0.0), np.where(x > 0, math.exp(-dl * tau) * ndtr(d1), 0.0)


def price_call_z_average(p: dict, x):
    """Level-N cell average of b(s) 1{s > K}, b(s) = b_x + b_1 s."""
    dx = (p["x_max"] - p["x_min"]) / (int(p["Nx"]) - 1)
    K = p["strike"]
    a, b = x - dx / 2, x + dx / 2
    lo = np.maximum(a, K)
    z = (p["b_x"] * (b - lo) + 0.5 * p["b_1"] * (b * b - lo * lo)) / dx
    return np.where(b <= K, 0.0, z)


# --- two space dimensions (Section 5, Examples 4 and 5) ----------------------

def ex4_problem(M: int = 128, N: int = 8, k: int = 3, L: int = 8, x_lim: float = 8.0) -> dict:
    """Example 4 (Eq. 34-35): f = y - z A, A = (1/2, 1/2)^T, g = sin(x1 + x2 + T),
    X = W in two dimensions, x in [-x_lim, x_lim]^2 with M intervals per
    dimension; exact (y_0, z_0) = (0, (1, 1))."""
    return dict(driver="LINEAR", terminal="SIN_SUM", T=1.0,
                x1_min=-x_lim, x1_max=x_lim, x2_min=-x_lim, x2_max=x_lim, x01=0.0, x02=0.0,
                a1=0.0, a2=0.0, b11=1.0, b21=0.0, b22=1.0,
                alpha=1.0, beta1=-0.5, beta2=-0.5,
                Nx1=M + 1, Nx2=M + 1, N=N, k=k, L=L, picard_max=30, picard_tol=1e-12)


def ex5_problem(M: int = 128, N: int = 8, k: int = 3, L: int = 8, width: float = 8.0,
                S0=(100.0, 100.0), sigma=(0.25, 0.3), rho: float = 0.0, r: float = 0.05,
                mu=(0.1, 0.1), T: float = 1.0) -> dict:
    """Example 5 (Eq. 36-37): zero-strike spread option (S1 - S2)^+ in log
    prices x = ln S, dX = (mu - sigma^2/2) dt + A dW with A the Cholesky factor
    [[s1, 0], [rho s2, s2 sqrt(1 - rho^2)]], f = -(r y + z A^{-1} M^T),
    M = mu - r; x in ln S0 +- width with M intervals per dimension.  T = 1:
    the paper's printed solution (15.48076, (14.4350, -12.6779)) is the
    Margrabe value at T = 1, which its text states as 0.1."""
    s1, s2 = sigma
    b11, b21, b22 = s1, rho * s2, s2 * math.sqrt(1.0 - rho * rho)
    m1, m2 = mu[0] - r, mu[1] - r
    # theta = A^{-1} M^T (A lower triangular)
    th1 = m1 / b11
    th2 = (m2 - b21 * th1) / b22
    c1, c2 = math.log(S0[0]), math.log(S0[1])
    return dict(driver="LINEAR", terminal="SPREAD_LOG", T=T,
                x1_min=c1 - width, x1_max=c1 + width, x2_min=c2 - width, x2_max=c2 + width,
                x01=c1, x02=c2, a1=mu[0] - 0.5 * s1 * s1, a2=mu[1] - 0.5 * s2 * s2,
                b11=b11, b21=b21, b22=b22, alpha=-r, beta1=-th1, beta2=-th2,
                Nx1=M + 1, Nx2=M + 1, N=N, k=k, L=L, picard_max=30, picard_tol=1e-12)


# --- general forward processes (Euler; Section 1's general Markovian X) -----

def vasicek_problem(kappa: float = 0.8, theta: float = 0.04, sigma: float = 0.02,
                    r0: float = 0.03, T: float = 2.0, Nx: int = 2049, N: int = 64, k: int = 3,
                    L: int = 16, width_sd: float = 8.0) -> dict:
    """Zero-coupon bond under the Vasicek short rate dX = kappa (theta - X) dt
    + sigma dW: f = -x y, g = 1, forward AFFINE (a(x) = kappa theta - kappa x,
    b = sigma); closed form A(tau) exp(-B(tau) x).  Grid: theta +- width_sd
    times the stationary standard deviation sigma / sqrt(2 kappa), widened to
    contain r0."""
    sd = sigma / math.sqrt(2.0 * kappa)
    lo, hi = min(theta, r0) - width_sd * sd, max(theta, r0) + width_sd * sd
    return dict(driver="SHORT_RATE", terminal="ONE", forward="AFFINE", T=T,
                x_min=lo, x_max=hi, x0=r0, a_x=kappa * theta, a_1=-kappa, b_x=sigma, b_1=0.0,
                Nx=Nx, N=N, k=k, L=L, smoothing=0, picard_max=30, picard_tol=1e-12)


def gbm_call_problem(S0: float = 100.0, strike: float = 100.0, r: float = 0.03,
                     mu: float = 0.05, sigma: float = 0.2, T: float = 1.0, Nx: int = 4097,
                     N: int = 64, k: int = 3, L: int = 16, width_sd: float = 6.0,
                     smoothing: int = 1) -> dict:
    """Black-Scholes call with the stock price itself as the grid variable:
    dS = mu S dt + sigma S dW (forward AFFINE with a(x) = mu x, b(x) = sigma x,
    advanced by Euler), f = -(r y + (mu - r) z / sigma), g = (x - K)^+.
    Grid: S0 exp(+-width_sd sigma sqrt(T)) (price space, positive)."""
    w = width_sd * sigma * math.sqrt(T)
    return dict(driver="BS", terminal="CALL_PRICE", forward="AFFINE", T=T,
                x_min=S0 * math.exp(-w), x_max=S0 * math.exp(w), x0=S0,
                a_x=0.0, a_1=mu, b_x=0.0, b_1=sigma, r=r, mu=mu, sigma=sigma, delta=0.0,
                strike=strike, Nx=Nx, N=N, k=k, L=L, smoothing=smoothing, picard_max=30,
                picard_tol=1e-12)
