/*
 * Plain FP64 CPU oracle for the multistep BSDE scheme of Kapllani & Teng,
 * "Multistep schemes for solving backward stochastic differential equations
 * on GPU" (arXiv:1909.13560).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  The
 * product path never calls it and shares no code, header, table or constant
 * generator with it.
 *
 * Everything is IEEE double, compiled without FMA contraction, evaluated in
 * the order the paper states it:
 *   - uniform grid x_i = x_min + i*dx, dt = T/N            (Section 3.1 step 1,
 *                                                           Section 2.1)
 *   - Gauss-Hermite nodes/weights for exp(-a^2)            (Eq. 21)
 *   - multistep coefficients gamma (Tables 1 and 2; Eq. 20 writes them b)
 *   - natural cubic spline in space, exact tridiagonal solve (Section 3.3,
 *     "the matrix is tridiagonal"), constant extrapolation off the domain
 *     (Section 3.2 first remark), cell found by int((X-x_min)/dx)
 *     (Section 3.2 third remark)
 *   - per point and level: z explicitly, then y by Picard (Eq. 20, Section
 *     3.1 step 3, Section 3.3 last two items)
 *
 * Readings of points where the paper is silent (each also listed in the
 * design notes of the repository):
 *   - b == gamma in Eq. 20.  K_y = k and K_z = kz (kz = 0: K_z = k); the
 *     loop keeps K = max(K_y, K_z) levels (Eq. 16), y takes the K_y-step
 *     coefficients of Table 1 and E[y^{n+K_y}], z the K_z-step ones of
 *     Table 2.
 *   - z form: Eq. 20 as printed takes E[z^{n+1}]; with zform = 1 that term
 *     is E[y^{n+1} DeltaW_1] / dt instead, the quantity it stands for in the
 *     reference equation of z (Eq. 12 with l = 1).
 *   - natural spatial spline (M_0 = M_{Nx-1} = 0), solved exactly (Thomas).
 *   - Picard starts from y^{n+1}_i and stops when |y^(p+1)-y^(p)| <= tol or
 *     after picard_max iterations.
 *   - initial levels N..N-K+1 from the closed-form solution (init_mode 0)
 *     or, init_mode 1, level N from the closed form and levels N-1..N-K+1
 *     by the 1-step scheme (K_y = K_z = 1) run backward from t_N with the
 *     step dt / init_substeps (Section 3.1 step 2); the level-N call payoff
 *     is replaced by its cell average (smoothing, Section 5, Example 3).
 *     The caller may also pass the K initial levels explicitly.
 *   - forward process X with constant drift a_x and volatility b_x: the
 *     off-grid point for j steps and GH node a_l is x_i + a_x*j*dt +
 *     b_x*sqrt(2*j*dt)*a_l, while the Brownian increment weighting the
 *     z-expectations is DeltaW = sqrt(2*j*dt)*a_l (Eq. 21, Eq. 33).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- problem description (layout mirrored by oracle/oracle.py) ---------- */
enum { ORC_DRV_LIN_SIN = 0, ORC_DRV_BS = 1, ORC_DRV_LB = 2, ORC_DRV_EX1 = 3,
       ORC_DRV_EX2 = 4, ORC_DRV_SHORT_RATE = 5 };
enum { ORC_TERM_SIN = 0, ORC_TERM_CALL_LOG = 1, ORC_TERM_LOGISTIC = 2,
       ORC_TERM_LNSIN = 3, ORC_TERM_ONE = 4, ORC_TERM_CALL_PRICE = 5 };
enum { ORC_FWD_CONST = 0, ORC_FWD_AFFINE = 1 };

typedef struct {
  int driver, terminal, smoothing, picard_max;
  double T, x_min, x_max, x0;
  double a_x, b_x;                       /* forward X: dX = a_x dt + b_x dW */
  double r, mu, sigma, R, delta, lb_sign, strike;
  double picard_tol;
  long long Nx;
  int N, k, L;
  int kz;             /* K_z; 0 means K_z = k (= K_y)                        */
  int zform;          /* 0: E[z^{n+1}] in the z line (Eq. 20); 1: E[y DW]/dt */
  int init_mode;      /* 0: closed-form levels; 1: one-step start-up        */
  int init_substeps;  /* start-up steps per dt (init_mode 1)                */
  int forward;        /* 0: a_x, b_x constant; 1: a_x + a_1 x, b_x + b_1 x  */
  int pad_f;
  double a_1, b_1;
} orc_problem;

enum { ORC_INIT_EXACT = 0, ORC_INIT_ONESTEP = 1 };

static int orc_kz(const orc_problem *p) { return p->kz > 0 ? p->kz : p->k; }
/* K = max(K_y, K_z): the levels one step reads (Eq. 16) */
static int orc_K(const orc_problem *p) { return p->k > orc_kz(p) ? p->k : orc_kz(p); }

/* Coefficients of the forward process at x: constant, or affine in x (the
 * general Markovian X of Section 1, advanced by one Euler step over j dt). */
static double orc_fwd_a(const orc_problem *p, double x) {
  return p->forward == ORC_FWD_AFFINE ? p->a_x + p->a_1 * x : p->a_x;
}
static double orc_fwd_b(const orc_problem *p, double x) {
  return p->forward == ORC_FWD_AFFINE ? p->b_x + p->b_1 * x : p->b_x;
}

typedef struct {
  double y0, z0;
  double picard_resid_max;
  long long levels_done;
  int status;           /* 0 ok, 1 Picard did not converge somewhere, <0 bad */
  int picard_iters_max;
} orc_result;

static const double ORC_PI = 3.14159265358979323846;

/* ---- Gauss-Hermite rule for weight exp(-a^2) (Eq. 21) ------------------- */
/* Golub-Welsch: the nodes are the eigenvalues of the symmetric Jacobi
 * matrix of the orthonormal Hermite polynomials (zero diagonal, off-diagonal
 * sqrt(m/2)).  Eigenvalues by cyclic Jacobi rotations, each then polished by
 * Newton on p_L in long double, with p_L' = sqrt(2L) p_{L-1}.  Weights by the
 * Christoffel function w = 1 / sum_{m<L} p_m(a)^2. */
static void orc_hermite_orthonormal(long double a, int L, long double *pL,
                                    long double *pLm1, long double *sumsq) {
  long double pm1 = 0.0L;
  long double p = 1.0L / sqrtl(sqrtl((long double)ORC_PI));
  long double s = 0.0L;
  for (int m = 0; m < L; ++m) {
    s += p * p;
    long double pn = a * sqrtl(2.0L / (m + 1)) * p - sqrtl((long double)m / (m + 1)) * pm1;
    pm1 = p;
    p = pn;
  }
  *pL = p;
  *pLm1 = pm1;
  *sumsq = s;
}

int orc_gauss_hermite(int L, double *nodes, double *weights) {
  if (L < 1 || L > 128) return -1;
  double *A = (double *)calloc((size_t)L * L, sizeof(double));
  if (!A) return -2;
  for (int m = 1; m < L; ++m) {
    double b = sqrt(m / 2.0);
    A[(m - 1) * L + m] = b;
    A[m * L + (m - 1)] = b;
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < L; ++p)
      for (int q = p + 1; q < L; ++q) off += A[p * L + q] * A[p * L + q];
    if (off < 1e-300) break;
    for (int p = 0; p < L; ++p) {
      for (int q = p + 1; q < L; ++q) {
        double apq = A[p * L + q];
        if (fabs(apq) < 1e-300) continue;
        double theta = (A[q * L + q] - A[p * L + p]) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0);
        double s = t * c;
        for (int r = 0; r < L; ++r) {
          if (r == p || r == q) continue;
          double arp = A[r * L + p], arq = A[r * L + q];
          double nrp = c * arp - s * arq;
          double nrq = s * arp + c * arq;
          A[r * L + p] = A[p * L + r] = nrp;
          A[r * L + q] = A[q * L + r] = nrq;
        }
        A[p * L + p] -= t * apq;
        A[q * L + q] += t * apq;
        A[p * L + q] = A[q * L + p] = 0.0;
      }
    }
  }
  for (int m = 0; m < L; ++m) nodes[m] = A[m * L + m];
  free(A);
  /* ascending order (insertion sort; L is small) */
  for (int m = 1; m < L; ++m) {
    double v = nodes[m];
    int q = m - 1;
    while (q >= 0 && nodes[q] > v) { nodes[q + 1] = nodes[q]; --q; }
    nodes[q + 1] = v;
  }
  for (int m = 0; m < L; ++m) {
    long double a = nodes[m], pL, pLm1, s;
    for (int it = 0; it < 8; ++it) {
      orc_hermite_orthonormal(a, L, &pL, &pLm1, &s);
      long double d = sqrtl(2.0L * L) * pLm1;
      if (d == 0.0L) break;
      a -= pL / d;
    }
    orc_hermite_orthonormal(a, L, &pL, &pLm1, &s);
    nodes[m] = (double)a;
    weights[m] = (double)(1.0L / s);
  }
  /* the rule is symmetric: 0 is a node for odd L */
  if (L % 2 == 1) nodes[L / 2] = 0.0;
  return 0;
}

/* ---- multistep coefficients, Tables 1 and 2 (exact rationals) ----------- */
static const int ORC_GY_NUM[6][7] = {
    {1, 1}, {1, 2, 1}, {1, 3, 3, 1}, {1, 1, 1, 1, 1},
    {41, 19, 107, 107, 19, 41}, {19, 3, 15, 4, 15, 3, 19}};
static const int ORC_GY_DEN[6][7] = {
    {2, 2}, {6, 3, 6}, {8, 8, 8, 8}, {12, 3, 6, 3, 12},
    {600, 75, 600, 600, 75, 600}, {336, 14, 112, 21, 112, 14, 336}};
static const int ORC_GZ_NUM[6][7] = {
    {1, 1}, {5, 2, -1}, {3, 19, -5, 1}, {35, 5, -13, 1, -1},
    {131, 151, -103, 37, -1, 1}, {163, 47, -129, 3, -37, 1, -1}};
static const int ORC_GZ_DEN[6][7] = {
    {2, 2}, {12, 3, 12}, {8, 24, 24, 24}, {96, 6, 48, 12, 96},
    {360, 180, 360, 360, 45, 360}, {448, 56, 448, 28, 1344, 168, 1344}};

/* gamma^K_{K,j} (Table 1) into gy[0..K], gamma^1_{K,j} (Table 2) into gz. */
int orc_gamma(int K, double *gy, double *gz) {
  if (K < 1 || K > 6) return -1;
  for (int j = 0; j <= K; ++j) {
    gy[j] = (double)ORC_GY_NUM[K - 1][j] / (double)ORC_GY_DEN[K - 1][j];
    gz[j] = (double)ORC_GZ_NUM[K - 1][j] / (double)ORC_GZ_DEN[K - 1][j];
  }
  return 0;
}

/* ---- natural cubic spline on the uniform grid (Section 3.3) ------------- */
/* Second derivatives M with M_0 = M_{n-1} = 0 and, for 0<i<n-1,
 * M_{i-1} + 4 M_i + M_{i+1} = 6 (v_{i-1} - 2 v_i + v_{i+1}) / dx^2,
 * solved by the Thomas algorithm (exact LU of the tridiagonal matrix). */
int orc_spline(long long n, double dx, const double *v, double *M) {
  if (n < 2) return -1;
  M[0] = 0.0;
  M[n - 1] = 0.0;
  long long u = n - 2;
  if (u <= 0) return 0;
  double *d = (double *)malloc((size_t)u * sizeof(double));
  double *g = (double *)malloc((size_t)u * sizeof(double));
  if (!d || !g) { free(d); free(g); return -2; }
  for (long long q = 0; q < u; ++q) {
    double rhs = 6.0 * (v[q] - 2.0 * v[q + 1] + v[q + 2]) / (dx * dx);
    if (q == 0) {
      d[q] = 4.0;
      g[q] = rhs;
    } else {
      d[q] = 4.0 - 1.0 / d[q - 1];
      g[q] = rhs - g[q - 1] / d[q - 1];
    }
  }
  M[u] = g[u - 1] / d[u - 1];
  for (long long q = u - 2; q >= 0; --q) M[q + 1] = (g[q] - M[q + 2]) / d[q];
  free(d);
  free(g);
  return 0;
}

/* Spline value at X.  Off the domain: the boundary value (Section 3.2 first
 * remark).  Inside: cell c = int((X-x_min)/dx) (Section 3.2 third remark),
 * theta the position inside the cell, and the cubic spline formula in terms
 * of the nodal values and second derivatives. */
double orc_interp(long long n, double x_min, double dx, const double *v,
                  const double *M, double X) {
  double s = (X - x_min) / dx;
  if (s <= 0.0) return v[0];
  if (s >= (double)(n - 1)) return v[n - 1];
  long long c = (long long)floor(s);
  if (c > n - 2) c = n - 2;
  double th = s - (double)c;
  double om = 1.0 - th;
  return om * v[c] + th * v[c + 1] +
         (dx * dx / 6.0) * ((om * om * om - om) * M[c] + (th * th * th - th) * M[c + 1]);
}

/* ---- drivers f(t, y, z) ------------------------------------------------- */
/* LIN_SIN: one-dimensional analogue of Example 4 (Eq. 34-35): the linear
 *          driver f = y/2 - z, for which sin(W_t + t) solves the BSDE with
 *          g(x) = sin(x + T) (u_t + u_xx/2 + f = 0 holds exactly);
 * BS:      Eq. 29 with constant r, mu, sigma and dividend yield delta;
 * LB:      Eq. 29 plus the borrowing-rate term lb_sign*(R-r)*min(y - z/sigma, 0);
 * EX1:     Eq. 22;  EX2: Eq. 24;
 * SHORT_RATE: f = -x y, discounting at the short rate x (the forward
 *          state at the point where f is evaluated; the zero-coupon bond). */
double orc_driver(const orc_problem *p, double t, double x, double y, double z) {
  switch (p->driver) {
    case ORC_DRV_LIN_SIN:
      return 0.5 * y - z;
    case ORC_DRV_BS:
      return -(p->r * y + (p->mu - p->r + p->delta) * z / p->sigma);
    case ORC_DRV_LB: {
      double m = y - z / p->sigma;
      if (m > 0.0) m = 0.0;
      return -(p->r * y + (p->mu - p->r) * z / p->sigma) + p->lb_sign * (p->R - p->r) * m;
    }
    case ORC_DRV_EX1:
      return -y * y * y + 2.5 * y * y - 1.5 * y;
    case ORC_DRV_EX2: {
      double e = exp(t * t);
      return 0.5 * (e - 4.0 * t * y - 3.0 * exp(t * t - y * exp(-t * t)) + z * z * exp(-t * t));
    }
    case ORC_DRV_SHORT_RATE:
      return -x * y;
    default:
      return 0.0;
  }
}

/* ---- closed-form solutions u(t,x) and z = b(x) du/dx -------------------- */
static double orc_ncdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Black-Scholes call with dividend yield in log price x = ln S (Eq. 31 with
 * the standard dividend d_1; the printed d_1 omits -delta, the paper's own
 * numbers follow the standard form). */
static void orc_bs_call(double x, double tau, double r, double dlt, double sig,
                        double K, double *u, double *ux) {
  double S = exp(x);
  if (tau <= 0.0) {
    *u = S > K ? S - K : 0.0;
    *ux = S > K ? S : 0.0;
    return;
  }
  double sq = sig * sqrt(tau);
  double d1 = (log(S / K) + (r - dlt + 0.5 * sig * sig) * tau) / sq;
  double d2 = d1 - sq;
  double a = S * exp(-dlt * tau) * orc_ncdf(d1);
  *u = a - K * exp(-r * tau) * orc_ncdf(d2);
  *ux = a;
}

int orc_exact(const orc_problem *p, double t, double x, double *u, double *z) {
  double ux = 0.0;
  switch (p->terminal) {
    case ORC_TERM_SIN:  /* Eq. 35 restricted to one dimension */
      *u = sin(x + t);
      ux = cos(x + t);
      break;
    case ORC_TERM_CALL_LOG: {
      double r = p->r, dlt = p->delta;
      if (p->driver == ORC_DRV_LB) { r = p->r - p->lb_sign * (p->R - p->r); dlt = 0.0; }
      orc_bs_call(x, p->T - t, r, dlt, p->sigma, p->strike, u, &ux);
      break;
    }
    case ORC_TERM_LOGISTIC: { /* Eq. 23 */
      double e = exp(x + t);
      *u = e / (e + 1.0);
      ux = e / ((e + 1.0) * (e + 1.0));
      break;
    }
    case ORC_TERM_ONE: {
      /* zero-coupon bond under the Vasicek short rate dX = kappa (theta - X)
       * dt + sigma dW (forward AFFINE with a_1 = -kappa < 0, a_x = kappa
       * theta, b_1 = 0, sigma = b_x) and f = -x y:
       * P = exp(ln A - B x), B = (1 - e^{-kappa tau}) / kappa,
       * ln A = (theta - sigma^2 / (2 kappa^2)) (B - tau) - sigma^2 B^2 / (4 kappa) */
      double tau = p->T - t;
      if (tau <= 0.0) { *u = 1.0; ux = 0.0; break; }
      if (p->forward != ORC_FWD_AFFINE || !(p->a_1 < 0.0) || p->b_1 != 0.0) return -1;
      double kap = -p->a_1, th = p->a_x / kap, sg = p->b_x;
      double B = -expm1(-kap * tau) / kap;
      double lnA = (th - sg * sg / (2.0 * kap * kap)) * (B - tau) - sg * sg * B * B / (4.0 * kap);
      *u = exp(lnA - B * x);
      ux = -B * *u;
      break;
    }
    case ORC_TERM_CALL_PRICE: {
      /* call (x - K)^+ in the price x = S itself, geometric Brownian motion
       * dX = a_1 X dt + b_1 X dW: Black-Scholes with volatility b_1 and the
       * driver's rate and dividend yield */
      double r = p->r, dlt = p->delta, tau = p->T - t, sg = p->b_1, K = p->strike;
      if (p->driver == ORC_DRV_LB) { r = p->r - p->lb_sign * (p->R - p->r); dlt = 0.0; }
      if (x <= 0.0) { *u = 0.0; ux = 0.0; break; }
      if (tau <= 0.0) { *u = x > K ? x - K : 0.0; ux = x > K ? 1.0 : 0.0; break; }
      double sq = sg * sqrt(tau);
      double d1 = (log(x / K) + (r - dlt + 0.5 * sg * sg) * tau) / sq, d2 = d1 - sq;
      *u = x * exp(-dlt * tau) * orc_ncdf(d1) - K * exp(-r * tau) * orc_ncdf(d2);
      ux = exp(-dlt * tau) * orc_ncdf(d1);
      break;
    }
    case ORC_TERM_LNSIN: { /* Eq. 25 */
      double e = exp(t * t);
      *u = log(sin(x) + 3.0) * e;
      ux = e * cos(x) / (sin(x) + 3.0);
      break;
    }
    default:
      return -1;
  }
  *z = orc_fwd_b(p, x) * ux;
  return 0;
}

/* Cell average of the call payoff (e^x - K)^+ and of b_x * d/dx of it over
 * [x - dx/2, x + dx/2]: the smoothing of the non-smooth terminal value. */
static void orc_call_cell_average(double x, double dx, double K, double bx,
                                  double *u, double *z) {
  double a = x - 0.5 * dx, b = x + 0.5 * dx, kap = log(K);
  if (b <= kap) {
    *u = 0.0;
    *z = 0.0;
  } else if (a >= kap) {
    double ea = exp(a);
    *u = ea * expm1(b - a) / dx - K;
    *z = bx * ea * expm1(b - a) / dx;
  } else {
    double d = b - kap;
    *u = K * (expm1(d) - d) / dx;
    *z = bx * K * expm1(d) / dx;
  }
}

/* Cell average of the call payoff (s - K)^+ in the price and of b(s) times
 * its derivative, b(s) = b_x + b_1 s, over [x - dx/2, x + dx/2]. */
static void orc_call_price_cell_average(const orc_problem *p, double x, double dx,
                                        double *u, double *z) {
  double a = x - 0.5 * dx, b = x + 0.5 * dx, K = p->strike;
  if (b <= K) { *u = 0.0; *z = 0.0; return; }
  double lo = a > K ? a : K;
  /* int_lo^b (s - K) ds and int_lo^b (b_x + b_1 s) ds */
  *u = 0.5 * ((b - K) * (b - K) - (lo - K) * (lo - K)) / dx;
  *z = (p->b_x * (b - lo) + 0.5 * p->b_1 * (b * b - lo * lo)) / dx;
}

/* K initial levels: row m (0 <= m < K) holds level N-m (Section 3.1 step 2,
 * read as the closed form at t_{N-m}). */
int orc_init_levels(const orc_problem *p, double *init_y, double *init_z) {
  double dt = p->T / p->N;
  double dx = (p->x_max - p->x_min) / (double)(p->Nx - 1);
  for (int m = 0; m < orc_K(p); ++m) {
    double t = (p->N - m) * dt;
    for (long long i = 0; i < p->Nx; ++i) {
      double x = p->x_min + (double)i * dx, u, z;
      if (m == 0 && p->smoothing && p->terminal == ORC_TERM_CALL_LOG)
        orc_call_cell_average(x, dx, p->strike, p->b_x, &u, &z);
      else if (m == 0 && p->smoothing && p->terminal == ORC_TERM_CALL_PRICE)
        orc_call_price_cell_average(p, x, dx, &u, &z);
      else if (orc_exact(p, t, x, &u, &z) != 0)
        return -1;
      init_y[(size_t)m * p->Nx + i] = u;
      init_z[(size_t)m * p->Nx + i] = z;
    }
  }
  return 0;
}

static int orc_check(const orc_problem *p) {
  if (p->k < 1 || p->k > 6 || p->kz < 0 || p->kz > 6 || orc_K(p) > p->N) return -1;
  if (p->zform < 0 || p->zform > 1 || p->init_mode < 0 || p->init_mode > 1) return -1;
  if (p->init_mode == ORC_INIT_ONESTEP &&
      (p->init_substeps < 1 || (long long)p->N * p->init_substeps > (1LL << 30)))
    return -1;
  if (p->Nx < 4 || p->L < 1 || p->L > 128) return -1;
  if (!(p->x_max > p->x_min) || !(p->T > 0.0)) return -1;
  if (p->driver < 0 || p->driver > 5) return -1;
  if (p->terminal < 0 || p->terminal > 5) return -1;
  if (p->forward < 0 || p->forward > 1) return -1;
  return 0;
}

/* Gauss-Hermite estimates (Eq. 21) of the conditional expectations at grid
 * point i for j = 1..K, given levels n+1..n+K (row j-1 of ly/lz, second
 * derivatives in lmy/lmz).  out[5*(j-1) + q], q = 0..4:
 *   E_j[z^], E_j[f(t_{n+j}, y^, z^)], E_j[f * DeltaW_j], E_j[y^], E_j[y^ DeltaW_j]. */
static void orc_point_expectations(const orc_problem *p, int n, long long i,
                                   const double *const *ly, const double *const *lmy,
                                   const double *const *lz, const double *const *lmz,
                                   const double *gh_a, const double *gh_w,
                                   double *out) {
  double dt = p->T / p->N;
  double dx = (p->x_max - p->x_min) / (double)(p->Nx - 1);
  double xi = p->x_min + (double)i * dx;
  double rpi = 1.0 / sqrt(ORC_PI);
  for (int j = 1; j <= orc_K(p); ++j) {
    double tj = (n + j) * dt;
    double sq = sqrt(2.0 * j * dt);
    double ez = 0.0, ef = 0.0, efw = 0.0, ey = 0.0, eyw = 0.0;
    for (int l = 0; l < p->L; ++l) {
      double dW = sq * gh_a[l];
      /* one Euler step of the forward process over j dt (exact for
       * constant coefficients) */
      double X = xi + orc_fwd_a(p, xi) * j * dt + orc_fwd_b(p, xi) * dW;
      double yh = orc_interp(p->Nx, p->x_min, dx, ly[j - 1], lmy[j - 1], X);
      double zh = orc_interp(p->Nx, p->x_min, dx, lz[j - 1], lmz[j - 1], X);
      double F = orc_driver(p, tj, X, yh, zh);
      double w = gh_w[l] * rpi;
      ez += w * zh;
      ef += w * F;
      efw += w * F * dW;
      ey += w * yh;
      eyw += w * yh * dW;
    }
    out[5 * (j - 1) + 0] = ez;
    out[5 * (j - 1) + 1] = ef;
    out[5 * (j - 1) + 2] = efw;
    out[5 * (j - 1) + 3] = ey;
    out[5 * (j - 1) + 4] = eyw;
  }
}

/* Public wrapper: expectations at the points idx[0..cnt) for level n, the K
 * later levels given as rows of levels_y/levels_z (row j-1 = level n+j). */
int orc_expectations(const orc_problem *p, int n, const double *levels_y,
                     const double *levels_z, const long long *idx, long long cnt,
                     double *out) {
  if (orc_check(p)) return -1;
  int k = orc_K(p);
  long long nx = p->Nx;
  double dx = (p->x_max - p->x_min) / (double)(nx - 1);
  double *my = (double *)malloc((size_t)k * nx * sizeof(double));
  double *mz = (double *)malloc((size_t)k * nx * sizeof(double));
  double *a = (double *)malloc((size_t)p->L * sizeof(double));
  double *w = (double *)malloc((size_t)p->L * sizeof(double));
  const double *ly[6], *lz[6], *lmy[6], *lmz[6];
  if (!my || !mz || !a || !w) { free(my); free(mz); free(a); free(w); return -2; }
  orc_gauss_hermite(p->L, a, w);
  for (int j = 0; j < k; ++j) {
    orc_spline(nx, dx, levels_y + (size_t)j * nx, my + (size_t)j * nx);
    orc_spline(nx, dx, levels_z + (size_t)j * nx, mz + (size_t)j * nx);
    ly[j] = levels_y + (size_t)j * nx;
    lz[j] = levels_z + (size_t)j * nx;
    lmy[j] = my + (size_t)j * nx;
    lmz[j] = mz + (size_t)j * nx;
  }
  for (long long q = 0; q < cnt; ++q)
    orc_point_expectations(p, n, idx[q], ly, lmy, lz, lmz, a, w, out + (size_t)q * 5 * k);
  free(my); free(mz); free(a); free(w);
  return 0;
}

/* The backward loop (Eq. 20, Section 3.1 step 3).
 * init_y/init_z: K x Nx, row m = level N-m; NULL -> the problem's start
 *         (closed form, or the one-step start-up, orc_onestep_levels).
 * levels: how many backward levels to compute (n = N-K, N-K-1, ...);
 *         0 or more than N-K+1 -> all of them, down to n = 0.
 * out_y/out_z (optional, Nx each): the last computed level.
 * res: readout at x0 of the last computed level (Section 3.1 step 3 target
 *      (y_0^0, z_0^0)), Picard statistics (start-up included).
 * threads: OpenMP threads over grid points (1 = serial). */
int orc_onestep_levels(const orc_problem *p, double *init_y, double *init_z,
                       orc_result *stats, int threads);

int orc_solve(const orc_problem *p, const double *init_y, const double *init_z,
              long long levels, double *out_y, double *out_z, orc_result *res,
              int threads) {
  memset(res, 0, sizeof(*res));
  if (orc_check(p)) { res->status = -1; return -1; }
  const int ky = p->k, kz = orc_kz(p), K = orc_K(p), N = p->N;
  const long long nx = p->Nx;
  const double dt = p->T / N;
  const double dx = (p->x_max - p->x_min) / (double)(nx - 1);
  const int nslot = K + 1;
  double gy[7], gz[7], unused[7];
  orc_gamma(ky, gy, unused);  /* Table 1 row K_y */
  orc_gamma(kz, unused, gz);  /* Table 2 row K_z */
  double *gh_a = (double *)malloc((size_t)p->L * sizeof(double));
  double *gh_w = (double *)malloc((size_t)p->L * sizeof(double));
  double *Y = (double *)malloc((size_t)nslot * nx * sizeof(double));
  double *Z = (double *)malloc((size_t)nslot * nx * sizeof(double));
  double *MY = (double *)malloc((size_t)nslot * nx * sizeof(double));
  double *MZ = (double *)malloc((size_t)nslot * nx * sizeof(double));
  int *iters = (int *)malloc((size_t)nx * sizeof(int));
  double *resid = (double *)malloc((size_t)nx * sizeof(double));
  if (!gh_a || !gh_w || !Y || !Z || !MY || !MZ || !iters || !resid) {
    free(gh_a); free(gh_w); free(Y); free(Z); free(MY); free(MZ); free(iters); free(resid);
    res->status = -2;
    return -2;
  }
  orc_gauss_hermite(p->L, gh_a, gh_w);
  int itmax = 0;
  double rmax = 0.0;
  int nonconv = 0;

  /* level N-m lives in slot (N-m) mod (K+1) */
  if (init_y && init_z) {
    for (int m = 0; m < K; ++m) {
      memcpy(Y + (size_t)((N - m) % nslot) * nx, init_y + (size_t)m * nx, (size_t)nx * sizeof(double));
      memcpy(Z + (size_t)((N - m) % nslot) * nx, init_z + (size_t)m * nx, (size_t)nx * sizeof(double));
    }
  } else {
    double *iy = (double *)malloc((size_t)K * nx * sizeof(double));
    double *iz = (double *)malloc((size_t)K * nx * sizeof(double));
    orc_result st;
    memset(&st, 0, sizeof(st));
    int bad = !iy || !iz;
    if (!bad) {
      if (p->init_mode == ORC_INIT_ONESTEP)
        bad = orc_onestep_levels(p, iy, iz, &st, threads) != 0;
      else
        bad = orc_init_levels(p, iy, iz) != 0;
    }
    if (bad) {
      free(iy); free(iz);
      free(gh_a); free(gh_w); free(Y); free(Z); free(MY); free(MZ); free(iters); free(resid);
      res->status = -1;
      return -1;
    }
    itmax = st.picard_iters_max;
    rmax = st.picard_resid_max;
    nonconv = st.status == 1;
    for (int m = 0; m < K; ++m) {
      memcpy(Y + (size_t)((N - m) % nslot) * nx, iy + (size_t)m * nx, (size_t)nx * sizeof(double));
      memcpy(Z + (size_t)((N - m) % nslot) * nx, iz + (size_t)m * nx, (size_t)nx * sizeof(double));
    }
    free(iy);
    free(iz);
  }
  for (int m = 0; m < K; ++m) {
    size_t o = (size_t)((N - m) % nslot) * nx;
    orc_spline(nx, dx, Y + o, MY + o);
    orc_spline(nx, dx, Z + o, MZ + o);
  }

  long long total = (long long)(N - K + 1);
  if (levels <= 0 || levels > total) levels = total;
  int last = N - K + 1;

  for (long long lv = 0; lv < levels; ++lv) {
    const int n = N - K - (int)lv;
    const double *ly[6], *lz[6], *lmy[6], *lmz[6];
    for (int j = 1; j <= K; ++j) {
      size_t o = (size_t)((n + j) % nslot) * nx;
      ly[j - 1] = Y + o; lz[j - 1] = Z + o; lmy[j - 1] = MY + o; lmz[j - 1] = MZ + o;
    }
    double *yn = Y + (size_t)(n % nslot) * nx;
    double *zn = Z + (size_t)(n % nslot) * nx;
    const double *yprev = ly[0];
    const double tn = n * dt;
    const double h = ky * dt;

#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (long long i = 0; i < nx; ++i) {
      double e[30];
      orc_point_expectations(p, n, i, ly, lmy, lz, lmz, gh_a, gh_w, e);
      /* z: second line of Eq. 20 (K_z steps) solved for z^n; its first term
       * E[z^{n+1}], or E[y^{n+1} DeltaW_1] / dt in the zform reading */
      double sfw = 0.0, sz = 0.0;
      for (int j = 1; j <= kz; ++j) {
        sfw += gz[j] * e[5 * (j - 1) + 2];
        sz += gz[j] * e[5 * (j - 1) + 0];
      }
      double first = p->zform ? e[4] / dt : e[0];
      double z = (first + sfw - sz) / gz[0];
      /* y: first line of Eq. 20 (K_y steps), implicit in f(t_n, y^n, z^n),
       * by Picard */
      double sf = 0.0;
      for (int j = 1; j <= ky; ++j) sf += gy[j] * e[5 * (j - 1) + 1];
      double A = e[5 * (ky - 1) + 3] + h * sf;
      const double xi = p->x_min + (double)i * dx;
      double y = yprev[i];
      double d = 0.0;
      int it = 0;
      while (it < p->picard_max) {
        double yn1 = A + h * gy[0] * orc_driver(p, tn, xi, y, z);
        d = fabs(yn1 - y);
        y = yn1;
        ++it;
        if (d <= p->picard_tol) break;
      }
      yn[i] = y;
      zn[i] = z;
      iters[i] = it;
      resid[i] = d;
    }
    for (long long i = 0; i < nx; ++i) {
      if (iters[i] > itmax) itmax = iters[i];
      if (resid[i] > rmax) rmax = resid[i];
      if (resid[i] > p->picard_tol) nonconv = 1;
    }
    orc_spline(nx, dx, yn, MY + (size_t)(n % nslot) * nx);
    orc_spline(nx, dx, zn, MZ + (size_t)(n % nslot) * nx);
    last = n;
  }

  size_t o = (size_t)(last % nslot) * nx;
  res->y0 = orc_interp(nx, p->x_min, dx, Y + o, MY + o, p->x0);
  res->z0 = orc_interp(nx, p->x_min, dx, Z + o, MZ + o, p->x0);
  res->levels_done = levels;
  res->picard_iters_max = itmax;
  res->picard_resid_max = rmax;
  res->status = nonconv ? 1 : 0;
  if (out_y) memcpy(out_y, Y + o, (size_t)nx * sizeof(double));
  if (out_z) memcpy(out_z, Z + o, (size_t)nx * sizeof(double));
  free(gh_a); free(gh_w); free(Y); free(Z); free(MY); free(MZ); free(iters); free(resid);
  return 0;
}

/* The start-up of Section 3.1 step 2: level N from the closed form (smoothed
 * as the problem says), then the 1-step scheme (K_y = K_z = 1, Table 1 and 2
 * row 1) backward from t_N with the step h = dt / S, S = init_substeps, on the
 * same grid, Gauss-Hermite rule and z form; level N-m is its level after m S
 * steps, at t_N - m S h = t_{N-m}.  Rows m = 0..K-1 of init_y/init_z.  The
 * 1-step runs work on the time grid t = n' h, n' = 0..N S, so every driver
 * sees the same absolute times as the main loop.  stats (nullable) receives
 * the start-up's Picard statistics. */
int orc_onestep_levels(const orc_problem *p, double *init_y, double *init_z,
                       orc_result *stats, int threads) {
  if (orc_check(p) || p->init_substeps < 1) return -1;
  const int K = orc_K(p), S = p->init_substeps;
  const long long nx = p->Nx;
  orc_problem q = *p;
  q.k = 1;
  q.kz = 0;
  q.N = p->N * S;
  q.init_mode = ORC_INIT_EXACT;
  orc_result acc;
  memset(&acc, 0, sizeof(acc));
  if (orc_init_levels(&q, init_y, init_z) != 0) return -1;  /* row 0: level N */
  for (int m = 1; m < K; ++m) {
    orc_result r;
    if (orc_solve(&q, NULL, NULL, (long long)m * S, init_y + (size_t)m * nx,
                  init_z + (size_t)m * nx, &r, threads) != 0)
      return -1;
    if (r.picard_iters_max > acc.picard_iters_max) acc.picard_iters_max = r.picard_iters_max;
    if (r.picard_resid_max > acc.picard_resid_max) acc.picard_resid_max = r.picard_resid_max;
    if (r.status == 1) acc.status = 1;
  }
  if (stats) *stats = acc;
  return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
