/*
 * Plain FP64 CPU oracle for the two-dimensional multistep BSDE scheme of
 * Kapllani & Teng (arXiv:1909.13560): Eq. 20-21 with d = 2 (Section 3.3,
 * Examples 4 and 5).
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: the slow, plain definition the
 * CUDA path is checked against.  It shares no code with the product.
 *
 * Everything is IEEE double, compiled without FMA contraction:
 *   - grid x_{i1,i2} = (x1_min + i1 dx1, x2_min + i2 dx2), dt = T/N
 *   - Gauss-Hermite tensor rule: nodes (a_l1, a_l2), weights w_l1 w_l2 / pi,
 *     DeltaW = sqrt(2 j dt) (a_l1, a_l2)                       (Eq. 21)
 *   - forward X = x + a j dt + B DeltaW, B lower triangular (constant)
 *   - bicubic interpolation (Section 3.3): per cell the bicubic Hermite
 *     polynomial of the corner values, first derivatives and mixed
 *     derivative; the derivatives by fourth-order finite differences,
 *     central where the five-point stencil fits, forward at the first two
 *     nodes and backward at the last two of each line; mixed derivative =
 *     the x1 operator applied to the x2 derivative
 *   - off the domain the point is projected onto the box (the boundary
 *     values, Section 3.2); cell c = floor((X - min)/dx) clamped to
 *     [0, n-2], theta = position inside the cell
 *   - per point and level: z = (z1, z2) explicitly, then y by Picard
 *     (Eq. 20 with the row vector z and DeltaW^T)
 * Readings where the paper is silent are listed in the design notes; the
 * two that shape this file: the boundary projection above, and the
 * one-sided stencils at the first and last two nodes of each line.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC2_DRV_LINEAR = 0 };
enum { ORC2_TERM_SIN_SUM = 0, ORC2_TERM_SPREAD_LOG = 1 };

typedef struct {
  int driver, terminal, picard_max, pad;
  double T, x1_min, x1_max, x2_min, x2_max, x01, x02;
  double a1, a2, b11, b21, b22;        /* dX = a dt + B dW, B = [[b11,0],[b21,b22]] */
  double alpha, beta1, beta2;          /* f = alpha y + beta1 z1 + beta2 z2          */
  double picard_tol;
  long long Nx1, Nx2;
  int N, k, L, pad2;
} orc2_problem;

typedef struct {
  double y0, z0[2];
  double picard_resid_max;
  long long levels_done;
  int status;
  int picard_iters_max;
} orc2_result;

int orc_gauss_hermite(int L, double *nodes, double *weights); /* oracle.c */
int orc_gamma(int K, double *gy, double *gz);                 /* oracle.c */

static const double ORC2_PI = 3.14159265358979323846;

static int orc2_check(const orc2_problem *p) {
  if (p->k < 1 || p->k > 6 || p->k > p->N) return -1;
  if (p->Nx1 < 6 || p->Nx2 < 6 || p->L < 1 || p->L > 64) return -1;
  if (!(p->x1_max > p->x1_min) || !(p->x2_max > p->x2_min) || !(p->T > 0.0)) return -1;
  if (p->driver != ORC2_DRV_LINEAR) return -1;
  if (p->terminal < 0 || p->terminal > 1) return -1;
  return 0;
}

/* ---- fourth-order finite differences along one line ---------------------- */
/* d[i] ~ h f'(x_i) (scaled by the spacing) for a line of n >= 6 values with
 * stride s: central (f_{i-2} - 8 f_{i-1} + 8 f_{i+1} - f_{i+2}) / 12 where
 * it fits, forward (-25 f_i + 48 f_{i+1} - 36 f_{i+2} + 16 f_{i+3} - 3 f_{i+4}) / 12
 * at i = 0, 1 and its mirror image (backward) at i = n-2, n-1. */
static void orc2_fd_line(long long n, const double *f, long long s, double *d, long long ds) {
  for (long long i = 0; i < n; ++i) {
    double v;
    if (i >= 2 && i <= n - 3) {
      v = (f[(i - 2) * s] - 8.0 * f[(i - 1) * s] + 8.0 * f[(i + 1) * s] - f[(i + 2) * s]) / 12.0;
    } else if (i < 2) {
      v = (-25.0 * f[i * s] + 48.0 * f[(i + 1) * s] - 36.0 * f[(i + 2) * s] +
           16.0 * f[(i + 3) * s] - 3.0 * f[(i + 4) * s]) / 12.0;
    } else {
      v = (25.0 * f[i * s] - 48.0 * f[(i - 1) * s] + 36.0 * f[(i - 2) * s] -
           16.0 * f[(i - 3) * s] + 3.0 * f[(i - 4) * s]) / 12.0;
    }
    d[i * ds] = v;
  }
}

/* Scaled derivatives of a field v (index i1 + Nx1 i2): fx = dx1 dv/dx1,
 * fy = dx2 dv/dx2, fxy = dx1 dx2 d2v/dx1dx2 (x1 operator applied to fy). */
int orc2_derivatives(long long n1, long long n2, const double *v, double *fx, double *fy,
                     double *fxy) {
  if (n1 < 6 || n2 < 6) return -1;
  for (long long i2 = 0; i2 < n2; ++i2) orc2_fd_line(n1, v + i2 * n1, 1, fx + i2 * n1, 1);
  for (long long i1 = 0; i1 < n1; ++i1) orc2_fd_line(n2, v + i1, n1, fy + i1, n1);
  for (long long i2 = 0; i2 < n2; ++i2) orc2_fd_line(n1, fy + i2 * n1, 1, fxy + i2 * n1, 1);
  return 0;
}

/* ---- bicubic Hermite interpolation --------------------------------------- */
/* cubic Hermite basis on [0, 1]: value weights h00 (left), h01 (right),
 * slope weights h10 (left), h11 (right), slopes in units of the cell. */
static void orc2_hermite(double t, double *h00, double *h01, double *h10, double *h11) {
  double t2 = t * t, t3 = t2 * t;
  *h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
  *h01 = -2.0 * t3 + 3.0 * t2;
  *h10 = t3 - 2.0 * t2 + t;
  *h11 = t3 - t2;
}

static void orc2_locate(double X, double xmin, double xmax, double dx, long long n,
                        long long *c, double *th) {
  if (X < xmin) X = xmin;
  if (X > xmax) X = xmax;
  double s = (X - xmin) / dx;
  long long q = (long long)floor(s);
  if (q < 0) q = 0;
  if (q > n - 2) q = n - 2;
  *c = q;
  *th = s - (double)q;
}

/* Value at (X1, X2) of the bicubic Hermite interpolant of v with scaled
 * derivatives fx, fy, fxy: the sum over the cell's four corners of
 * v H0(t1) H0(t2) + fx H1(t1) H0(t2) + fy H0(t1) H1(t2) + fxy H1(t1) H1(t2),
 * H0 / H1 the value / slope basis function of that corner. */
double orc2_interp(const orc2_problem *p, const double *v, const double *fx,
                   const double *fy, const double *fxy, double X1, double X2) {
  double dx1 = (p->x1_max - p->x1_min) / (double)(p->Nx1 - 1);
  double dx2 = (p->x2_max - p->x2_min) / (double)(p->Nx2 - 1);
  long long c1, c2;
  double t1, t2;
  orc2_locate(X1, p->x1_min, p->x1_max, dx1, p->Nx1, &c1, &t1);
  orc2_locate(X2, p->x2_min, p->x2_max, dx2, p->Nx2, &c2, &t2);
  double a0, a1, b0, b1, c0v, c1v, d0, d1;
  orc2_hermite(t1, &a0, &a1, &b0, &b1);  /* x1: H0 = (a0, a1), H1 = (b0, b1) */
  orc2_hermite(t2, &c0v, &c1v, &d0, &d1); /* x2: H0 = (c0v, c1v), H1 = (d0, d1) */
  double H0x[2] = {a0, a1}, H1x[2] = {b0, b1}, H0y[2] = {c0v, c1v}, H1y[2] = {d0, d1};
  double s = 0.0;
  for (int e2 = 0; e2 < 2; ++e2) {
    for (int e1 = 0; e1 < 2; ++e1) {
      long long q = (c1 + e1) + p->Nx1 * (c2 + e2);
      s += v[q] * H0x[e1] * H0y[e2] + fx[q] * H1x[e1] * H0y[e2] +
           fy[q] * H0x[e1] * H1y[e2] + fxy[q] * H1x[e1] * H1y[e2];
    }
  }
  return s;
}

/* ---- driver and closed forms --------------------------------------------- */
double orc2_driver(const orc2_problem *p, double y, double z1, double z2) {
  return p->alpha * y + p->beta1 * z1 + p->beta2 * z2;
}

static double orc2_ncdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* u(t, x) and z = (u_x1, u_x2) B.
 * SIN_SUM: u = sin(x1 + x2 + t) (Eq. 35; solves the PDE for X = W and
 *          f = y - (z1 + z2)/2, Example 4).
 * SPREAD_LOG: the zero-strike spread option (e^{x1} - e^{x2})^+ in log prices
 *          by Margrabe's formula (Eq. 37), sigma1 = b11, sigma2 =
 *          sqrt(b21^2 + b22^2), rho sigma1 sigma2 = b11 b21. */
int orc2_exact(const orc2_problem *p, double t, double x1, double x2, double *u, double *z) {
  double u1, u2;
  if (p->terminal == ORC2_TERM_SIN_SUM) {
    *u = sin(x1 + x2 + t);
    u1 = u2 = cos(x1 + x2 + t);
  } else if (p->terminal == ORC2_TERM_SPREAD_LOG) {
    double S1 = exp(x1), S2 = exp(x2), tau = p->T - t;
    double s1 = p->b11, s2 = sqrt(p->b21 * p->b21 + p->b22 * p->b22);
    double var = s1 * s1 + s2 * s2 - 2.0 * p->b11 * p->b21;
    if (tau <= 0.0 || var <= 0.0) {
      *u = S1 > S2 ? S1 - S2 : 0.0;
      u1 = S1 > S2 ? S1 : 0.0;
      u2 = S1 > S2 ? -S2 : 0.0;
    } else {
      double sq = sqrt(var * tau);
      double d1 = (x1 - x2 + 0.5 * var * tau) / sq, d2 = d1 - sq;
      *u = S1 * orc2_ncdf(d1) - S2 * orc2_ncdf(d2);
      u1 = S1 * orc2_ncdf(d1);   /* S1 dV/dS1 */
      u2 = -S2 * orc2_ncdf(d2);  /* S2 dV/dS2 */
    }
  } else {
    return -1;
  }
  z[0] = u1 * p->b11 + u2 * p->b21;
  z[1] = u2 * p->b22;
  return 0;
}

/* K initial levels from the closed form: row m = level N - m, fields
 * y, z1, z2 each Nx1 Nx2 values (i1 fastest). */
int orc2_init_levels(const orc2_problem *p, double *iy, double *iz1, double *iz2) {
  double dt = p->T / p->N;
  double dx1 = (p->x1_max - p->x1_min) / (double)(p->Nx1 - 1);
  double dx2 = (p->x2_max - p->x2_min) / (double)(p->Nx2 - 1);
  long long np = p->Nx1 * p->Nx2;
  for (int m = 0; m < p->k; ++m) {
    double t = (p->N - m) * dt;
    for (long long i2 = 0; i2 < p->Nx2; ++i2)
      for (long long i1 = 0; i1 < p->Nx1; ++i1) {
        double u, z[2];
        if (orc2_exact(p, t, p->x1_min + i1 * dx1, p->x2_min + i2 * dx2, &u, z)) return -1;
        long long q = m * np + i1 + p->Nx1 * i2;
        iy[q] = u;
        iz1[q] = z[0];
        iz2[q] = z[1];
      }
  }
  return 0;
}

/* ---- the backward loop (Eq. 20 with d = 2) ------------------------------- */
/* init_*: k x Nx1 Nx2 (row m = level N - m), or NULL for the closed form.
 * levels: as in orc_solve (0 = all).  out_*: the last computed level. */
int orc2_solve(const orc2_problem *p, const double *init_y, const double *init_z1,
               const double *init_z2, long long levels, double *out_y, double *out_z1,
               double *out_z2, orc2_result *res, int threads) {
  memset(res, 0, sizeof(*res));
  if (orc2_check(p)) { res->status = -1; return -1; }
  const int k = p->k, N = p->N, L = p->L, ns = k + 1;
  const long long n1 = p->Nx1, n2 = p->Nx2, np = n1 * n2;
  const double dt = p->T / N;
  const double dx1 = (p->x1_max - p->x1_min) / (double)(n1 - 1);
  const double dx2 = (p->x2_max - p->x2_min) / (double)(n2 - 1);
  double gy[7], gz[7];
  orc_gamma(k, gy, gz);
  double *a = malloc(sizeof(double) * L), *w = malloc(sizeof(double) * L);
  /* per slot and field: value, fx, fy, fxy */
  double *V = malloc(sizeof(double) * (size_t)ns * 3 * 4 * np);
  int *iters = malloc(sizeof(int) * (size_t)np);
  double *resid = malloc(sizeof(double) * (size_t)np);
  double *iy = NULL, *iz1 = NULL, *iz2 = NULL;
  if (!a || !w || !V || !iters || !resid) {
    free(a); free(w); free(V); free(iters); free(resid);
    res->status = -2;
    return -2;
  }
  orc_gauss_hermite(L, a, w);
#define FIELD(slot, f, c) (V + (((size_t)(slot) * 3 + (f)) * 4 + (c)) * (size_t)np)
  if (!(init_y && init_z1 && init_z2)) {
    iy = malloc(sizeof(double) * (size_t)k * np);
    iz1 = malloc(sizeof(double) * (size_t)k * np);
    iz2 = malloc(sizeof(double) * (size_t)k * np);
    if (!iy || !iz1 || !iz2 || orc2_init_levels(p, iy, iz1, iz2)) {
      free(iy); free(iz1); free(iz2);
      free(a); free(w); free(V); free(iters); free(resid);
      res->status = -1;
      return -1;
    }
    init_y = iy; init_z1 = iz1; init_z2 = iz2;
  }
  for (int m = 0; m < k; ++m) {
    int slot = (N - m) % ns;
    const double *src[3] = {init_y + (size_t)m * np, init_z1 + (size_t)m * np,
                            init_z2 + (size_t)m * np};
    for (int f = 0; f < 3; ++f) {
      memcpy(FIELD(slot, f, 0), src[f], sizeof(double) * (size_t)np);
      orc2_derivatives(n1, n2, FIELD(slot, f, 0), FIELD(slot, f, 1), FIELD(slot, f, 2),
                       FIELD(slot, f, 3));
    }
  }
  free(iy); free(iz1); free(iz2);

  long long total = N - k + 1;
  if (levels <= 0 || levels > total) levels = total;
  int last = N - k + 1, itmax = 0, nonconv = 0;
  double rmax = 0.0;
  const double rpi = 1.0 / ORC2_PI;
  for (long long lv = 0; lv < levels; ++lv) {
    const int n = N - k - (int)lv;
    const int sn = n % ns;
    const double h = k * dt;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (long long q = 0; q < np; ++q) {
      const long long i1 = q % n1, i2 = q / n1;
      const double x1 = p->x1_min + i1 * dx1, x2 = p->x2_min + i2 * dx2;
      /* per j: E[z1], E[z2], E[F], E[F dW1], E[F dW2], E[y] */
      double E[6][6];
      for (int j = 1; j <= k; ++j) {
        const int sl = (n + j) % ns;
        const double sq = sqrt(2.0 * j * dt);
        double ez1 = 0, ez2 = 0, ef = 0, efw1 = 0, efw2 = 0, ey = 0;
        for (int l1 = 0; l1 < L; ++l1) {
          for (int l2 = 0; l2 < L; ++l2) {
            const double dW1 = sq * a[l1], dW2 = sq * a[l2];
            const double X1 = x1 + p->a1 * j * dt + p->b11 * dW1;
            const double X2 = x2 + p->a2 * j * dt + p->b21 * dW1 + p->b22 * dW2;
            const double yh = orc2_interp(p, FIELD(sl, 0, 0), FIELD(sl, 0, 1), FIELD(sl, 0, 2),
                                          FIELD(sl, 0, 3), X1, X2);
            const double z1h = orc2_interp(p, FIELD(sl, 1, 0), FIELD(sl, 1, 1),
                                           FIELD(sl, 1, 2), FIELD(sl, 1, 3), X1, X2);
            const double z2h = orc2_interp(p, FIELD(sl, 2, 0), FIELD(sl, 2, 1),
                                           FIELD(sl, 2, 2), FIELD(sl, 2, 3), X1, X2);
            const double F = orc2_driver(p, yh, z1h, z2h);
            const double wt = w[l1] * w[l2] * rpi;
            ez1 += wt * z1h;
            ez2 += wt * z2h;
            ef += wt * F;
            efw1 += wt * F * dW1;
            efw2 += wt * F * dW2;
            ey += wt * yh;
          }
        }
        E[j - 1][0] = ez1; E[j - 1][1] = ez2; E[j - 1][2] = ef;
        E[j - 1][3] = efw1; E[j - 1][4] = efw2; E[j - 1][5] = ey;
      }
      /* z: second line of Eq. 20, componentwise */
      double z[2];
      for (int d = 0; d < 2; ++d) {
        double s = E[0][d];
        for (int j = 1; j <= k; ++j) s += gz[j] * (E[j - 1][3 + d] - E[j - 1][d]);
        z[d] = s / gz[0];
      }
      /* y: first line of Eq. 20 by Picard from y^{n+1} */
      double sf = 0.0;
      for (int j = 1; j <= k; ++j) sf += gy[j] * E[j - 1][2];
      const double A = E[k - 1][5] + h * sf;
      double y = FIELD((n + 1) % ns, 0, 0)[q], d = 0.0;
      int it = 0;
      while (it < p->picard_max) {
        const double y1 = A + h * gy[0] * orc2_driver(p, y, z[0], z[1]);
        d = fabs(y1 - y);
        y = y1;
        ++it;
        if (d <= p->picard_tol) break;
      }
      FIELD(sn, 0, 0)[q] = y;
      FIELD(sn, 1, 0)[q] = z[0];
      FIELD(sn, 2, 0)[q] = z[1];
      iters[q] = it;
      resid[q] = d;
    }
    for (long long q = 0; q < np; ++q) {
      if (iters[q] > itmax) itmax = iters[q];
      if (resid[q] > rmax) rmax = resid[q];
      if (resid[q] > p->picard_tol) nonconv = 1;
    }
    for (int f = 0; f < 3; ++f)
      orc2_derivatives(n1, n2, FIELD(sn, f, 0), FIELD(sn, f, 1), FIELD(sn, f, 2),
                       FIELD(sn, f, 3));
    last = n;
  }
  const int sl = last % ns;
  res->y0 = orc2_interp(p, FIELD(sl, 0, 0), FIELD(sl, 0, 1), FIELD(sl, 0, 2), FIELD(sl, 0, 3),
                        p->x01, p->x02);
  res->z0[0] = orc2_interp(p, FIELD(sl, 1, 0), FIELD(sl, 1, 1), FIELD(sl, 1, 2),
                           FIELD(sl, 1, 3), p->x01, p->x02);
  res->z0[1] = orc2_interp(p, FIELD(sl, 2, 0), FIELD(sl, 2, 1), FIELD(sl, 2, 2),
                           FIELD(sl, 2, 3), p->x01, p->x02);
  res->levels_done = levels;
  res->picard_iters_max = itmax;
  res->picard_resid_max = rmax;
  res->status = nonconv ? 1 : 0;
  if (out_y) memcpy(out_y, FIELD(sl, 0, 0), sizeof(double) * (size_t)np);
  if (out_z1) memcpy(out_z1, FIELD(sl, 1, 0), sizeof(double) * (size_t)np);
  if (out_z2) memcpy(out_z2, FIELD(sl, 2, 0), sizeof(double) * (size_t)np);
#undef FIELD
  free(a); free(w); free(V); free(iters); free(resid);
  return 0;
}
