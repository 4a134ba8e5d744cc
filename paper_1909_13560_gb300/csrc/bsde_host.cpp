// Host-side plan constants for the multistep BSDE solver: validation, the
// Gauss-Hermite rule, the multistep coefficients and the per-(j, l) node
// tables (Section 2.2, Eq. 20-21; Section 3.2 remarks on the uniform grid).
#include <cmath>
#include <cstring>
#include <mutex>

#include "bsde_internal.h"

namespace bsde {

int validate(const bsde_problem &p) {
  if (p.k < 1 || p.k > kMaxK || p.k_z < 0 || p.k_z > kMaxK || p.N < 1) return BSDE_EINVAL;
  if (problem_K(p) > p.N) return BSDE_EINVAL;
  if (p.z_form != BSDE_ZFORM_EZ && p.z_form != BSDE_ZFORM_EYDW) return BSDE_EINVAL;
  if (p.init_mode != BSDE_INIT_EXACT && p.init_mode != BSDE_INIT_ONESTEP) return BSDE_EINVAL;
  if (p.init_mode == BSDE_INIT_ONESTEP &&
      (p.init_substeps < 1 || int64_t(p.N) * p.init_substeps > (int64_t(1) << 30)))
    return BSDE_EINVAL;
  if (p.Nx < 4 || p.Nx > (int64_t(1) << 30)) return BSDE_EINVAL;
  if (p.L < 1 || p.L > kMaxL) return BSDE_EINVAL;
  if (!(p.T > 0.0) || !(p.x_max > p.x_min)) return BSDE_EINVAL;
  if (!(p.x0 >= p.x_min && p.x0 <= p.x_max)) return BSDE_EINVAL;
  if (p.driver < BSDE_DRIVER_LIN_SIN || p.driver > BSDE_DRIVER_SHORT_RATE) return BSDE_EINVAL;
  if (p.terminal < BSDE_TERMINAL_SIN || p.terminal > BSDE_TERMINAL_CALL_PRICE) return BSDE_EINVAL;
  if (p.forward != BSDE_FORWARD_CONST && p.forward != BSDE_FORWARD_AFFINE) return BSDE_EINVAL;
  // terminals whose closed form (initial levels, and the start-up's level N)
  // needs a particular forward process
  if (p.terminal == BSDE_TERMINAL_ONE &&
      !(p.forward == BSDE_FORWARD_AFFINE && p.a_1 < 0.0 && p.b_1 == 0.0))
    return BSDE_EINVAL;
  if (p.terminal == BSDE_TERMINAL_CALL_PRICE &&
      !(p.forward == BSDE_FORWARD_AFFINE && p.a_x == 0.0 && p.b_x == 0.0 && p.b_1 > 0.0 &&
        p.x_min > 0.0))
    return BSDE_EINVAL;
  if (p.precision != BSDE_FP64 && p.precision != BSDE_FP32C) return BSDE_EINVAL;
  if (p.step_kernel < BSDE_STEP_AUTO || p.step_kernel > BSDE_STEP_FLAT) return BSDE_EINVAL;
  if (p.picard_max < 1 || !(p.picard_tol >= 0.0)) return BSDE_EINVAL;
  if ((p.driver == BSDE_DRIVER_BS || p.driver == BSDE_DRIVER_LB) && p.sigma == 0.0) return BSDE_EINVAL;
  return BSDE_OK;
}

// ---- Gauss-Hermite rule for the weight exp(-a^2) (Eq. 21) -----------------
// Nodes: eigenvalues of the symmetric tridiagonal Jacobi matrix of the Hermite
// recurrence (zero diagonal, off-diagonal sqrt(m/2)), isolated one by one by
// bisection on the Sturm sequence count, then polished by Newton steps on the
// scaled Hermite polynomial h_m = H_m / sqrt(2^m m!),
//   h_{m+1} = sqrt(2/(m+1)) a h_m - sqrt(m/(m+1)) h_{m-1},  h'_L = sqrt(2L) h_{L-1}.
// Weights: w = sqrt(pi) / (L h_{L-1}(a)^2), the classical formula
// 2^{L-1} L! sqrt(pi) / (L^2 H_{L-1}(a)^2) rewritten in the scaled basis.
static int sturm_count_below(int L, double lam) {
  // number of eigenvalues < lam of tridiag(beta, 0, beta)
  int cnt = 0;
  double q = -lam;
  if (q < 0) ++cnt;
  for (int m = 1; m < L; ++m) {
    double b2 = 0.5 * m;
    if (q == 0.0) q = 1e-300;
    q = -lam - b2 / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

static void scaled_hermite(long double a, int L, long double &hL, long double &hLm1) {
  long double h0 = 1.0L, h1 = std::sqrt(2.0L) * a;
  if (L == 0) { hL = h0; hLm1 = 0; return; }
  if (L == 1) { hL = h1; hLm1 = h0; return; }
  for (int m = 1; m < L; ++m) {
    long double h2 = std::sqrt(2.0L / (m + 1)) * a * h1 - std::sqrt((long double)m / (m + 1)) * h0;
    h0 = h1;
    h1 = h2;
  }
  hL = h1;
  hLm1 = h0;
}

int gauss_hermite(int L, double *nodes, double *weights) {
  if (L < 1 || L > 128) return BSDE_EINVAL;
  const double bound = std::sqrt(2.0 * L + 1.0) + 1.0;
  for (int m = 0; m < L; ++m) {
    // the m-th smallest eigenvalue: count(lo) <= m < count(hi)
    double lo = -bound, hi = bound;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * (1.0 + std::fabs(lo)); ++it) {
      double mid = 0.5 * (lo + hi);
      if (sturm_count_below(L, mid) > m) hi = mid; else lo = mid;
    }
    long double a = 0.5L * ((long double)lo + (long double)hi);
    for (int it = 0; it < 6; ++it) {
      long double hL, hLm1;
      scaled_hermite(a, L, hL, hLm1);
      long double d = std::sqrt(2.0L * L) * hLm1;
      if (d == 0.0L) break;
      a -= hL / d;
    }
    long double hL, hLm1;
    scaled_hermite(a, L, hL, hLm1);
    nodes[m] = (double)a;
    weights[m] = (double)(std::sqrt((long double)M_PI) / ((long double)L * hLm1 * hLm1));
  }
  // the rule is symmetric: make it so to the last bit (a_{L-1-l} = -a_l,
  // equal weights), which the pairwise kernels rely on
  for (int m = 0; m < L / 2; ++m) {
    const double a = 0.5 * (nodes[L - 1 - m] - nodes[m]);
    const double w = 0.5 * (weights[m] + weights[L - 1 - m]);
    nodes[m] = -a;
    nodes[L - 1 - m] = a;
    weights[m] = w;
    weights[L - 1 - m] = w;
  }
  if (L % 2 == 1) nodes[L / 2] = 0.0;
  return BSDE_OK;
}

// ---- multistep coefficients (Table 1: gamma^k_{k,j}; Table 2: gamma^1_{k,j}) --
struct Frac { int num, den; };
static const Frac kTable1[6][7] = {
    {{1, 2}, {1, 2}},
    {{1, 6}, {2, 3}, {1, 6}},
    {{1, 8}, {3, 8}, {3, 8}, {1, 8}},
    {{1, 12}, {1, 3}, {1, 6}, {1, 3}, {1, 12}},
    {{41, 600}, {19, 75}, {107, 600}, {107, 600}, {19, 75}, {41, 600}},
    {{19, 336}, {3, 14}, {15, 112}, {4, 21}, {15, 112}, {3, 14}, {19, 336}}};
static const Frac kTable2[6][7] = {
    {{1, 2}, {1, 2}},
    {{5, 12}, {2, 3}, {-1, 12}},
    {{3, 8}, {19, 24}, {-5, 24}, {1, 24}},
    {{35, 96}, {5, 6}, {-13, 48}, {1, 12}, {-1, 96}},
    {{131, 360}, {151, 180}, {-103, 360}, {37, 360}, {-1, 45}, {1, 360}},
    {{163, 448}, {47, 56}, {-129, 448}, {3, 28}, {-37, 1344}, {1, 168}, {-1, 1344}}};

int gamma_tables(int k, double *gy, double *gz) {
  if (k < 1 || k > kMaxK) return BSDE_EINVAL;
  for (int j = 0; j <= k; ++j) {
    gy[j] = double(kTable1[k - 1][j].num) / double(kTable1[k - 1][j].den);
    gz[j] = double(kTable2[k - 1][j].num) / double(kTable2[k - 1][j].den);
  }
  return BSDE_OK;
}

int fill_params(const bsde_problem &p, Params &P) {
  int rc = validate(p);
  if (rc) return rc;
  std::memset(&P, 0, sizeof(P));
  P.Nx = p.Nx;
  P.N = p.N;
  P.k = problem_K(p);
  P.ky = p.k;
  P.kz = problem_kz(p);
  P.zform = p.z_form;
  P.general = problem_general(p) ? 1 : 0;
  // resolved by the work split when automatic (-1)
  P.flat = p.step_kernel == BSDE_STEP_FLAT ? 1 : p.step_kernel == BSDE_STEP_GROUPED ? 0 : -1;
  P.a_1 = p.forward == BSDE_FORWARD_AFFINE ? p.a_1 : 0.0;
  P.b_1 = p.forward == BSDE_FORWARD_AFFINE ? p.b_1 : 0.0;
  P.L = p.L;
  P.driver = p.driver;
  P.terminal = p.terminal;
  P.precision = p.precision;
  P.smoothing = p.smoothing;
  P.picard_max = p.picard_max;
  P.nslot = P.k + 1;
  P.T = p.T;
  P.dt = p.T / p.N;
  P.dx = (p.x_max - p.x_min) / double(p.Nx - 1);
  P.x_min = p.x_min;
  P.x_max = p.x_max;
  P.x0 = p.x0;
  P.a_x = p.a_x;
  P.b_x = p.b_x;
  P.r = p.r;
  P.mu = p.mu;
  P.sigma = p.sigma;
  P.R = p.R;
  P.delta = p.delta;
  P.lb_sign = p.lb_sign;
  P.strike = p.strike;
  P.picard_tol = p.picard_tol;
  {
    // |d| <= tol for a float d is exactly |d| <= the largest float <= tol
    float tf = (float)p.picard_tol;
    if ((double)tf > p.picard_tol) tf = std::nextafter(tf, 0.0f);
    P.picard_tol_f = tf;
  }
  {
    // y: Table 1 row K_y; z: Table 2 row K_z; zero beyond
    double unused[kMaxK + 1];
    gamma_tables(P.ky, P.gy, unused);
    gamma_tables(P.kz, unused, P.gz);
  }
  P.h = P.ky * P.dt;
  P.hg0 = P.h * P.gy[0];
  P.hg0_f = float(P.hg0);
  P.inv_gz0 = 1.0 / P.gz[0];
  P.inv_dx2_6 = 6.0 / (P.dx * P.dx);
  P.inv_dx = 1.0 / P.dx;
  // LU pivots of tridiag(1, 4, 1): d_0 = 4, d_m = 4 - 1/d_{m-1}; they reach
  // 2 + sqrt(3) to double precision long before m = 64.
  double d = 4.0;
  for (int m = 0; m < kInvPivots; ++m) {
    P.invd[m] = 1.0 / d;
    d = 4.0 - 1.0 / d;
  }
  return BSDE_OK;
}

bool has_startup(const bsde_problem &p) {
  return p.init_mode == BSDE_INIT_ONESTEP && problem_K(p) > 1;
}

Params startup_params(const Params &P, int substeps) {
  Params Q = P;
  Q.N = P.N * substeps;
  Q.dt = P.T / Q.N;  // the time grid t = n' T / (N S): t_{N-m} is n' = (N - m) S
  Q.k = Q.ky = Q.kz = 1;
  Q.nslot = 2;
  for (int j = 0; j <= kMaxK; ++j) Q.gy[j] = Q.gz[j] = 0.0;
  gamma_tables(1, Q.gy, Q.gz);
  Q.h = Q.dt;
  Q.hg0 = Q.h * Q.gy[0];
  Q.hg0_f = float(Q.hg0);
  Q.inv_gz0 = 1.0 / Q.gz[0];
  return Q;
}

Layout layout_for(const bsde_problem &p) {
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  Layout L{};
  const int K = problem_K(p);
  const size_t nx = size_t(p.Nx), ns = size_t(K + 1);
  size_t off = 0;
  if (p.precision == BSDE_FP64) {
    L.ring64 = off; off = up(off + ns * nx * 32);
  } else {
    L.ringA = off; off = up(off + ns * nx * 16);
    L.ringB = off; off = up(off + ns * nx * 8);  // second derivatives (M_y, M_z)
  }
  const size_t node = p.precision == BSDE_FP64 ? sizeof(NodeF64) : sizeof(NodeF32);
  L.table = off; off = up(off + size_t(K) * p.L * node);
  L.ptable = off; off = up(off + size_t(K) * ((p.L + 1) / 2) * sizeof(PairF32));
  L.stage = off; off = up(off + 2 * size_t(K) * nx * 8);
  if (has_startup(p)) {
    if (p.precision == BSDE_FP64) {
      L.sub_ring64 = off; off = up(off + 2 * nx * 32);
    } else {
      L.sub_ringA = off; off = up(off + 2 * nx * 16);
      L.sub_ringB = off; off = up(off + 2 * nx * 8);
    }
    L.sub_table = off; off = up(off + size_t(p.L) * node);
    L.sub_ptable = off; off = up(off + size_t((p.L + 1) / 2) * sizeof(PairF32));
  }
  L.stats = off; off = up(off + sizeof(Stats));
  L.total = off;
  return L;
}

// Work split of the step kernels: enough (j, l-chunk) groups per point that a
// level of a modest grid still fills the GPU (at least target_groups), but no
// more threads per level than the GPU holds at once when that is known
// (resident_threads > 0): a level that fits one wave is not split further.
static void work_split(Params &P, int target_groups, int max_groups, long resident_threads) {
  // FP64 splits the L nodes, FP32C the ceil(L/2) symmetric pairs
  P.Lp = (P.L + 1) / 2;
  const int units = P.precision == BSDE_FP64 ? P.L : P.Lp;
  int S = (target_groups + P.k - 1) / P.k;
  if (S * P.k > max_groups) S = max_groups / P.k;
  if (S > units) S = units;
  while (S > 1 && resident_threads > 0 && long(P.Nx) * P.k * S > resident_threads) --S;
  if (S < 1) S = 1;
  P.S = S;
  P.Lg = (units + S - 1) / S;
  P.G = P.k * S;
  // automatic: a grid whose points alone fill the resident threads twice
  // takes the flat kernel (same split, same order of operations)
  const bool big = P.precision == BSDE_FP32C && resident_threads > 0 &&
                   long(P.Nx) >= 2 * resident_threads;
  if (P.flat < 0) P.flat = big;
  P.wide_spline = big;
}

// Node tables.  On the uniform grid with a constant-coefficient forward
// process the off-grid point of (j, l) is x_i + o_jl dx with the same o_jl for
// every i (Section 3.2, third remark: the cell index is found without a
// search); its cell is i + floor(o_jl) and its position inside the cell
// theta = o_jl - floor(o_jl).
// The Gauss-Hermite rule depends on L only: computed once per L and kept.
static void cached_rule(int L, double *a, double *w) {
  static std::mutex mu;
  static bool have[kMaxL + 1];
  static double na[kMaxL + 1][kMaxL], nw[kMaxL + 1][kMaxL];
  std::lock_guard<std::mutex> lk(mu);
  if (!have[L]) {
    gauss_hermite(L, na[L], nw[L]);
    have[L] = true;
  }
  std::memcpy(a, na[L], sizeof(double) * L);
  std::memcpy(w, nw[L], sizeof(double) * L);
}

void build_tables(Params &P, NodeF64 *t64, NodeF32 *t32, PairF32 *tp, int target_groups,
                  int max_groups, long resident_threads) {
  work_split(P, target_groups, max_groups, resident_threads);
  double a[kMaxL], w[kMaxL];
  cached_rule(P.L, a, w);
  for (int q = 0; q < P.Lp && q < kMaxL / 2; ++q) {
    P.gh_hi[q] = float(a[q]);
    P.gh_lo[q] = float(a[q] - double(P.gh_hi[q]));
  }
  const double rpi = 1.0 / std::sqrt(M_PI);
  const double c6 = P.dx * P.dx / 6.0;
  P.c6 = c6;
  P.c6_f = float(c6);
  P.xmin_f[0] = float(P.x_min);
  P.xmin_f[1] = float(P.x_min - double(P.xmin_f[0]));
  P.dx_f[0] = float(P.dx);
  P.dx_f[1] = float(P.dx - double(P.dx_f[0]));
  for (int j = 1; j <= P.k; ++j) {
    const double sq = std::sqrt(2.0 * j * P.dt);
    {
      const double g[4] = {P.a_x * double(j) * P.dt * P.inv_dx, P.a_1 * double(j) * P.dt * P.inv_dx,
                           P.b_x * sq * P.inv_dx, P.b_1 * sq * P.inv_dx};
      for (int q = 0; q < 4; ++q) {
        P.gen_f[j - 1][2 * q] = float(g[q]);
        P.gen_f[j - 1][2 * q + 1] = float(g[q] - double(P.gen_f[j - 1][2 * q]));
      }
    }
    int smin = 0x7fffffff, smax = -0x7fffffff;
    for (int l = 0; l < P.L; ++l) {
      const double dW = sq * a[l];
      const double o = (P.a_x * j * P.dt + P.b_x * dW) / P.dx;
      // a shift beyond the grid only ever clamps: keep |shift| <= Nx + 1 so
      // that i + shift stays in 32-bit range
      const double lim = double(P.Nx + 1);
      const double s = std::fmin(std::fmax(std::floor(o), -lim), lim);
      const double th = o - std::floor(o);
      const double om = 1.0 - th;
      const double wt = w[l] * rpi;
      NodeF64 e{};
      e.shift = (int32_t)s;
      e.w0 = om;
      e.w1 = th;
      e.w2 = c6 * (om * om * om - om);
      e.w3 = c6 * (th * th * th - th);
      // gy[j] = 0 for j > K_y and gz[j] = 0 for j > K_z
      const bool ez1 = j == 1 && !P.zform;
      e.cz = wt * ((ez1 ? 1.0 : 0.0) - P.gz[j]) * P.inv_gz0;
      e.cfz = P.gz[j] * wt * dW * P.inv_gz0;
      e.cfy = P.h * P.gy[j] * wt;
      e.cy = (j == P.ky) ? wt : 0.0;
      e.cyz = (j == 1 && P.zform) ? wt * dW / P.dt * P.inv_gz0 : 0.0;
      e.dW = dW;
      if (e.shift < smin) smin = e.shift;
      if (e.shift > smax) smax = e.shift;
      const int idx = (j - 1) * P.L + l;
      if (t64) t64[idx] = e;
      if (t32) {
        NodeF32 f{};
        f.shift = e.shift;
        f.w0 = (float)e.w0;
        f.w1 = (float)e.w1;
        f.w2 = (float)e.w2;
        f.w3 = (float)e.w3;
        f.czh = (float)e.cz;
        f.czl = (float)(e.cz - (double)f.czh);
        f.cfz = (float)e.cfz;
        f.cfy = (float)e.cfy;
        f.cyh = (float)e.cy;
        f.cyl = (float)(e.cy - (double)f.cyh);
        f.cyzh = (float)e.cyz;
        f.cyzl = (float)(e.cyz - (double)f.cyzh);
        t32[idx] = f;
      }
    }
    P.smin[j - 1] = smin;
    P.smax[j - 1] = smax;
    if (tp && t32) {
      for (int q = 0; q < P.Lp; ++q) {
        const NodeF32 &na = t32[(j - 1) * P.L + q];
        const NodeF32 &nb = t32[(j - 1) * P.L + (P.L - 1 - q)];
        const bool single = (q == P.L - 1 - q);
        const float half = single ? 0.5f : 1.0f;  // exact in binary
        PairF32 pr{};
        pr.shift_a = na.shift;
        pr.shift_b = nb.shift;
        pr.cfz = na.cfz;  // zero for the middle node (DeltaW = 0)
        pr.cfy = na.cfy * half;
        const double tha = double(na.w1), thb = double(nb.w1);
        const float kaa = float(-c6 * tha * (1.0 - tha)), kab = float(-c6 * thb * (1.0 - thb));
        for (int v = 0; v < 2; ++v) {
          pr.tha[v] = na.w1;
          pr.kaa[v] = kaa;
          pr.thb[v] = nb.w1;
          pr.kab[v] = kab;
        }
        // lanes (y, z)
        pr.ch[0] = na.cyh * half;
        pr.ch[1] = na.czh * half;
        pr.nch[0] = -pr.ch[0];
        pr.nch[1] = -pr.ch[1];
        pr.ncl[0] = -(na.cyl * half);
        pr.ncl[1] = -(na.czl * half);
        // node b's y weight is -cyz (opposite DeltaW); the middle node has 0
        pr.cyz[0] = na.cyzh;
        pr.cyz[1] = na.cyzl;
        tp[(j - 1) * P.Lp + q] = pr;
      }
    }
  }
}

}  // namespace bsde
