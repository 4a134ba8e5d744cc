// Two-dimensional solver (Eq. 20-21 with d = 2; Section 3.3; Examples 4
// and 5): kernels, plan and the C ABI of include/bsde2d.h.  Included by
// bsde_cuda.cu after bsde_kernels.cuh (one translation unit).
#pragma once

#include "../../include/bsde2d.h"

namespace bsde {

constexpr int kMaxL2 = 16;      // Gauss-Hermite nodes per dimension
constexpr int kStep2TP = 64;    // grid points per CTA in the 2-D step kernel
constexpr int kDerTX = 32, kDerTY = 8, kDerH = 4;  // derivative tile and halo

struct Params2 {
  int64_t Nx1, Nx2, Np;
  int32_t N, k, L, LL, nslot, picard_max, terminal, pad;
  double T, dt, dx1, dx2, x1_min, x1_max, x2_min, x2_max, x01, x02;
  double a1, a2, b11, b21, b22, alpha, beta1, beta2, picard_tol;
  double gy[kMaxK + 1], gz[kMaxK + 1];
  double h, hg0;
  // work split: S chunks of Lg nodes per j, G = k S groups per point;
  // per j the range of cell shifts in each dimension (clamp-free fast path)
  int32_t S, Lg, G, pad2;
  int32_t s1min[kMaxK], s1max[kMaxK], s2min[kMaxK], s2max[kMaxK];
};

// Per (j, l1, l2) node: the cell shift in each dimension, the cubic Hermite
// basis of the position theta inside the cell in each dimension (value
// weights of the left and right node, slope weights of the left and right
// node, slopes scaled by the spacing), and the weights of Eq. 20-21 with
// wt = omega_l1 omega_l2 / pi, DeltaW = sqrt(2 j dt) (a_l1, a_l2):
//   z_d^n = sum cz z^_d + cfz_d F,   cz = wt (delta_j1 - gz_j) / gz_0,
//                                    cfz_d = gz_j wt DeltaW_d / gz_0
//   A     = sum cy y^ + cfy F,       cy = wt (j = k), cfy = k dt gy_j wt.
struct Node2 {
  int32_t s1, s2;
  double h1[4], h2[4];
  double cz, cfz1, cfz2, cfy, cy;
};

struct Stats2 {
  Stats s;       // y0 and the Picard statistics (z0 holds z1)
  double z0b;    // z2 at the readout point
};

__host__ __device__ inline void hermite4(double t, double *h) {
  const double t2 = t * t, t3 = t2 * t;
  h[0] = 2.0 * t3 - 3.0 * t2 + 1.0;  // value, left node
  h[1] = -2.0 * t3 + 3.0 * t2;       // value, right node
  h[2] = t3 - 2.0 * t2 + t;          // slope, left node
  h[3] = t3 - t2;                    // slope, right node
}

// ---------------------------------------------------------------------------
// Closed forms (initial levels): u and z = (u_x1, u_x2) B.
// ---------------------------------------------------------------------------
__device__ void closed_form2(const Params2 &P, double t, double x1, double x2, double &u,
                             double &z1, double &z2) {
  double u1, u2;
  if (P.terminal == BSDE2_TERMINAL_SIN_SUM) {
    u = sin(x1 + x2 + t);
    u1 = u2 = cos(x1 + x2 + t);
  } else {
    // rounded separately (no contraction with the caller's t = n dt): at
    // the terminal level tau is exactly 0 and the payoff branch is taken
    const double S1 = exp(x1), S2 = exp(x2), tau = __dsub_rn(P.T, t);
    const double s2 = sqrt(P.b21 * P.b21 + P.b22 * P.b22);
    const double var = P.b11 * P.b11 + s2 * s2 - 2.0 * P.b11 * P.b21;
    if (tau <= 0.0 || var <= 0.0) {
      u = S1 > S2 ? S1 - S2 : 0.0;
      u1 = S1 > S2 ? S1 : 0.0;
      u2 = S1 > S2 ? -S2 : 0.0;
    } else {
      const double sq = sqrt(var * tau);
      const double d1 = (x1 - x2 + 0.5 * var * tau) / sq, d2 = d1 - sq;
      u = S1 * ncdf(d1) - S2 * ncdf(d2);
      u1 = S1 * ncdf(d1);
      u2 = -S2 * ncdf(d2);
    }
  }
  z1 = u1 * P.b11 + u2 * P.b21;
  z2 = u2 * P.b22;
}

// Level values of the closed form at t_{N-m} into the new-value plane V
// (fields y, z1, z2; i1 fastest).
__global__ void k2_init_closed(const Params2 P, double *V, int m) {
  const double t = __dmul_rn(double(P.N - m), P.dt);
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < P.Np;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i1 = q % P.Nx1, i2 = q / P.Nx1;
    double u, z1, z2;
    closed_form2(P, t, P.x1_min + double(i1) * P.dx1, P.x2_min + double(i2) * P.dx2, u, z1, z2);
    V[q] = u;
    V[P.Np + q] = z1;
    V[2 * P.Np + q] = z2;
  }
}

// Level m of the caller's initial levels (staging area: y, z1, z2 planes of
// k levels each) into V.
__global__ void k2_import(const Params2 P, double *V, const double *stage, int m) {
  const int64_t kp = int64_t(P.k) * P.Np;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < P.Np;
       q += int64_t(gridDim.x) * blockDim.x) {
    for (int f = 0; f < 3; ++f) V[f * P.Np + q] = stage[f * kp + int64_t(m) * P.Np + q];
  }
}

// ---------------------------------------------------------------------------
// Derivatives of a new level (Section 3.3): fourth-order finite differences
// of the three fields, scaled by the spacings, into the ring slot as
// double4 (v, dx1 v_x1, dx2 v_x2, dx1 dx2 v_x1x2) per field and point.
// One CTA per kDerTX x kDerTY tile; the tile and a halo of 4 in each
// direction (the one-sided stencils reach 4 nodes) staged in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fd4(const double *f, int s, int i, int n) {
  // f points at node i of a line (stride s); n nodes on the line
  if (i >= 2 && i <= n - 3)
    return (f[-2 * s] - 8.0 * f[-s] + 8.0 * f[s] - f[2 * s]) / 12.0;
  if (i < 2)
    return (-25.0 * f[0] + 48.0 * f[s] - 36.0 * f[2 * s] + 16.0 * f[3 * s] - 3.0 * f[4 * s]) /
           12.0;
  return (25.0 * f[0] - 48.0 * f[-s] + 36.0 * f[-2 * s] - 16.0 * f[-3 * s] + 3.0 * f[-4 * s]) /
         12.0;
}

__global__ void __launch_bounds__(kDerTX * kDerTY)
    k2_deriv(const Params2 P, const double *__restrict__ V, double4_32a *__restrict__ ring,
             int slot) {
  constexpr int W = kDerTX + 2 * kDerH, H = kDerTY + 2 * kDerH;
  __shared__ double sv[H][W];
  __shared__ double sy[kDerTY][W];
  wait_predecessor();
  const int x0 = blockIdx.x * kDerTX, y0 = blockIdx.y * kDerTY;
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  const int tid = threadIdx.x;
  for (int f = 0; f < 3; ++f) {
    const double *v = V + int64_t(f) * P.Np;
    // tile + halo, indices clamped onto the grid (halo entries off the grid
    // are never read by an on-grid stencil)
    for (int e = tid; e < H * W; e += blockDim.x) {
      const int r = e / W, c = e % W;
      int g2 = y0 - kDerH + r, g1 = x0 - kDerH + c;
      g2 = g2 < 0 ? 0 : (g2 >= n2 ? n2 - 1 : g2);
      g1 = g1 < 0 ? 0 : (g1 >= n1 ? n1 - 1 : g1);
      sv[r][c] = v[int64_t(g2) * n1 + g1];
    }
    __syncthreads();
    // x2 derivative on the tile's rows, every column of the staged span
    for (int e = tid; e < kDerTY * W; e += blockDim.x) {
      const int r = e / W, c = e % W;
      const int i2 = y0 + r;
      sy[r][c] = i2 < n2 ? fd4(&sv[r + kDerH][c], W, i2, n2) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < kDerTX * kDerTY; e += blockDim.x) {
      const int r = e / kDerTX, c = e % kDerTX;
      const int i1 = x0 + c, i2 = y0 + r;
      if (i1 < n1 && i2 < n2) {
        const double val = sv[r + kDerH][c + kDerH];
        const double fx = fd4(&sv[r + kDerH][c + kDerH], 1, i1, n1);
        const double fy = sy[r][c + kDerH];
        const double fxy = fd4(&sy[r][c + kDerH], 1, i1, n1);
        ring[(int64_t(slot) * 3 + f) * P.Np + int64_t(i2) * n1 + i1] =
            make_double4_32a(val, fx, fy, fxy);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The 2-D step kernel: one CTA per kStep2TP consecutive grid points (i1
// fastest), G = k S groups of kStep2TP threads; group g takes j = g / S + 1
// and a chunk of the L^2 tensor nodes.  Per node a thread forms the three
// bicubic values (y^, z1^, z2^) from the four corner records of its cell
// (separably: along x1 on the two rows, then along x2), the driver, and adds
// the weighted terms; the groups' partial sums meet in shared memory and the
// first group forms z^n, A and y^n by Picard.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double bicubic(const double4_32a &a, const double4_32a &b,
                                          const double4_32a &c, const double4_32a &d,
                                          const double *h1, const double *h2) {
  // rows c2 (a, b) and c2 + 1 (c, d): value and x2-slope along x1
  const double r0 = a.x * h1[0] + b.x * h1[1] + a.y * h1[2] + b.y * h1[3];
  const double s0 = a.z * h1[0] + b.z * h1[1] + a.w * h1[2] + b.w * h1[3];
  const double r1 = c.x * h1[0] + d.x * h1[1] + c.y * h1[2] + d.y * h1[3];
  const double s1 = c.z * h1[0] + d.z * h1[1] + c.w * h1[2] + d.w * h1[3];
  return r0 * h2[0] + r1 * h2[1] + s0 * h2[2] + s1 * h2[3];
}

template <bool CLAMP>
__device__ __forceinline__ void nodes2(const Params2 &P, const double4_32a *__restrict__ lev,
                                       const Node2 *__restrict__ row, int q0, int q1, int i1,
                                       int i2, double &Z1, double &Z2, double &Ys) {
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  const int64_t Np = P.Np;
#pragma unroll 1
  for (int q = q0; q < q1; ++q) {
    const Node2 &e = row[q];
    int c1 = i1 + e.s1, c2 = i2 + e.s2;
    double h1[4], h2[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      h1[u] = e.h1[u];
      h2[u] = e.h2[u];
    }
    if (CLAMP) {
      // off the box: the value at the projection (theta 0 at the low end,
      // 1 at the high end)
      if (c1 < 0 || c1 > n1 - 2) {
        const bool lo = c1 < 0;
        c1 = lo ? 0 : n1 - 2;
        h1[0] = lo ? 1.0 : 0.0;
        h1[1] = lo ? 0.0 : 1.0;
        h1[2] = h1[3] = 0.0;
      }
      if (c2 < 0 || c2 > n2 - 2) {
        const bool lo = c2 < 0;
        c2 = lo ? 0 : n2 - 2;
        h2[0] = lo ? 1.0 : 0.0;
        h2[1] = lo ? 0.0 : 1.0;
        h2[2] = h2[3] = 0.0;
      }
    }
    const int64_t o = int64_t(c2) * n1 + c1;
    double v[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const double4_32a *L = lev + f * Np + o;
      v[f] = bicubic(L[0], L[1], L[n1], L[n1 + 1], h1, h2);
    }
    const double F = P.alpha * v[0] + P.beta1 * v[1] + P.beta2 * v[2];
    Z1 += e.cz * v[1] + e.cfz1 * F;
    Z2 += e.cz * v[2] + e.cfz2 * F;
    Ys += e.cfy * F + e.cy * v[0];
  }
}

__global__ void __launch_bounds__(kStep2TP * kMaxGroups)
    k2_step(const Params2 P, const double4_32a *__restrict__ ring, double *__restrict__ V,
            const Node2 *__restrict__ table, int n, Stats *st) {
  __shared__ double part[3][kMaxGroups][kStep2TP];
  wait_predecessor();
  const int tp = threadIdx.x % kStep2TP, g = threadIdx.x / kStep2TP;
  const int64_t q0p = int64_t(blockIdx.x) * kStep2TP;
  const int64_t qq = q0p + tp;
  const bool active = qq < P.Np;
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  double Z1 = 0.0, Z2 = 0.0, Ys = 0.0;
  if (active) {
    const int j = g / P.S + 1, lc = g % P.S;
    const int a0 = lc * P.Lg, a1 = a0 + P.Lg < P.LL ? a0 + P.Lg : P.LL;
    const int i1 = int(qq % n1), i2 = int(qq / n1);
    // the tile's rows and columns (it may wrap onto the next row)
    const int64_t qe = (q0p + kStep2TP <= P.Np ? q0p + kStep2TP : P.Np) - 1;
    const int r0 = int(q0p / n1), r1 = int(qe / n1);
    const int cmin = r0 == r1 ? int(q0p % n1) : 0, cmax = r0 == r1 ? int(qe % n1) : n1 - 1;
    const bool interior = cmin + P.s1min[j - 1] >= 0 && cmax + P.s1max[j - 1] <= n1 - 2 &&
                          r0 + P.s2min[j - 1] >= 0 && r1 + P.s2max[j - 1] <= n2 - 2;
    const double4_32a *lev = ring + int64_t((n + j) % P.nslot) * 3 * P.Np;
    const Node2 *row = table + int64_t(j - 1) * P.LL;
    if (interior)
      nodes2<false>(P, lev, row, a0, a1, i1, i2, Z1, Z2, Ys);
    else
      nodes2<true>(P, lev, row, a0, a1, i1, i2, Z1, Z2, Ys);
  }
  part[0][g][tp] = Z1;
  part[1][g][tp] = Z2;
  part[2][g][tp] = Ys;
  __syncthreads();
  if (g != 0) return;
  int it = 0;
  double d = 0.0;
  if (active) {
    double z1 = 0.0, z2 = 0.0, A = 0.0;
    for (int u = 0; u < P.G; ++u) {
      z1 += part[0][u][tp];
      z2 += part[1][u][tp];
      A += part[2][u][tp];
    }
    double y = ring[(int64_t((n + 1) % P.nslot) * 3) * P.Np + qq].x;
    while (it < P.picard_max) {
      const double y1 = A + P.hg0 * (P.alpha * y + P.beta1 * z1 + P.beta2 * z2);
      d = fabs(y1 - y);
      y = y1;
      ++it;
      if (d <= P.picard_tol) break;
    }
    V[qq] = y;
    V[P.Np + qq] = z1;
    V[2 * P.Np + qq] = z2;
  }
  record_picard(st, active, it, d, P.picard_tol);
}

// Readout at (x01, x02) of the level in `slot` (projection onto the box, the
// cell by floor, the bicubic Hermite value), and the level's export.
__device__ double interp2_point(const Params2 &P, const double4_32a *lev, double X1, double X2) {
  auto locate = [](double X, double xmin, double xmax, double dx, int64_t n, int64_t &c,
                   double &th) {
    X = X < xmin ? xmin : (X > xmax ? xmax : X);
    const double s = (X - xmin) / dx;
    int64_t q = int64_t(floor(s));
    q = q < 0 ? 0 : (q > n - 2 ? n - 2 : q);
    c = q;
    th = s - double(q);
  };
  int64_t c1, c2;
  double t1, t2, h1[4], h2[4];
  locate(X1, P.x1_min, P.x1_max, P.dx1, P.Nx1, c1, t1);
  locate(X2, P.x2_min, P.x2_max, P.dx2, P.Nx2, c2, t2);
  hermite4(t1, h1);
  hermite4(t2, h2);
  const double4_32a *L = lev + c2 * P.Nx1 + c1;
  return bicubic(L[0], L[1], L[P.Nx1], L[P.Nx1 + 1], h1, h2);
}

__global__ void k2_readout(const Params2 P, const double4_32a *ring, int slot, Stats2 *st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double4_32a *lev = ring + int64_t(slot) * 3 * P.Np;
  st->s.y0 = interp2_point(P, lev, P.x01, P.x02);
  st->s.z0 = interp2_point(P, lev + P.Np, P.x01, P.x02);
  st->z0b = interp2_point(P, lev + 2 * P.Np, P.x01, P.x02);
}

__global__ void k2_export(const Params2 P, const double4_32a *ring, int slot, double *out) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < P.Np;
       q += int64_t(gridDim.x) * blockDim.x)
    for (int f = 0; f < 3; ++f) out[f * P.Np + q] = ring[(int64_t(slot) * 3 + f) * P.Np + q].x;
}

__global__ void k2_reset_stats(Stats2 *s) {
  if (threadIdx.x == 0) {
    s->s.y0 = s->s.z0 = s->z0b = 0.0;
    s->s.resid_bits = 0ull;
    s->s.iters_max = s->s.nonconv = s->s.timeout = 0;
  }
}

// ---------------------------------------------------------------------------
// Host side: validation, constants, layout.
// ---------------------------------------------------------------------------
struct Layout2 {
  size_t ring, vals, table, stage, stats, total;
};

static int validate2(const bsde2_problem &p) {
  if (p.k < 1 || p.k > kMaxK || p.k > p.N || p.N < 1) return BSDE_EINVAL;
  if (p.Nx1 < 6 || p.Nx2 < 6 || p.Nx1 > (int64_t(1) << 20) || p.Nx2 > (int64_t(1) << 20) ||
      p.Nx1 * p.Nx2 > (int64_t(1) << 31))
    return BSDE_EINVAL;
  if (p.L < 1 || p.L > kMaxL2) return BSDE_EINVAL;
  if (!(p.T > 0.0) || !(p.x1_max > p.x1_min) || !(p.x2_max > p.x2_min)) return BSDE_EINVAL;
  if (!(p.x01 >= p.x1_min && p.x01 <= p.x1_max && p.x02 >= p.x2_min && p.x02 <= p.x2_max))
    return BSDE_EINVAL;
  if (p.driver != BSDE2_DRIVER_LINEAR) return BSDE_EINVAL;
  if (p.terminal != BSDE2_TERMINAL_SIN_SUM && p.terminal != BSDE2_TERMINAL_SPREAD_LOG)
    return BSDE_EINVAL;
  if (p.precision != BSDE_FP64) return BSDE_EINVAL;
  if (p.picard_max < 1 || !(p.picard_tol >= 0.0)) return BSDE_EINVAL;
  return BSDE_OK;
}

static Layout2 layout2(const bsde2_problem &p) {
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t np = size_t(p.Nx1) * size_t(p.Nx2), ns = size_t(p.k + 1);
  Layout2 L{};
  size_t off = 0;
  L.ring = off; off = up(off + ns * 3 * np * 32);
  L.vals = off; off = up(off + 3 * np * 8);
  L.table = off; off = up(off + size_t(p.k) * p.L * p.L * sizeof(Node2));
  L.stage = off; off = up(off + 3 * size_t(p.k) * np * 8);
  L.stats = off; off = up(off + sizeof(Stats2));
  L.total = off;
  return L;
}

static void plan2_constants(const bsde2_problem &p, Params2 &P, std::vector<Node2> &tab,
                            long resident_threads) {
  std::memset(&P, 0, sizeof(P));
  P.Nx1 = p.Nx1;
  P.Nx2 = p.Nx2;
  P.Np = p.Nx1 * p.Nx2;
  P.N = p.N;
  P.k = p.k;
  P.L = p.L;
  P.LL = p.L * p.L;
  P.nslot = p.k + 1;
  P.picard_max = p.picard_max;
  P.terminal = p.terminal;
  P.T = p.T;
  P.dt = p.T / p.N;
  P.dx1 = (p.x1_max - p.x1_min) / double(p.Nx1 - 1);
  P.dx2 = (p.x2_max - p.x2_min) / double(p.Nx2 - 1);
  P.x1_min = p.x1_min;
  P.x1_max = p.x1_max;
  P.x2_min = p.x2_min;
  P.x2_max = p.x2_max;
  P.x01 = p.x01;
  P.x02 = p.x02;
  P.a1 = p.a1;
  P.a2 = p.a2;
  P.b11 = p.b11;
  P.b21 = p.b21;
  P.b22 = p.b22;
  P.alpha = p.alpha;
  P.beta1 = p.beta1;
  P.beta2 = p.beta2;
  P.picard_tol = p.picard_tol;
  gamma_tables(p.k, P.gy, P.gz);
  P.h = p.k * P.dt;
  P.hg0 = P.h * P.gy[0];
  // work split as in 1-D: >= 4 groups per point, at most kMaxGroups, no
  // more threads per level than the GPU holds at once when that is known
  int S = (4 + P.k - 1) / P.k;
  if (S * P.k > kMaxGroups) S = kMaxGroups / P.k;
  if (S > P.LL) S = P.LL;
  while (S > 1 && resident_threads > 0 && long(P.Np) * P.k * S > resident_threads) --S;
  if (S < 1) S = 1;
  P.S = S;
  P.Lg = (P.LL + S - 1) / S;
  P.G = P.k * S;
  double a[kMaxL2], w[kMaxL2];
  gauss_hermite(p.L, a, w);
  tab.assign(size_t(P.k) * P.LL, Node2{});
  for (int j = 1; j <= P.k; ++j) {
    const double sq = std::sqrt(2.0 * j * P.dt);
    int s1lo = 0x7fffffff, s1hi = -0x7fffffff, s2lo = 0x7fffffff, s2hi = -0x7fffffff;
    for (int l1 = 0; l1 < p.L; ++l1) {
      for (int l2 = 0; l2 < p.L; ++l2) {
        const double dW1 = sq * a[l1], dW2 = sq * a[l2];
        const double o1 = (P.a1 * j * P.dt + P.b11 * dW1) / P.dx1;
        const double o2 = (P.a2 * j * P.dt + P.b21 * dW1 + P.b22 * dW2) / P.dx2;
        const double lim1 = double(P.Nx1 + 1), lim2 = double(P.Nx2 + 1);
        Node2 e{};
        e.s1 = int32_t(std::fmin(std::fmax(std::floor(o1), -lim1), lim1));
        e.s2 = int32_t(std::fmin(std::fmax(std::floor(o2), -lim2), lim2));
        hermite4(o1 - std::floor(o1), e.h1);
        hermite4(o2 - std::floor(o2), e.h2);
        const double wt = w[l1] * w[l2] / M_PI;
        e.cz = wt * ((j == 1 ? 1.0 : 0.0) - P.gz[j]) / P.gz[0];
        e.cfz1 = P.gz[j] * wt * dW1 / P.gz[0];
        e.cfz2 = P.gz[j] * wt * dW2 / P.gz[0];
        e.cfy = P.h * P.gy[j] * wt;
        e.cy = j == P.k ? wt : 0.0;
        s1lo = std::min(s1lo, e.s1);
        s1hi = std::max(s1hi, e.s1);
        s2lo = std::min(s2lo, e.s2);
        s2hi = std::max(s2hi, e.s2);
        tab[size_t(j - 1) * P.LL + size_t(l1) * p.L + l2] = e;
      }
    }
    P.s1min[j - 1] = s1lo;
    P.s1max[j - 1] = s1hi;
    P.s2min[j - 1] = s2lo;
    P.s2max[j - 1] = s2hi;
  }
}

}  // namespace bsde

struct bsde2_plan_s {
  bsde2_problem prob;
  bsde::Params2 P;
  bsde::Layout2 lay;
  int device;
  unsigned char *ws;
  cudaGraphExec_t graph[2];  // [closed-form start, imported start]
  int64_t launches;
  bsde::Stats2 *host_stats;  // pinned
};

namespace bsde {

static void launch2_step(bsde2_plan_t *pl, cudaStream_t s, int n) {
  const Params2 &P = pl->P;
  const unsigned blocks = unsigned((P.Np + kStep2TP - 1) / kStep2TP);
  launch_pdl(k2_step, blocks, unsigned(kStep2TP * P.G), 0, s, P,
             reinterpret_cast<const double4_32a *>(pl->ws + pl->lay.ring),
             reinterpret_cast<double *>(pl->ws + pl->lay.vals),
             reinterpret_cast<const Node2 *>(pl->ws + pl->lay.table), n,
             reinterpret_cast<Stats *>(pl->ws + pl->lay.stats));
}

static void launch2_deriv(bsde2_plan_t *pl, cudaStream_t s, int slot) {
  const Params2 &P = pl->P;
  cudaLaunchConfig_t lc{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.gridDim = dim3(unsigned((P.Nx1 + kDerTX - 1) / kDerTX), unsigned((P.Nx2 + kDerTY - 1) / kDerTY), 1);
  lc.blockDim = dim3(kDerTX * kDerTY, 1, 1);
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaLaunchKernelEx(&lc, k2_deriv, P, reinterpret_cast<const double *>(pl->ws + pl->lay.vals),
                     reinterpret_cast<double4_32a *>(pl->ws + pl->lay.ring), slot);
}

static int64_t enqueue2_solve(bsde2_plan_t *pl, cudaStream_t s, bool imported) {
  const Params2 &P = pl->P;
  double *V = reinterpret_cast<double *>(pl->ws + pl->lay.vals);
  const double *stage = reinterpret_cast<const double *>(pl->ws + pl->lay.stage);
  const double4_32a *ring = reinterpret_cast<const double4_32a *>(pl->ws + pl->lay.ring);
  Stats2 *st = reinterpret_cast<Stats2 *>(pl->ws + pl->lay.stats);
  const unsigned eb = unsigned((P.Np + 255) / 256 < 4096 ? (P.Np + 255) / 256 : 4096);
  int64_t launches = 0;
  k2_reset_stats<<<1, 32, 0, s>>>(st);
  ++launches;
  for (int m = 0; m < P.k; ++m) {
    if (imported)
      k2_import<<<eb, 256, 0, s>>>(P, V, stage, m);
    else
      k2_init_closed<<<eb, 256, 0, s>>>(P, V, m);
    launch2_deriv(pl, s, (P.N - m) % P.nslot);
    launches += 2;
  }
  for (int n = P.N - P.k; n >= 0; --n) {
    launch2_step(pl, s, n);
    launch2_deriv(pl, s, n % P.nslot);
    launches += 2;
  }
  k2_readout<<<1, 32, 0, s>>>(P, ring, 0, st);
  // level 0 into the staging area (its first 3 planes)
  k2_export<<<eb, 256, 0, s>>>(P, ring, 0, reinterpret_cast<double *>(pl->ws + pl->lay.stage));
  launches += 2;
  return launches;
}

static int build2_graph(bsde2_plan_t *pl, int which) {
  cudaStream_t cs;
  BSDE_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(BSDE_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  }
  const int64_t n = enqueue2_solve(pl, cs, which == 1);
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(BSDE_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&pl->graph[which], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return fail(BSDE_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  pl->launches = n;
  return BSDE_OK;
}

static int fill2_result(bsde2_plan_t *pl, bsde2_result *r) {
  const Stats2 &s = *pl->host_stats;
  r->y0 = s.s.y0;
  r->z0[0] = s.s.z0;
  r->z0[1] = s.z0b;
  double d;
  unsigned long long b = s.s.resid_bits;
  std::memcpy(&d, &b, sizeof(d));
  r->picard_resid_max = d;
  r->picard_iters_max = s.s.iters_max;
  r->levels_done = pl->P.N - pl->P.k + 1;
  r->status = s.s.nonconv ? BSDE_WARN_NOCONV : BSDE_OK;
  return r->status;
}

}  // namespace bsde

extern "C" {

int bsde2_workspace_bytes(const bsde2_problem *p, size_t *bytes) {
  if (!p || !bytes) return bsde::fail(BSDE_EINVAL, "null argument");
  if (bsde::validate2(*p)) return bsde::fail(BSDE_EINVAL, "invalid 2-D problem");
  *bytes = bsde::layout2(*p).total;
  return BSDE_OK;
}

int bsde2_plan(const bsde2_problem *p, void *dev_workspace, size_t bytes, bsde2_plan_t **out) {
  using namespace bsde;
  if (!p || !out) return fail(BSDE_EINVAL, "null argument");
  *out = nullptr;
  if (validate2(*p)) return fail(BSDE_EINVAL, "invalid 2-D problem");
  const Layout2 lay = layout2(*p);
  if (!dev_workspace || bytes < lay.total)
    return fail(BSDE_ENOSPC, "workspace smaller than bsde2_workspace_bytes()");
  if (reinterpret_cast<uintptr_t>(dev_workspace) % 256)
    return fail(BSDE_EINVAL, "workspace must be 256-byte aligned");
  bsde2_plan_t *pl = new (std::nothrow) bsde2_plan_t();
  if (!pl) return fail(BSDE_ENOMEM, "plan allocation");
  pl->prob = *p;
  pl->lay = lay;
  cudaGetDevice(&pl->device);
  pl->ws = static_cast<unsigned char *>(dev_workspace);
  std::vector<Node2> tab;
  plan2_constants(*p, pl->P, tab, resident_step_threads(pl->device));
  cudaError_t e = cudaMemcpy(pl->ws + lay.table, tab.data(), sizeof(Node2) * tab.size(),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMallocHost(&pl->host_stats, sizeof(Stats2));
  if (e != cudaSuccess) {
    delete pl;
    return fail(BSDE_ECUDA, std::string("plan: ") + cudaGetErrorString(e));
  }
  *out = pl;
  return BSDE_OK;
}

int bsde2_solve(bsde2_plan_t *pl, void *stream, const double *init_y, const double *init_z1,
                const double *init_z2, int init_on_host, double *out_y, double *out_z1,
                double *out_z2, int out_on_host, bsde2_result *result) {
  using namespace bsde;
  if (!pl) return fail(BSDE_EINVAL, "null plan");
  const bool any = init_y || init_z1 || init_z2, all = init_y && init_z1 && init_z2;
  if (any && !all) return fail(BSDE_EINVAL, "give all three initial fields or none");
  DeviceGuard guard(pl->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Params2 &P = pl->P;
  const int which = all ? 1 : 0;
  if (!pl->graph[which]) {
    int rc = build2_graph(pl, which);
    if (rc) return rc;
  }
  double *stage = reinterpret_cast<double *>(pl->ws + pl->lay.stage);
  const size_t plane = size_t(P.Np) * sizeof(double), lev = plane * size_t(P.k);
  if (all) {
    const cudaMemcpyKind kind = init_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const double *src[3] = {init_y, init_z1, init_z2};
    for (int f = 0; f < 3; ++f)
      BSDE_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<unsigned char *>(stage) + f * lev, src[f],
                                    lev, kind, s));
  }
  BSDE_CUDA_TRY(cudaGraphLaunch(pl->graph[which], s));
  const cudaMemcpyKind okind = out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  double *outs[3] = {out_y, out_z1, out_z2};
  for (int f = 0; f < 3; ++f)
    if (outs[f]) BSDE_CUDA_TRY(cudaMemcpyAsync(outs[f], stage + f * P.Np, plane, okind, s));
  BSDE_CUDA_TRY(cudaMemcpyAsync(pl->host_stats, pl->ws + pl->lay.stats, sizeof(Stats2),
                                cudaMemcpyDeviceToHost, s));
  const bool host_ptrs = (all && init_on_host) || ((out_y || out_z1 || out_z2) && out_on_host);
  if (result || host_ptrs) BSDE_CUDA_TRY(cudaStreamSynchronize(s));
  if (result) return fill2_result(pl, result);
  return BSDE_OK;
}

int bsde2_result_fetch(bsde2_plan_t *pl, void *stream, bsde2_result *result) {
  using namespace bsde;
  if (!pl || !result) return fail(BSDE_EINVAL, "null argument");
  DeviceGuard guard(pl->device);
  BSDE_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return fill2_result(pl, result);
}

int bsde2_enqueue_level(bsde2_plan_t *pl, void *stream, int n, int parts) {
  using namespace bsde;
  if (!pl) return fail(BSDE_EINVAL, "null plan");
  if (n < 0 || n > pl->P.N - pl->P.k) return fail(BSDE_EINVAL, "level out of range");
  DeviceGuard guard(pl->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (parts & 1) launch2_step(pl, s, n);
  if (parts & 2) launch2_deriv(pl, s, n % pl->P.nslot);
  BSDE_CUDA_TRY(cudaGetLastError());
  return BSDE_OK;
}

int64_t bsde2_plan_launches(const bsde2_plan_t *pl) {
  if (!pl) return 0;
  const bsde::Params2 &P = pl->P;
  return 1 + 2 * int64_t(P.k) + 2 * int64_t(P.N - P.k + 1) + 2;
}

void bsde2_free(bsde2_plan_t *pl) {
  if (!pl) return;
  bsde::DeviceGuard guard(pl->device);
  for (int w = 0; w < 2; ++w)
    if (pl->graph[w]) cudaGraphExecDestroy(pl->graph[w]);
  if (pl->host_stats) cudaFreeHost(pl->host_stats);
  delete pl;
}

}  // extern "C"
