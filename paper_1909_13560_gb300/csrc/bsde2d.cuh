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
  int32_t N, k, L, LL, nslot, picard_max, terminal, precision;
  float picard_tol_f, alpha_f, beta1_f, beta2_f, hg0_f, pad_f[3];
  double T, dt, dx1, dx2, x1_min, x1_max, x2_min, x2_max, x01, x02;
  double a1, a2, b11, b21, b22, alpha, beta1, beta2, picard_tol;
  double gy[kMaxK + 1], gz[kMaxK + 1];
  double h, hg0;
  // work split: S chunks of Lg nodes per j, G = k S groups per point;
  // per j the range of cell shifts in each dimension (clamp-free fast path)
  int32_t S, Lg, G, LLp;  // LLp = ceil(L^2 / 2) mirror pairs (FP32C)
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

// FP32C pair entry (112 B): tensor nodes a = (l1, l2) and b = (L-1-l1,
// L-1-l2) mirror each other (DeltaW_b = -DeltaW_a, equal weight), so the pair
// is processed together: the two values' hi parts are added exactly before
// one compensated product, and the driver terms enter as cfz (F_a - F_b) and
// cfy (F_a + F_b), whose FP32 rounding scales with the small difference
// rather than with F.  Per node the cell shift and the Hermite basis of theta
// in each dimension; weights as floats (cz, cy split hi + lo).  The middle
// node of an odd L pairs with itself at half weight.
struct Node2f {
  int32_t s1a, s2a, s1b, s2b;
  float h1a[4], h2a[4], h1b[4], h2b[4];
  float czh, czl, cyh, cyl;
  float cfz1, cfz2, cfy, pad;
};

// FP32C level record of a grid point (64 B, four float4): the three fields'
// values as float pairs hi + lo and their scaled derivatives as floats
//   V0 = (y_hi, z1_hi, z2_hi, y_lo)       V1 = (z1_lo, z2_lo, y_fx, z1_fx)
//   V2 = (z2_fx, y_fy, z1_fy, z2_fy)      V3 = (y_fxy, z1_fxy, z2_fxy, 0)
// The ring keeps the four float4 of a record in four planes of Np entries
// per level (a warp's 16-byte loads of one plane are then contiguous).
struct Rec2f {
  float4 v0, v1, v2, v3;
};
struct Lev2f {
  const float4 *p0, *p1, *p2, *p3;
};
__host__ __device__ inline Lev2f lev2f(const float4 *ring, int64_t Np, int slot) {
  const float4 *b = ring + int64_t(slot) * 4 * Np;
  return Lev2f{b, b + Np, b + 2 * Np, b + 3 * Np};
}
__device__ __forceinline__ Rec2f load_rec(const Lev2f &L, int64_t q) {
  return Rec2f{L.p0[q], L.p1[q], L.p2[q], L.p3[q]};
}

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

// The new-value plane V holds the three fields of a new level (y, z1, z2;
// Np entries each, i1 fastest): doubles in FP64, float pairs (hi, lo) with
// |lo| <= ulp(hi)/2 in FP32C (the same 8 bytes per entry), so that the FP32C
// derivative kernel needs no FP64 arithmetic.
__device__ __forceinline__ void put_v(const Params2 &P, double *V, int f, int64_t q, double x) {
  if (P.precision == BSDE_FP32C) {
    const float h = __double2float_rn(x);
    reinterpret_cast<float2 *>(V)[f * P.Np + q] =
        make_float2(h, __double2float_rn(__dsub_rn(x, double(h))));
  } else {
    V[f * P.Np + q] = x;
  }
}

// Level values of the closed form at t_{N-m} into V.
__global__ void k2_init_closed(const Params2 P, double *V, int m) {
  const double t = __dmul_rn(double(P.N - m), P.dt);
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < P.Np;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i1 = q % P.Nx1, i2 = q / P.Nx1;
    double u, z1, z2;
    closed_form2(P, t, P.x1_min + double(i1) * P.dx1, P.x2_min + double(i2) * P.dx2, u, z1, z2);
    put_v(P, V, 0, q, u);
    put_v(P, V, 1, q, z1);
    put_v(P, V, 2, q, z2);
  }
}

// Level m of the caller's initial levels (staging area: y, z1, z2 planes of
// k levels each) into V.
__global__ void k2_import(const Params2 P, double *V, const double *stage, int m) {
  const int64_t kp = int64_t(P.k) * P.Np;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < P.Np;
       q += int64_t(gridDim.x) * blockDim.x) {
    for (int f = 0; f < 3; ++f) put_v(P, V, f, q, stage[f * kp + int64_t(m) * P.Np + q]);
  }
}

// y^n = A + delta of the FP32C tails as a float pair (TwoSum: A's hi part
// need not dominate when y^n is near zero), and z as the exact pairs.
__device__ __forceinline__ void put_new32(const Params2 &P, double *V, int64_t q, float Ah,
                                          float Al, float dl, float z1h, float z1l, float z2h,
                                          float z2l) {
  float yh = Ah, yl = 0.f;
  two_sum_into(yh, yl, __fadd_rn(Al, dl));  // yl: the exact error, |yl| <= ulp(yh)/2
  float2 *V2 = reinterpret_cast<float2 *>(V);
  V2[q] = make_float2(yh, yl);
  V2[P.Np + q] = make_float2(z1h, z1l);
  V2[2 * P.Np + q] = make_float2(z2h, z2l);
}

// ---------------------------------------------------------------------------
// Derivatives of a new level (Section 3.3): fourth-order finite differences
// of the three fields, scaled by the spacings, into the ring slot as
// double4 (v, dx1 v_x1, dx2 v_x2, dx1 dx2 v_x1x2) per field and point.
// One CTA per kDerTX x kDerTY tile; the tile and a halo of 4 in each
// direction (the one-sided stencils reach 4 nodes) staged in shared memory.
// ---------------------------------------------------------------------------
// (a product with the rounded 1/12 instead of a division: FP64 division is a
// multi-instruction sequence on the FP64 pipe, which bounds this kernel)
constexpr double kInv12 = 1.0 / 12.0;
__device__ __forceinline__ double fd4(const double *f, int s, int i, int n) {
  // f points at node i of a line (stride s); n nodes on the line
  if (i >= 2 && i <= n - 3)
    return (f[-2 * s] - 8.0 * f[-s] + 8.0 * f[s] - f[2 * s]) * kInv12;
  if (i < 2)
    return (-25.0 * f[0] + 48.0 * f[s] - 36.0 * f[2 * s] + 16.0 * f[3 * s] - 3.0 * f[4 * s]) *
           kInv12;
  return (25.0 * f[0] - 48.0 * f[-s] + 36.0 * f[-2 * s] - 16.0 * f[-3 * s] + 3.0 * f[-4 * s]) *
         kInv12;
}

// The same differences in FP32 on values given as float pairs hi + lo: the
// stencil's weights sum to zero, so it is written over the increments
// f_m - f_0 = (hi_m - hi_0) + (lo_m - lo_0), whose FP32 rounding is relative
// to the increment, and the result is the stored float derivative.
// (LO false: plain float values, l unused)
template <bool LO>
__device__ __forceinline__ float dinc(const float *h, const float *l, int a, int b) {
  return LO ? __fadd_rn(__fsub_rn(h[a], h[b]), __fsub_rn(l[a], l[b])) : __fsub_rn(h[a], h[b]);
}
template <bool LO>
__device__ __forceinline__ float fd4f(const float *h, const float *l, int s, int i, int n) {
  const float c12 = float(1.0 / 12.0);
  if (i >= 2 && i <= n - 3)
    return __fmul_rn(__fmaf_rn(8.f, dinc<LO>(h, l, s, -s), dinc<LO>(h, l, -2 * s, 2 * s)), c12);
  if (i < 2) {
    float t = __fmul_rn(48.f, dinc<LO>(h, l, s, 0));
    t = __fmaf_rn(-36.f, dinc<LO>(h, l, 2 * s, 0), t);
    t = __fmaf_rn(16.f, dinc<LO>(h, l, 3 * s, 0), t);
    t = __fmaf_rn(-3.f, dinc<LO>(h, l, 4 * s, 0), t);
    return __fmul_rn(t, c12);
  }
  float t = __fmul_rn(48.f, dinc<LO>(h, l, 0, -s));
  t = __fmaf_rn(-36.f, dinc<LO>(h, l, 0, -2 * s), t);
  t = __fmaf_rn(16.f, dinc<LO>(h, l, 0, -3 * s), t);
  t = __fmaf_rn(-3.f, dinc<LO>(h, l, 0, -4 * s), t);
  return __fmul_rn(t, c12);
}

__global__ void __launch_bounds__(kDerTX * kDerTY)
    k2_deriv(const Params2 P, const double *__restrict__ V, double4_32a *__restrict__ ring,
             int slot) {
  constexpr int W = kDerTX + 2 * kDerH, H = kDerTY + 2 * kDerH;
  __shared__ double sv[H][W];
  __shared__ double sy[kDerTY][W];
  wait_predecessor();
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kDerTX;
  // rows of tiles beyond the grid's y extent (65535) taken in turn
  for (int ty = blockIdx.y; ty * kDerTY < n2; ty += gridDim.y) {
    const int y0 = ty * kDerTY;
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
      if (d <= P.picard_tol || !isfinite(d)) break;  // a non-finite step cannot converge
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
// FP32C form of the 2-D path.  A bicubic value is kept as hi_00 + del: the
// corner (c1, c2)'s value hi part plus, in FP32, the increments of the other
// corners' values over it (the value weights sum to one), the corner's lo
// part and the derivative terms -- all of size dx |grad v|, so their
// rounding is far below that of the value.  The expectations take the exact
// product of the weight's hi part with hi_00 (FMA error term) and add it by
// TwoSum (comp_acc1); the driver terms are summed in plain FP32; z^n and A
// are formed as float pairs and y^n by Picard on the increment, as in the 1-D
// FP32C step.  Derivatives of a new level: the fourth-order differences in
// FP32 over the new values split into float pairs (fd4f).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kDerTX * kDerTY)
    k2_deriv32(const Params2 P, const double *__restrict__ V, float4 *__restrict__ ring,
               int slot) {
  constexpr int W = kDerTX + 2 * kDerH, H = kDerTY + 2 * kDerH;
  __shared__ float sh[H][W], sl[H][W];
  __shared__ float sy[kDerTY][W];
  wait_predecessor();
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kDerTX;
  // rows of tiles beyond the grid's y extent (65535) taken in turn
  for (int ty = blockIdx.y; ty * kDerTY < n2; ty += gridDim.y) {
    const int y0 = ty * kDerTY;
    // one point per thread (kDerTX * kDerTY threads)
    const int r = tid / kDerTX, c = tid % kDerTX;
    const int i1 = x0 + c, i2 = y0 + r;
    float hi[3], lo[3], fx[3], fy[3], fxy[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const float2 *v = reinterpret_cast<const float2 *>(V) + int64_t(f) * P.Np;
      for (int e = tid; e < H * W; e += blockDim.x) {
        const int rr = e / W, cc = e % W;
        int g2 = y0 - kDerH + rr, g1 = x0 - kDerH + cc;
        g2 = g2 < 0 ? 0 : (g2 >= n2 ? n2 - 1 : g2);
        g1 = g1 < 0 ? 0 : (g1 >= n1 ? n1 - 1 : g1);
        const float2 x = v[int64_t(g2) * n1 + g1];
        sh[rr][cc] = x.x;
        sl[rr][cc] = x.y;
      }
      __syncthreads();
      // x2 derivative on the tile's rows, every column of the staged span
      for (int e = tid; e < kDerTY * W; e += blockDim.x) {
        const int rr = e / W, cc = e % W;
        const int j2 = y0 + rr;
        sy[rr][cc] = j2 < n2 ? fd4f<true>(&sh[rr + kDerH][cc], &sl[rr + kDerH][cc], W, j2, n2) : 0.f;
      }
      __syncthreads();
      hi[f] = lo[f] = fx[f] = fy[f] = fxy[f] = 0.f;
      if (i1 < n1 && i2 < n2) {
        hi[f] = sh[r + kDerH][c + kDerH];
        lo[f] = sl[r + kDerH][c + kDerH];
        fx[f] = fd4f<true>(&sh[r + kDerH][c + kDerH], &sl[r + kDerH][c + kDerH], 1, i1, n1);
        fy[f] = sy[r][c + kDerH];
        fxy[f] = fd4f<false>(&sy[r][c + kDerH], nullptr, 1, i1, n1);
      }
      __syncthreads();
    }
    if (i1 < n1 && i2 < n2) {
      float4 *b = ring + int64_t(slot) * 4 * P.Np + int64_t(i2) * n1 + i1;
      b[0] = make_float4(hi[0], hi[1], hi[2], lo[0]);
      b[P.Np] = make_float4(lo[1], lo[2], fx[0], fx[1]);
      b[2 * P.Np] = make_float4(fx[2], fy[0], fy[1], fy[2]);
      b[3 * P.Np] = make_float4(fxy[0], fxy[1], fxy[2], 0.f);
    }
  }
}

// hi_00 and del of one field from the four corner records (see Rec2f);
// w: W10 W01 W11 | X00 X10 X01 X11 | Y00 Y10 Y01 Y11 | Z00 Z10 Z01 Z11
__device__ __forceinline__ void field2f(float h00, float l00, float h10, float l10, float h01,
                                        float l01, float h11, float l11, float4 fx, float4 fy,
                                        float4 fxy, const float *w, float &hi, float &del) {
  const float d10 = __fadd_rn(__fsub_rn(h10, h00), __fsub_rn(l10, l00));
  const float d01 = __fadd_rn(__fsub_rn(h01, h00), __fsub_rn(l01, l00));
  const float d11 = __fadd_rn(__fsub_rn(h11, h00), __fsub_rn(l11, l00));
  float s = l00;
  s = __fmaf_rn(d10, w[0], s);
  s = __fmaf_rn(d01, w[1], s);
  s = __fmaf_rn(d11, w[2], s);
  s = __fmaf_rn(fx.x, w[3], s);
  s = __fmaf_rn(fx.y, w[4], s);
  s = __fmaf_rn(fx.z, w[5], s);
  s = __fmaf_rn(fx.w, w[6], s);
  s = __fmaf_rn(fy.x, w[7], s);
  s = __fmaf_rn(fy.y, w[8], s);
  s = __fmaf_rn(fy.z, w[9], s);
  s = __fmaf_rn(fy.w, w[10], s);
  s = __fmaf_rn(fxy.x, w[11], s);
  s = __fmaf_rn(fxy.y, w[12], s);
  s = __fmaf_rn(fxy.z, w[13], s);
  s = __fmaf_rn(fxy.w, w[14], s);
  hi = h00;
  del = s;
}

struct Acc2f {
  float Sy, Cy, S1, C1, S2, C2, Fy, F1, F2, FyC;  // Fy + FyC: the y driver terms (TwoSum)
};

// The bicubic value (hi, del) of the three fields at one node, from its cell
// shift and Hermite basis (clamped onto the box in CLAMP mode).
template <bool CLAMP>
__device__ __forceinline__ void node2f_values(const Params2 &P, const Lev2f &lev,
                                              int i1, int i2, int s1, int s2, const float *h1in,
                                              const float *h2in, float *hi, float *del) {
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  int c1 = i1 + s1, c2 = i2 + s2;
  float h1[4], h2[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    h1[u] = h1in[u];
    h2[u] = h2in[u];
  }
  if (CLAMP) {
    if (c1 < 0 || c1 > n1 - 2) {
      const bool lo = c1 < 0;
      c1 = lo ? 0 : n1 - 2;
      h1[0] = lo ? 1.f : 0.f;
      h1[1] = lo ? 0.f : 1.f;
      h1[2] = h1[3] = 0.f;
    }
    if (c2 < 0 || c2 > n2 - 2) {
      const bool lo = c2 < 0;
      c2 = lo ? 0 : n2 - 2;
      h2[0] = lo ? 1.f : 0.f;
      h2[1] = lo ? 0.f : 1.f;
      h2[2] = h2[3] = 0.f;
    }
  }
  float w[15];
  w[0] = h1[1] * h2[0];
  w[1] = h1[0] * h2[1];
  w[2] = h1[1] * h2[1];
  w[3] = h1[2] * h2[0];
  w[4] = h1[3] * h2[0];
  w[5] = h1[2] * h2[1];
  w[6] = h1[3] * h2[1];
  w[7] = h1[0] * h2[2];
  w[8] = h1[1] * h2[2];
  w[9] = h1[0] * h2[3];
  w[10] = h1[1] * h2[3];
  w[11] = h1[2] * h2[2];
  w[12] = h1[3] * h2[2];
  w[13] = h1[2] * h2[3];
  w[14] = h1[3] * h2[3];
  const int64_t q00 = int64_t(c2) * n1 + c1;
  const Rec2f A = load_rec(lev, q00), Bq = load_rec(lev, q00 + 1), C = load_rec(lev, q00 + n1),
              D = load_rec(lev, q00 + n1 + 1);
  field2f(A.v0.x, A.v0.w, Bq.v0.x, Bq.v0.w, C.v0.x, C.v0.w, D.v0.x, D.v0.w,
          make_float4(A.v1.z, Bq.v1.z, C.v1.z, D.v1.z), make_float4(A.v2.y, Bq.v2.y, C.v2.y, D.v2.y),
          make_float4(A.v3.x, Bq.v3.x, C.v3.x, D.v3.x), w, hi[0], del[0]);
  field2f(A.v0.y, A.v1.x, Bq.v0.y, Bq.v1.x, C.v0.y, C.v1.x, D.v0.y, D.v1.x,
          make_float4(A.v1.w, Bq.v1.w, C.v1.w, D.v1.w), make_float4(A.v2.z, Bq.v2.z, C.v2.z, D.v2.z),
          make_float4(A.v3.y, Bq.v3.y, C.v3.y, D.v3.y), w, hi[1], del[1]);
  field2f(A.v0.z, A.v1.y, Bq.v0.z, Bq.v1.y, C.v0.z, C.v1.y, D.v0.z, D.v1.y,
          make_float4(A.v2.x, Bq.v2.x, C.v2.x, D.v2.x), make_float4(A.v2.w, Bq.v2.w, C.v2.w, D.v2.w),
          make_float4(A.v3.z, Bq.v3.z, C.v3.z, D.v3.z), w, hi[2], del[2]);
}

template <bool CLAMP>
__device__ __forceinline__ void nodes2f(const Params2 &P, const Lev2f &lev,
                                        const Node2f *row, int q0, int q1, int i1, int i2,
                                        bool yj, Acc2f &a) {
#pragma unroll 1
  for (int q = q0; q < q1; ++q) {
    const Node2f &e = row[q];
    float ha[3], da[3], hb[3], db[3];
    node2f_values<CLAMP>(P, lev, i1, i2, e.s1a, e.s2a, e.h1a, e.h2a, ha, da);
    node2f_values<CLAMP>(P, lev, i1, i2, e.s1b, e.s2b, e.h1b, e.h2b, hb, db);
    const float Fa = __fmaf_rn(P.alpha_f, __fadd_rn(ha[0], da[0]),
                               __fmaf_rn(P.beta1_f, __fadd_rn(ha[1], da[1]),
                                         __fmul_rn(P.beta2_f, __fadd_rn(ha[2], da[2]))));
    const float Fb = __fmaf_rn(P.alpha_f, __fadd_rn(hb[0], db[0]),
                               __fmaf_rn(P.beta1_f, __fadd_rn(hb[1], db[1]),
                                         __fmul_rn(P.beta2_f, __fadd_rn(hb[2], db[2]))));
    // F_a - F_b of the linear driver from the fields' differences: the hi
    // parts of neighbouring values subtract exactly, so the difference keeps
    // the accuracy of its small size rather than inheriting F's rounding
    float dv[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) dv[f] = __fadd_rn(__fsub_rn(ha[f], hb[f]), __fsub_rn(da[f], db[f]));
    const float dF = __fmaf_rn(P.alpha_f, dv[0], __fmaf_rn(P.beta1_f, dv[1], __fmul_rn(P.beta2_f, dv[2])));
    a.F1 = __fmaf_rn(e.cfz1, dF, a.F1);
    a.F2 = __fmaf_rn(e.cfz2, dF, a.F2);
    // sum k dt gy_j E[f] reaches O(k dt |f|): accumulated with its error
    two_sum_into(a.Fy, a.FyC, __fmul_rn(e.cfy, __fadd_rn(Fa, Fb)));
    // the pair's hi parts summed exactly, then one compensated product
    float hs, he;
#pragma unroll
    for (int f = 1; f < 3; ++f) {
      hs = ha[f];
      he = 0.f;
      two_sum_into(hs, he, hb[f]);
      const float dd = __fadd_rn(__fadd_rn(da[f], db[f]), he);
      if (f == 1)
        comp_acc1(a.S1, a.C1, e.czh, e.czl, hs, dd);
      else
        comp_acc1(a.S2, a.C2, e.czh, e.czl, hs, dd);
    }
    if (yj) {
      hs = ha[0];
      he = 0.f;
      two_sum_into(hs, he, hb[0]);
      comp_acc1(a.Sy, a.Cy, e.cyh, e.cyl, hs, __fadd_rn(__fadd_rn(da[0], db[0]), he));
    }
  }
}

// One tile of kStep2TP points of level n, by every thread of the CTA: `tab`
// is the pair table (in shared memory or in the kernel's parameters), `part`
// the groups' partial sums in shared memory.
__device__ __forceinline__ void step2_tile32(const Params2 &P, const float4 *__restrict__ ring,
                                             double *__restrict__ V, const Node2f *tab,
                                             float *part, int n, Stats *st) {
  const int tp = threadIdx.x % kStep2TP, g = threadIdx.x / kStep2TP;
  const int64_t q0p = int64_t(blockIdx.x) * kStep2TP;
  const int64_t qq = q0p + tp;
  const bool active = qq < P.Np;
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  Acc2f a{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // the Picard start y^{n+1} of this thread's point, loaded early
  float prev_h = 0.f, prev_l = 0.f;
  if (g == 0 && active) {
    const float4 v0 = lev2f(ring, P.Np, (n + 1) % P.nslot).p0[qq];
    prev_h = v0.x;
    prev_l = v0.w;
  }
  if (active) {
    const int j = g / P.S + 1, lc = g % P.S;
    const int a0 = lc * P.Lg, a1 = a0 + P.Lg < P.LLp ? a0 + P.Lg : P.LLp;
    const int i1 = int(qq % n1), i2 = int(qq / n1);
    const int64_t qe = (q0p + kStep2TP <= P.Np ? q0p + kStep2TP : P.Np) - 1;
    const int r0 = int(q0p / n1), r1 = int(qe / n1);
    const int cmin = r0 == r1 ? int(q0p % n1) : 0, cmax = r0 == r1 ? int(qe % n1) : n1 - 1;
    const bool interior = cmin + P.s1min[j - 1] >= 0 && cmax + P.s1max[j - 1] <= n1 - 2 &&
                          r0 + P.s2min[j - 1] >= 0 && r1 + P.s2max[j - 1] <= n2 - 2;
    const Lev2f lev = lev2f(ring, P.Np, (n + j) % P.nslot);
    const Node2f *row = tab + (j - 1) * P.LLp;
    if (interior)
      nodes2f<false>(P, lev, row, a0, a1, i1, i2, j == P.k, a);
    else
      nodes2f<true>(P, lev, row, a0, a1, i1, i2, j == P.k, a);
  }
  const int G = P.G, gs = G * kStep2TP, o = g * kStep2TP + tp;
  part[0 * gs + o] = a.Sy;
  part[1 * gs + o] = a.Cy;
  part[2 * gs + o] = a.S1;
  part[3 * gs + o] = a.C1;
  part[4 * gs + o] = a.S2;
  part[5 * gs + o] = a.C2;
  part[6 * gs + o] = a.Fy;
  part[7 * gs + o] = a.F1;
  part[8 * gs + o] = a.F2;
  part[9 * gs + o] = a.FyC;
  __syncthreads();
  if (g != 0) return;
  int it = 0;
  float d = 0.f;
  if (active) {
    float yS = 0.f, yC = 0.f, z1S = 0.f, z1C = 0.f, z2S = 0.f, z2C = 0.f, fy = 0.f, f1 = 0.f,
          f2 = 0.f, fyC = 0.f;
    for (int u = 0; u < G; ++u) {
      const int ou = u * kStep2TP + tp;
      two_sum_into(yS, yC, part[0 * gs + ou]);
      yC = __fadd_rn(yC, part[1 * gs + ou]);
      two_sum_into(z1S, z1C, part[2 * gs + ou]);
      z1C = __fadd_rn(z1C, part[3 * gs + ou]);
      two_sum_into(z2S, z2C, part[4 * gs + ou]);
      z2C = __fadd_rn(z2C, part[5 * gs + ou]);
      two_sum_into(fy, fyC, part[6 * gs + ou]);
      fyC = __fadd_rn(fyC, part[9 * gs + ou]);
      f1 = __fadd_rn(f1, part[7 * gs + ou]);
      f2 = __fadd_rn(f2, part[8 * gs + ou]);
    }
    // z_d = S + (C + F) and A = S + (C + F) as exact float pairs
    float z1h = z1S, z1l = 0.f, z2h = z2S, z2l = 0.f, Ah = yS, Al = 0.f;
    two_sum_into(z1h, z1l, __fadd_rn(z1C, f1));
    two_sum_into(z2h, z2l, __fadd_rn(z2C, f2));
    two_sum_into(Ah, Al, fy);
    two_sum_into(Ah, Al, __fadd_rn(yC, fyC));
    const float zlin = __fmaf_rn(P.beta1_f, z1h, __fmul_rn(P.beta2_f, z2h));
    // Picard on the increment delta = y^n - A: delta = hg0 f(A + delta, z)
    float dl = __fadd_rn(__fsub_rn(prev_h, Ah), __fsub_rn(prev_l, Al));
    float dpp = __int_as_float(0x7fc00000);
    while (it < P.picard_max) {
      const float dn = __fmul_rn(P.hg0_f, __fmaf_rn(P.alpha_f, __fadd_rn(Ah, dl), zlin));
      ++it;
      d = fabsf(__fsub_rn(dn, dl));
      const bool cyc = dn == dpp && picard_cycle_ok(d, __fadd_rn(Ah, dl), dn);
      dpp = dl;
      dl = dn;
      if (cyc) d = 0.f;
      if (d <= P.picard_tol_f || !isfinite(d)) break;  // a non-finite step cannot converge
    }
    put_new32(P, V, qq, Ah, Al, dl, z1h, z1l, z2h, z2l);
  }
  record_picard32(st, active, it, d, P.picard_tol_f);
}

// The FP32C 2-D step with the pair table copied into shared memory by every
// CTA (tables beyond the parameter capacity below).
__global__ void __launch_bounds__(kStep2TP * kMaxGroups, 1)
    k2_step32(const Params2 P, const float4 *__restrict__ ring, double *__restrict__ V,
              const Node2f *__restrict__ table, int n, Stats *st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int kLL = P.k * P.LLp;
  Node2f *tab = reinterpret_cast<Node2f *>(smem_raw);
  float *part = reinterpret_cast<float *>(tab + kLL);  // [10][G][kStep2TP]
  {
    const float4 *src = reinterpret_cast<const float4 *>(table);
    float4 *dst = reinterpret_cast<float4 *>(tab);
    const int nv = kLL * int(sizeof(Node2f) / 16);
    for (int t = threadIdx.x; t < nv; t += blockDim.x) dst[t] = src[t];
  }
  __syncthreads();
  wait_predecessor();
  step2_tile32(P, ring, V, tab, part, n, st);
}

// The pair table as a kernel parameter (up to K = 6 with L <= 8, the
// paper's 2-D settings): a group's threads read the same entry, so it comes
// through the constant cache and leaves the L1 data path to the level
// records.
constexpr int kPairTab2Cap = kMaxK * 32;
struct PairTab2 {
  Node2f e[kPairTab2Cap];
};
static_assert(sizeof(Params2) + sizeof(PairTab2) + 32 <= 32764,
              "k2_step32p parameters exceed the kernel parameter limit");

__global__ void __launch_bounds__(kStep2TP * kMaxGroups, 1)
    k2_step32p(const Params2 P, const float4 *__restrict__ ring, double *__restrict__ V,
               const __grid_constant__ PairTab2 tab, int n, Stats *st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float *part = reinterpret_cast<float *>(smem_raw);  // [10][G][kStep2TP]
  wait_predecessor();
  step2_tile32(P, ring, V, tab.e, part, n, st);
}

// ---------------------------------------------------------------------------
// The 2-D step as two tensor-product passes (linear driver, uncorrelated
// forward process b21 = 0).  A node's cell shift and Hermite basis then
// split into an x1 part of l1 and an x2 part of l2, and the weights of
// Eq. 20-21 into products of one-dimensional ones: wt = u_l1 u_l2,
// wt DeltaW1 = ua_l1 u_l2, wt DeltaW2 = u_l1 ua_l2 with u_l = omega_l /
// sqrt(pi) and ua_l = u_l a_l sqrt(2 j dt).  The bicubic value regroups as
//   v = h1_0 R(c1) + h1_1 R(c1+1) + h1_2 S(c1) + h1_3 S(c1+1),
// R(m1) = x2 interpolant of (v, dx2 v_x2) on column m1, S(m1) = that of
// (dx1 v_x1, dx1 dx2 v_x1x2), so every expectation the step needs is
//   pass 1 (x2): R_u, S_u = sum_l2 u_l2 (R, S at i2 + s2_l2), and R_a, S_a
//                with ua_l2, at every point and step j;
//   pass 2 (x1): E00[v] = sum_l1 u_l1 (h1 . (R_u, S_u) at i1 + s1_l1),
//                E10[v] with ua_l1, E01[v] = sum_l1 u_l1 (h1 . (R_a, S_a)).
// With f = alpha y + beta . z linear, E[f] and E[f DeltaW] are the same
// combinations of these, and the lines of Eq. 20 read
//   z1 = sum_j cz_j E00_j[z1] + cf_j E10_j[f],  z2 likewise with E01,
//   A  = sum_j cy_j E00_j[y] + cfy_j E00_j[f],
// cz_j = (delta_j1 - gz_j) / gz_0, cf_j = gz_j / gz_0, cy_j = [j = k],
// cfy_j = k dt gy_j.  Work per point and step: 48 L + 36 L multiply-adds
// against ~46 L^2 for the node-wise kernel.
// ---------------------------------------------------------------------------
struct TPTab2d {
  int32_t s1[kMaxK][kMaxL2], s2[kMaxK][kMaxL2];
  double h1[kMaxK][kMaxL2][4], h2[kMaxK][kMaxL2][4];
  double u[kMaxL2], ua[kMaxK][kMaxL2];
  double cz[kMaxK], cf[kMaxK], cy[kMaxK], cfy[kMaxK];
};
static_assert(sizeof(Params2) + sizeof(TPTab2d) + 64 <= 32764,
              "tensor-product tables exceed the kernel parameter limit");

// off the box: the value at the projection (theta 0 at the low end, 1 at the
// high end), as the node-wise kernels do it per dimension
template <typename T>
__device__ __forceinline__ void tp_clamp(int &c, int n, T *h) {
  if (c < 0 || c > n - 2) {
    const bool lo = c < 0;
    c = lo ? 0 : n - 2;
    h[0] = lo ? T(1) : T(0);
    h[1] = lo ? T(0) : T(1);
    h[2] = h[3] = T(0);
  }
}

constexpr int kTPThreads = 256;
constexpr int kTP1X = 32, kTP1Y = kTPThreads / kTP1X;  // FP32C x2-pass tile

// FP64 pass 1: per point and step j (blockIdx.y = j - 1), per field the
// double4 (R_u, S_u, R_a, S_a) into tp[((j - 1) * 3 + f) * Np + point].
__global__ void __launch_bounds__(kTPThreads)
    k2_tp1(const Params2 P, const double4_32a *__restrict__ ring, double4_32a *__restrict__ tp,
           const __grid_constant__ TPTab2d T, int n) {
  wait_predecessor();
  const int64_t qq = int64_t(blockIdx.x) * kTPThreads + threadIdx.x;
  const int jm = blockIdx.y;
  if (qq >= P.Np) return;
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  const int i1 = int(qq % n1), i2 = int(qq / n1);
  const double4_32a *lev = ring + int64_t((n + jm + 1) % P.nslot) * 3 * P.Np;
  double acc[3][4];
#pragma unroll
  for (int f = 0; f < 3; ++f) acc[f][0] = acc[f][1] = acc[f][2] = acc[f][3] = 0.0;
#pragma unroll 1
  for (int l = 0; l < P.L; ++l) {
    int c2 = i2 + T.s2[jm][l];
    double h[4] = {T.h2[jm][l][0], T.h2[jm][l][1], T.h2[jm][l][2], T.h2[jm][l][3]};
    tp_clamp(c2, n2, h);
    const int64_t o = int64_t(c2) * n1 + i1;
    const double u = T.u[l], ua = T.ua[jm][l];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const double4_32a a = lev[f * P.Np + o], c = lev[f * P.Np + o + n1];
      const double R = a.x * h[0] + c.x * h[1] + a.z * h[2] + c.z * h[3];
      const double S = a.y * h[0] + c.y * h[1] + a.w * h[2] + c.w * h[3];
      acc[f][0] += u * R;
      acc[f][1] += u * S;
      acc[f][2] += ua * R;
      acc[f][3] += ua * S;
    }
  }
#pragma unroll
  for (int f = 0; f < 3; ++f)
    tp[(int64_t(jm) * 3 + f) * P.Np + qq] =
        make_double4_32a(acc[f][0], acc[f][1], acc[f][2], acc[f][3]);
}

// FP64 pass 2 and the tail: the expectations of every step j, z^n, A and y^n
// by Picard (as k2_step), into the plane of new values V.
__global__ void __launch_bounds__(kTPThreads)
    k2_tp2(const Params2 P, const double4_32a *__restrict__ ring,
           const double4_32a *__restrict__ tp, double *__restrict__ V,
           const __grid_constant__ TPTab2d T, int n, Stats *st) {
  wait_predecessor();
  const int64_t qq = int64_t(blockIdx.x) * kTPThreads + threadIdx.x;
  const bool active = qq < P.Np;
  int it = 0;
  double d = 0.0;
  if (active) {
    const int n1 = int(P.Nx1);
    const int i1 = int(qq % n1), i2 = int(qq / n1);
    double z1 = 0.0, z2 = 0.0, A = 0.0;
    for (int jm = 0; jm < P.k; ++jm) {
      const double4_32a *tj = tp + int64_t(jm) * 3 * P.Np;
      double e00[3] = {0.0, 0.0, 0.0}, e10[3] = {0.0, 0.0, 0.0}, e01[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
      for (int l = 0; l < P.L; ++l) {
        int c1 = i1 + T.s1[jm][l];
        double h[4] = {T.h1[jm][l][0], T.h1[jm][l][1], T.h1[jm][l][2], T.h1[jm][l][3]};
        tp_clamp(c1, n1, h);
        const int64_t o = int64_t(i2) * n1 + c1;
        const double u = T.u[l], ua = T.ua[jm][l];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          const double4_32a a = tj[f * P.Np + o], b = tj[f * P.Np + o + 1];
          const double v = a.x * h[0] + b.x * h[1] + a.y * h[2] + b.y * h[3];
          const double va = a.z * h[0] + b.z * h[1] + a.w * h[2] + b.w * h[3];
          e00[f] += u * v;
          e10[f] += ua * v;
          e01[f] += u * va;
        }
      }
      const double F00 = P.alpha * e00[0] + P.beta1 * e00[1] + P.beta2 * e00[2];
      const double F10 = P.alpha * e10[0] + P.beta1 * e10[1] + P.beta2 * e10[2];
      const double F01 = P.alpha * e01[0] + P.beta1 * e01[1] + P.beta2 * e01[2];
      z1 += T.cz[jm] * e00[1] + T.cf[jm] * F10;
      z2 += T.cz[jm] * e00[2] + T.cf[jm] * F01;
      A += T.cy[jm] * e00[0] + T.cfy[jm] * F00;
    }
    double y = ring[(int64_t((n + 1) % P.nslot) * 3) * P.Np + qq].x;
    while (it < P.picard_max) {
      const double y1 = A + P.hg0 * (P.alpha * y + P.beta1 * z1 + P.beta2 * z2);
      d = fabs(y1 - y);
      y = y1;
      ++it;
      if (d <= P.picard_tol || !isfinite(d)) break;  // a non-finite step cannot converge
    }
    V[qq] = y;
    V[P.Np + qq] = z1;
    V[2 * P.Np + qq] = z2;
  }
  record_picard(st, active, it, d, P.picard_tol);
}

// FP32C tables: the Hermite bases as floats; pass 1 weights u and ua; pass 2
// weights per step with the multistep coefficients folded in: cz_j u, cy_j u,
// cfy_j u, cf_j ua, cf_j u.  Each weight but cfy_j u is a float pair (hi, lo):
// the lo part takes the weight's own rounding out of the sums, which would
// otherwise repeat identically at every point and level.  Nodes l and
// L-1-l mirror each other (u equal, ua opposite) and are taken as a pair; the
// middle node of an odd L stands alone.
struct TPTab2f {
  int32_t s1[kMaxK][kMaxL2], s2[kMaxK][kMaxL2];
  float h1[kMaxK][kMaxL2][4], h2[kMaxK][kMaxL2][4];
  float uh[kMaxL2], ul[kMaxL2], uah[kMaxK][kMaxL2], ual[kMaxK][kMaxL2];
  float czh[kMaxK][kMaxL2], czl[kMaxK][kMaxL2], cyh[kMaxK][kMaxL2], cyl[kMaxK][kMaxL2];
  float cfy[kMaxK][kMaxL2], cfah[kMaxK][kMaxL2], cfal[kMaxK][kMaxL2], cfuh[kMaxK][kMaxL2],
      cful[kMaxK][kMaxL2];
};
static_assert(sizeof(Params2) + sizeof(TPTab2f) + 64 <= 32764,
              "tensor-product tables exceed the kernel parameter limit");

// The x2 interpolants (value part hi + del, slope part) of the three fields
// at one node of pass 1, from the records of rows c2 (a) and c2 + 1 (c).
__device__ __forceinline__ void tp1_node32(const Rec2f &a, const Rec2f &c, const float *h,
                                           float *hi, float *del, float *sl) {
  // per field: hi, lo, dx1 v_x1, dx2 v_x2, dx1 dx2 v_x1x2 (see Rec2f)
  const float ah[3] = {a.v0.x, a.v0.y, a.v0.z}, al[3] = {a.v0.w, a.v1.x, a.v1.y};
  const float ch[3] = {c.v0.x, c.v0.y, c.v0.z}, cl[3] = {c.v0.w, c.v1.x, c.v1.y};
  const float afx[3] = {a.v1.z, a.v1.w, a.v2.x}, cfx[3] = {c.v1.z, c.v1.w, c.v2.x};
  const float afy[3] = {a.v2.y, a.v2.z, a.v2.w}, cfy[3] = {c.v2.y, c.v2.z, c.v2.w};
  const float afxy[3] = {a.v3.x, a.v3.y, a.v3.z}, cfxy[3] = {c.v3.x, c.v3.y, c.v3.z};
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    // h_0 + h_1 = 1: the value is the row-c2 value plus increments
    const float dv = __fadd_rn(__fsub_rn(ch[f], ah[f]), __fsub_rn(cl[f], al[f]));
    hi[f] = ah[f];
    del[f] = __fmaf_rn(h[3], cfy[f], __fmaf_rn(h[2], afy[f], __fmaf_rn(h[1], dv, al[f])));
    sl[f] = __fmaf_rn(h[3], cfxy[f],
                      __fmaf_rn(h[2], afxy[f], __fmaf_rn(h[1], cfx[f], __fmul_rn(h[0], afx[f]))));
  }
}

// FP32C pass 1: per point and step, the four float4 planes
//   W0 = (Ru_hi y, z1, z2, Ru_lo y)   W1 = (Ru_lo z1, z2, Su y, z1)
//   W2 = (Su z2, Ra y, z1, z2)        W3 = (Sa y, z1, z2, 0)
// R_u a compensated sum (float pair), the other three plain FP32 (slope
// terms, and the ua-weighted value differences of mirror nodes, all small).
__global__ void __launch_bounds__(kTPThreads)
    k2_tp1_32(const Params2 P, const float4 *__restrict__ ring, float4 *__restrict__ tp,
              const __grid_constant__ TPTab2f T, int n) {
  wait_predecessor();
  // a CTA takes a tile of kTP1X columns x kTP1Y rows, a warp one row: for a
  // node the warps read rows i2 + s2 and i2 + s2 + 1, so the tile's warps
  // share all but one of their rows through L1 (L2 traffic ~ (Y + 1) / 2Y
  // of one-row tiles')
  const int n1 = int(P.Nx1), n2 = int(P.Nx2);
  const int i1 = blockIdx.x * kTP1X + threadIdx.x % kTP1X;
  const int jm = blockIdx.z;
  if (i1 >= n1) return;
  // rows of tiles beyond the grid's y extent (65535) taken in turn
  for (int ty = blockIdx.y; ty * kTP1Y < n2; ty += gridDim.y) {
    const int i2 = ty * kTP1Y + threadIdx.x / kTP1X;
    if (i2 >= n2) continue;
    const int64_t qq = int64_t(i2) * n1 + i1;
    const Lev2f lev = lev2f(ring, P.Np, (n + jm + 1) % P.nslot);
    float RS[3] = {0.f, 0.f, 0.f}, RC[3] = {0.f, 0.f, 0.f}, Su[3] = {0.f, 0.f, 0.f},
          Ra[3] = {0.f, 0.f, 0.f}, Sa[3] = {0.f, 0.f, 0.f};
    const int L = P.L, Lh = P.L / 2;
#pragma unroll 1
    for (int q = 0; q < (L + 1) / 2; ++q) {
      const int la = q, lb = L - 1 - q;
      int ca = i2 + T.s2[jm][la], cb = i2 + T.s2[jm][lb];
      float ha[4] = {T.h2[jm][la][0], T.h2[jm][la][1], T.h2[jm][la][2], T.h2[jm][la][3]};
      float hb[4] = {T.h2[jm][lb][0], T.h2[jm][lb][1], T.h2[jm][lb][2], T.h2[jm][lb][3]};
      tp_clamp(ca, n2, ha);
      tp_clamp(cb, n2, hb);
      const int64_t oa = int64_t(ca) * n1 + i1, ob = int64_t(cb) * n1 + i1;
      float hia[3], dea[3], sla[3];
      tp1_node32(load_rec(lev, oa), load_rec(lev, oa + n1), ha, hia, dea, sla);
      if (q < Lh) {
        float hib[3], deb[3], slb[3];
        tp1_node32(load_rec(lev, ob), load_rec(lev, ob + n1), hb, hib, deb, slb);
        const float uah = T.uah[jm][la], ual = T.ual[jm][la];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          float hs = hia[f], he = 0.f;
          two_sum_into(hs, he, hib[f]);
          comp_acc1(RS[f], RC[f], T.uh[la], T.ul[la], hs, __fadd_rn(__fadd_rn(dea[f], deb[f]), he));
          Su[f] = __fmaf_rn(T.uh[la], __fadd_rn(sla[f], slb[f]), Su[f]);
          const float dv = __fadd_rn(__fsub_rn(hia[f], hib[f]), __fsub_rn(dea[f], deb[f]));
          Ra[f] = __fmaf_rn(ual, dv, __fmaf_rn(uah, dv, Ra[f]));
          Sa[f] = __fmaf_rn(uah, __fsub_rn(sla[f], slb[f]), Sa[f]);
        }
      } else {
        // the middle node of an odd L (a = 0: no ua terms)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          comp_acc1(RS[f], RC[f], T.uh[la], T.ul[la], hia[f], dea[f]);
          Su[f] = __fmaf_rn(T.uh[la], sla[f], Su[f]);
        }
      }
    }
    float Rh[3], Rl[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      // renormalized: |lo| within half an ulp of hi
      const float sm = __fadd_rn(RS[f], RC[f]);
      Rl[f] = __fsub_rn(RC[f], __fsub_rn(sm, RS[f]));
      Rh[f] = sm;
    }
    float4 *b = tp + int64_t(jm) * 4 * P.Np + qq;
    b[0] = make_float4(Rh[0], Rh[1], Rh[2], Rl[0]);
    b[P.Np] = make_float4(Rl[1], Rl[2], Su[0], Su[1]);
    b[2 * P.Np] = make_float4(Su[2], Ra[0], Ra[1], Ra[2]);
    b[3 * P.Np] = make_float4(Sa[0], Sa[1], Sa[2], 0.f);
  }
}

// One node of pass 2: the x1 interpolants of the three fields from the
// pass-1 records of columns c1 (A) and c1 + 1 (B): value hi + del of (R_u,
// S_u), and the plain value of (R_a, S_a).
__device__ __forceinline__ void tp2_node32(const Rec2f &A, const Rec2f &B, const float *h,
                                           float *hi, float *del, float *va) {
  const float ah[3] = {A.v0.x, A.v0.y, A.v0.z}, al[3] = {A.v0.w, A.v1.x, A.v1.y};
  const float bh[3] = {B.v0.x, B.v0.y, B.v0.z}, bl[3] = {B.v0.w, B.v1.x, B.v1.y};
  const float as[3] = {A.v1.z, A.v1.w, A.v2.x}, bs[3] = {B.v1.z, B.v1.w, B.v2.x};
  const float ar[3] = {A.v2.y, A.v2.z, A.v2.w}, br[3] = {B.v2.y, B.v2.z, B.v2.w};
  const float aS[3] = {A.v3.x, A.v3.y, A.v3.z}, bS[3] = {B.v3.x, B.v3.y, B.v3.z};
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const float dv = __fadd_rn(__fsub_rn(bh[f], ah[f]), __fsub_rn(bl[f], al[f]));
    hi[f] = ah[f];
    del[f] = __fmaf_rn(h[3], bs[f], __fmaf_rn(h[2], as[f], __fmaf_rn(h[1], dv, al[f])));
    va[f] = __fmaf_rn(h[3], bS[f],
                      __fmaf_rn(h[2], aS[f], __fmaf_rn(h[1], br[f], __fmul_rn(h[0], ar[f]))));
  }
}

// FP32C pass 2 and the tail: per point, every step's x1 pass over mirror
// pairs of l1 (compensated z and y sums, plain driver terms, as the
// node-wise FP32C kernel keeps them), then z^n, A and y^n as there.
__global__ void __launch_bounds__(kTPThreads)
    k2_tp2_32(const Params2 P, const float4 *__restrict__ ring, const float4 *__restrict__ tp,
              double *__restrict__ V, const __grid_constant__ TPTab2f T, int n, Stats *st) {
  wait_predecessor();
  const int64_t qq = int64_t(blockIdx.x) * kTPThreads + threadIdx.x;
  const bool active = qq < P.Np;
  int it = 0;
  float d = 0.f;
  if (active) {
    const int n1 = int(P.Nx1);
    const int i1 = int(qq % n1), i2 = int(qq / n1);
    const int L = P.L, Lh = P.L / 2;
    Acc2f a{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int jm = 0; jm < P.k; ++jm) {
      const Lev2f W = lev2f(tp, P.Np, jm);
      const bool yj = jm == P.k - 1;
#pragma unroll 1
      for (int q = 0; q < (L + 1) / 2; ++q) {
        const int la = q, lb = L - 1 - q;
        int ca = i1 + T.s1[jm][la], cb = i1 + T.s1[jm][lb];
        float ha[4] = {T.h1[jm][la][0], T.h1[jm][la][1], T.h1[jm][la][2], T.h1[jm][la][3]};
        float hb[4] = {T.h1[jm][lb][0], T.h1[jm][lb][1], T.h1[jm][lb][2], T.h1[jm][lb][3]};
        tp_clamp(ca, n1, ha);
        tp_clamp(cb, n1, hb);
        const int64_t oa = int64_t(i2) * n1 + ca, ob = int64_t(i2) * n1 + cb;
        float hia[3], dea[3], vaa[3];
        tp2_node32(load_rec(W, oa), load_rec(W, oa + 1), ha, hia, dea, vaa);
        const float Fa = __fmaf_rn(P.alpha_f, __fadd_rn(hia[0], dea[0]),
                                   __fmaf_rn(P.beta1_f, __fadd_rn(hia[1], dea[1]),
                                             __fmul_rn(P.beta2_f, __fadd_rn(hia[2], dea[2]))));
        const float Ga = __fmaf_rn(P.alpha_f, vaa[0],
                                   __fmaf_rn(P.beta1_f, vaa[1], __fmul_rn(P.beta2_f, vaa[2])));
        if (q < Lh) {
          float hib[3], deb[3], vab[3];
          tp2_node32(load_rec(W, ob), load_rec(W, ob + 1), hb, hib, deb, vab);
          const float Fb = __fmaf_rn(P.alpha_f, __fadd_rn(hib[0], deb[0]),
                                     __fmaf_rn(P.beta1_f, __fadd_rn(hib[1], deb[1]),
                                               __fmul_rn(P.beta2_f, __fadd_rn(hib[2], deb[2]))));
          const float Gb = __fmaf_rn(P.alpha_f, vab[0],
                                     __fmaf_rn(P.beta1_f, vab[1], __fmul_rn(P.beta2_f, vab[2])));
          // F_a - F_b from the fields' differences (their hi parts subtract
          // exactly), as the node-wise kernel forms it
          float dv[3];
#pragma unroll
          for (int f = 0; f < 3; ++f)
            dv[f] = __fadd_rn(__fsub_rn(hia[f], hib[f]), __fsub_rn(dea[f], deb[f]));
          const float dF = __fmaf_rn(P.alpha_f, dv[0],
                                     __fmaf_rn(P.beta1_f, dv[1], __fmul_rn(P.beta2_f, dv[2])));
          a.F1 = __fmaf_rn(T.cfal[jm][la], dF, __fmaf_rn(T.cfah[jm][la], dF, a.F1));
          const float G = __fadd_rn(Ga, Gb);
          a.F2 = __fmaf_rn(T.cful[jm][la], G, __fmaf_rn(T.cfuh[jm][la], G, a.F2));
          two_sum_into(a.Fy, a.FyC, __fmul_rn(T.cfy[jm][la], __fadd_rn(Fa, Fb)));
          float hs, he;
#pragma unroll
          for (int f = 1; f < 3; ++f) {
            hs = hia[f];
            he = 0.f;
            two_sum_into(hs, he, hib[f]);
            const float dd = __fadd_rn(__fadd_rn(dea[f], deb[f]), he);
            if (f == 1)
              comp_acc1(a.S1, a.C1, T.czh[jm][la], T.czl[jm][la], hs, dd);
            else
              comp_acc1(a.S2, a.C2, T.czh[jm][la], T.czl[jm][la], hs, dd);
          }
          if (yj) {
            hs = hia[0];
            he = 0.f;
            two_sum_into(hs, he, hib[0]);
            comp_acc1(a.Sy, a.Cy, T.cyh[jm][la], T.cyl[jm][la], hs,
                      __fadd_rn(__fadd_rn(dea[0], deb[0]), he));
          }
        } else {
          // the middle node of an odd L (a = 0: no ua term)
          a.F2 = __fmaf_rn(T.cful[jm][la], Ga, __fmaf_rn(T.cfuh[jm][la], Ga, a.F2));
          two_sum_into(a.Fy, a.FyC, __fmul_rn(T.cfy[jm][la], Fa));
          comp_acc1(a.S1, a.C1, T.czh[jm][la], T.czl[jm][la], hia[1], dea[1]);
          comp_acc1(a.S2, a.C2, T.czh[jm][la], T.czl[jm][la], hia[2], dea[2]);
          if (yj) comp_acc1(a.Sy, a.Cy, T.cyh[jm][la], T.cyl[jm][la], hia[0], dea[0]);
        }
      }
    }
    // z_d = S + (C + F) and A = S + (C + F) as exact float pairs
    float z1h = a.S1, z1l = 0.f, z2h = a.S2, z2l = 0.f, Ah = a.Sy, Al = 0.f;
    two_sum_into(z1h, z1l, __fadd_rn(a.C1, a.F1));
    two_sum_into(z2h, z2l, __fadd_rn(a.C2, a.F2));
    two_sum_into(Ah, Al, a.Fy);
    two_sum_into(Ah, Al, __fadd_rn(a.Cy, a.FyC));
    const float zlin = __fmaf_rn(P.beta1_f, z1h, __fmul_rn(P.beta2_f, z2h));
    // Picard on the increment delta = y^n - A: delta = hg0 f(A + delta, z)
    const float4 v0 = lev2f(ring, P.Np, (n + 1) % P.nslot).p0[qq];
    float dl = __fadd_rn(__fsub_rn(v0.x, Ah), __fsub_rn(v0.w, Al));
    float dpp = __int_as_float(0x7fc00000);
    while (it < P.picard_max) {
      const float dn = __fmul_rn(P.hg0_f, __fmaf_rn(P.alpha_f, __fadd_rn(Ah, dl), zlin));
      ++it;
      d = fabsf(__fsub_rn(dn, dl));
      const bool cyc = dn == dpp && picard_cycle_ok(d, __fadd_rn(Ah, dl), dn);
      dpp = dl;
      dl = dn;
      if (cyc) d = 0.f;
      if (d <= P.picard_tol_f || !isfinite(d)) break;  // a non-finite step cannot converge
    }
    put_new32(P, V, qq, Ah, Al, dl, z1h, z1l, z2h, z2l);
  }
  record_picard32(st, active, it, d, P.picard_tol_f);
}

__device__ double interp2_point32(const Params2 &P, const Lev2f &lev, int field, double X1,
                                  double X2) {
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
  auto rec = [&](int64_t q) {
    const Rec2f R = load_rec(lev, q);
    double4_32a o;
    if (field == 0) {
      o = make_double4_32a(double(R.v0.x) + double(R.v0.w), R.v1.z, R.v2.y, R.v3.x);
    } else if (field == 1) {
      o = make_double4_32a(double(R.v0.y) + double(R.v1.x), R.v1.w, R.v2.z, R.v3.y);
    } else {
      o = make_double4_32a(double(R.v0.z) + double(R.v1.y), R.v2.x, R.v2.w, R.v3.z);
    }
    return o;
  };
  const int64_t b = c2 * P.Nx1 + c1;
  return bicubic(rec(b), rec(b + 1), rec(b + P.Nx1), rec(b + P.Nx1 + 1), h1, h2);
}

__global__ void k2_readout32(const Params2 P, const float4 *ring, int slot, Stats2 *st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const Lev2f lev = lev2f(ring, P.Np, slot);
  st->s.y0 = interp2_point32(P, lev, 0, P.x01, P.x02);
  st->s.z0 = interp2_point32(P, lev, 1, P.x01, P.x02);
  st->z0b = interp2_point32(P, lev, 2, P.x01, P.x02);
}

__global__ void k2_export32(const Params2 P, const float4 *ring, int slot, double *out) {
  const Lev2f lev = lev2f(ring, P.Np, slot);
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < P.Np;
       q += int64_t(gridDim.x) * blockDim.x) {
    const Rec2f R = load_rec(lev, q);
    out[q] = double(R.v0.x) + double(R.v0.w);
    out[P.Np + q] = double(R.v0.y) + double(R.v1.x);
    out[2 * P.Np + q] = double(R.v0.z) + double(R.v1.y);
  }
}

// ---------------------------------------------------------------------------
// Host side: validation, constants, layout.
// ---------------------------------------------------------------------------
struct Layout2 {
  size_t ring, vals, table, stage, stats, tp, total;
};

static bool tensor_form2(const bsde2_problem &p) {
  return p.step_form == BSDE2_STEP_TENSOR || (p.step_form == BSDE2_STEP_AUTO && p.b21 == 0.0);
}

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
  if (p.precision != BSDE_FP64 && p.precision != BSDE_FP32C) return BSDE_EINVAL;
  if (p.picard_max < 1 || !(p.picard_tol >= 0.0)) return BSDE_EINVAL;
  if (p.step_form < BSDE2_STEP_AUTO || p.step_form > BSDE2_STEP_TENSOR) return BSDE_EINVAL;
  if (p.step_form == BSDE2_STEP_TENSOR && p.b21 != 0.0) return BSDE_EINVAL;
  return BSDE_OK;
}

static Layout2 layout2(const bsde2_problem &p) {
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t np = size_t(p.Nx1) * size_t(p.Nx2), ns = size_t(p.k + 1);
  Layout2 L{};
  size_t off = 0;
  // FP64: 3 fields x 32-byte records per point; FP32C: four float4 planes
  L.ring = off; off = up(off + ns * np * (p.precision == BSDE_FP64 ? 96 : sizeof(Rec2f)));
  L.vals = off; off = up(off + 3 * np * 8);
  L.table = off; off = up(off + size_t(p.k) * p.L * p.L * sizeof(Node2));
  L.stage = off; off = up(off + 3 * size_t(p.k) * np * 8);
  L.stats = off; off = up(off + sizeof(Stats2));
  L.tp = off;
  if (tensor_form2(p)) off = up(off + size_t(p.k) * np * (p.precision == BSDE_FP64 ? 96 : 64));
  L.total = off;
  return L;
}

// The FP32C pair table from the FP64 node table: pair q of level j joins
// nodes q and L^2 - 1 - q ((l1, l2) and (L-1-l1, L-1-l2)); the middle node
// of an odd L is a pair with itself at half weight.
static void build_pairs2f(const Params2 &P, const std::vector<Node2> &tab,
                          std::vector<Node2f> &out) {
  out.assign(size_t(P.k) * P.LLp, Node2f{});
  for (int j = 0; j < P.k; ++j) {
    for (int q = 0; q < P.LLp; ++q) {
      const Node2 &a = tab[size_t(j) * P.LL + q];
      const Node2 &b = tab[size_t(j) * P.LL + (P.LL - 1 - q)];
      const double half = (q == P.LL - 1 - q) ? 0.5 : 1.0;
      Node2f f{};
      f.s1a = a.s1;
      f.s2a = a.s2;
      f.s1b = b.s1;
      f.s2b = b.s2;
      for (int u = 0; u < 4; ++u) {
        f.h1a[u] = float(a.h1[u]);
        f.h2a[u] = float(a.h2[u]);
        f.h1b[u] = float(b.h1[u]);
        f.h2b[u] = float(b.h2[u]);
      }
      const double cz = a.cz * half, cy = a.cy * half;
      f.czh = float(cz);
      f.czl = float(cz - double(f.czh));
      f.cyh = float(cy);
      f.cyl = float(cy - double(f.cyh));
      f.cfz1 = float(a.cfz1);  // node b's is -cfz (opposite DeltaW); 0 for the middle
      f.cfz2 = float(a.cfz2);
      f.cfy = float(a.cfy * half);
      out[size_t(j) * P.LLp + q] = f;
    }
  }
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
  P.precision = p.precision;
  {
    // |d| <= tol for a float d is exactly |d| <= the largest float <= tol
    float tf = (float)p.picard_tol;
    if ((double)tf > p.picard_tol) tf = std::nextafter(tf, 0.0f);
    P.picard_tol_f = tf;
  }
  gamma_tables(p.k, P.gy, P.gz);
  P.h = p.k * P.dt;
  P.hg0 = P.h * P.gy[0];
  P.alpha_f = float(P.alpha);
  P.beta1_f = float(P.beta1);
  P.beta2_f = float(P.beta2);
  P.hg0_f = float(P.hg0);
  // work split as in 1-D: >= 4 groups per point, at most kMaxGroups, no
  // more threads per level than the GPU holds at once when that is known
  P.LLp = (P.LL + 1) / 2;
  const int units = P.precision == BSDE_FP32C ? P.LLp : P.LL;
  int S = (4 + P.k - 1) / P.k;
  if (S * P.k > kMaxGroups) S = kMaxGroups / P.k;
  if (S > units) S = units;
  while (S > 1 && resident_threads > 0 && long(P.Np) * P.k * S > resident_threads) --S;
  if (S < 1) S = 1;
  P.S = S;
  P.Lg = (units + S - 1) / S;
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

// The tensor-product tables from the node table (whose shift and basis in
// x1 depend on l1 alone and in x2 on l2 alone when b21 = 0) and the
// one-dimensional quadrature weights.
static void build_tp2(const bsde2_problem &p, const Params2 &P, const std::vector<Node2> &tab,
                      TPTab2d &D, TPTab2f &F) {
  std::memset(&D, 0, sizeof(D));
  std::memset(&F, 0, sizeof(F));
  double a[kMaxL2], w[kMaxL2];
  gauss_hermite(p.L, a, w);
  const double rpi = std::sqrt(M_PI);
  auto split = [](double v, float &hi, float &lo) {
    hi = float(v);
    lo = float(v - double(hi));
  };
  for (int l = 0; l < p.L; ++l) {
    D.u[l] = w[l] / rpi;
    split(D.u[l], F.uh[l], F.ul[l]);
  }
  for (int jm = 0; jm < P.k; ++jm) {
    const int j = jm + 1;
    const double sq = std::sqrt(2.0 * j * P.dt);
    D.cz[jm] = ((j == 1 ? 1.0 : 0.0) - P.gz[j]) / P.gz[0];
    D.cf[jm] = P.gz[j] / P.gz[0];
    D.cy[jm] = j == P.k ? 1.0 : 0.0;
    D.cfy[jm] = P.h * P.gy[j];
    for (int l = 0; l < p.L; ++l) {
      const Node2 &e1 = tab[size_t(jm) * P.LL + size_t(l) * p.L];  // (l1 = l, l2 = 0)
      const Node2 &e2 = tab[size_t(jm) * P.LL + size_t(l)];        // (l1 = 0, l2 = l)
      D.s1[jm][l] = F.s1[jm][l] = e1.s1;
      D.s2[jm][l] = F.s2[jm][l] = e2.s2;
      for (int u = 0; u < 4; ++u) {
        D.h1[jm][l][u] = e1.h1[u];
        D.h2[jm][l][u] = e2.h2[u];
        F.h1[jm][l][u] = float(e1.h1[u]);
        F.h2[jm][l][u] = float(e2.h2[u]);
      }
      D.ua[jm][l] = D.u[l] * sq * a[l];
      split(D.ua[jm][l], F.uah[jm][l], F.ual[jm][l]);
      split(D.cz[jm] * D.u[l], F.czh[jm][l], F.czl[jm][l]);
      split(D.cy[jm] * D.u[l], F.cyh[jm][l], F.cyl[jm][l]);
      F.cfy[jm][l] = float(D.cfy[jm] * D.u[l]);
      split(D.cf[jm] * D.ua[jm][l], F.cfah[jm][l], F.cfal[jm][l]);
      split(D.cf[jm] * D.u[l], F.cfuh[jm][l], F.cful[jm][l]);
    }
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
  bool tab_param;            // FP32C: the pair table fits the step's parameters
  bsde::PairTab2 tab;        // ... and is passed by value (k2_step32p)
  bool tensor;               // the step as two tensor-product passes
  bsde::TPTab2d tpd;         // their tables (FP64, FP32C), by value
  bsde::TPTab2f tpf;
};

namespace bsde {

static size_t step32_2d_smem(const Params2 &P) {
  return sizeof(Node2f) * size_t(P.k) * P.LLp + sizeof(float) * 10 * size_t(P.G) * kStep2TP;
}

// The tensor-product passes of level n: parts & 1 the x2 pass, & 2 the x1
// pass and the tail.
static void launch2_tp(bsde2_plan_t *pl, cudaStream_t s, int n, int parts) {
  const Params2 &P = pl->P;
  cudaLaunchConfig_t lc{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  const unsigned blocks = unsigned((P.Np + kTPThreads - 1) / kTPThreads);
  lc.blockDim = dim3(kTPThreads, 1, 1);
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  Stats *st = reinterpret_cast<Stats *>(pl->ws + pl->lay.stats);
  double *V = reinterpret_cast<double *>(pl->ws + pl->lay.vals);
  if (parts & 1) {
    lc.gridDim = dim3(blocks, unsigned(P.k), 1);
    if (P.precision == BSDE_FP32C) {
      lc.gridDim = dim3(unsigned((P.Nx1 + kTP1X - 1) / kTP1X),
                        unsigned(std::min<int64_t>((P.Nx2 + kTP1Y - 1) / kTP1Y, 65535)),
                        unsigned(P.k));
      cudaLaunchKernelEx(&lc, k2_tp1_32, P, reinterpret_cast<const float4 *>(pl->ws + pl->lay.ring),
                         reinterpret_cast<float4 *>(pl->ws + pl->lay.tp), pl->tpf, n);
    } else {
      cudaLaunchKernelEx(&lc, k2_tp1, P,
                         reinterpret_cast<const double4_32a *>(pl->ws + pl->lay.ring),
                         reinterpret_cast<double4_32a *>(pl->ws + pl->lay.tp), pl->tpd, n);
    }
  }
  if (parts & 2) {
    lc.gridDim = dim3(blocks, 1, 1);
    if (P.precision == BSDE_FP32C)
      cudaLaunchKernelEx(&lc, k2_tp2_32, P, reinterpret_cast<const float4 *>(pl->ws + pl->lay.ring),
                         reinterpret_cast<const float4 *>(pl->ws + pl->lay.tp), V, pl->tpf, n, st);
    else
      cudaLaunchKernelEx(&lc, k2_tp2, P,
                         reinterpret_cast<const double4_32a *>(pl->ws + pl->lay.ring),
                         reinterpret_cast<const double4_32a *>(pl->ws + pl->lay.tp), V, pl->tpd,
                         n, st);
  }
}

static void launch2_step(bsde2_plan_t *pl, cudaStream_t s, int n) {
  const Params2 &P = pl->P;
  if (pl->tensor) {
    launch2_tp(pl, s, n, 3);
    return;
  }
  const unsigned blocks = unsigned((P.Np + kStep2TP - 1) / kStep2TP);
  if (P.precision == BSDE_FP32C && pl->tab_param) {
    launch_pdl(k2_step32p, blocks, unsigned(kStep2TP * P.G),
               sizeof(float) * 10 * size_t(P.G) * kStep2TP, s, P,
               reinterpret_cast<const float4 *>(pl->ws + pl->lay.ring),
               reinterpret_cast<double *>(pl->ws + pl->lay.vals), pl->tab, n,
               reinterpret_cast<Stats *>(pl->ws + pl->lay.stats));
    return;
  }
  if (P.precision == BSDE_FP32C) {
    launch_pdl(k2_step32, blocks, unsigned(kStep2TP * P.G), step32_2d_smem(P), s, P,
               reinterpret_cast<const float4 *>(pl->ws + pl->lay.ring),
               reinterpret_cast<double *>(pl->ws + pl->lay.vals),
               reinterpret_cast<const Node2f *>(pl->ws + pl->lay.table), n,
               reinterpret_cast<Stats *>(pl->ws + pl->lay.stats));
    return;
  }
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
  lc.gridDim = dim3(unsigned((P.Nx1 + kDerTX - 1) / kDerTX),
                    unsigned(std::min<int64_t>((P.Nx2 + kDerTY - 1) / kDerTY, 65535)), 1);
  lc.blockDim = dim3(kDerTX * kDerTY, 1, 1);
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  if (P.precision == BSDE_FP32C)
    cudaLaunchKernelEx(&lc, k2_deriv32, P,
                       reinterpret_cast<const double *>(pl->ws + pl->lay.vals),
                       reinterpret_cast<float4 *>(pl->ws + pl->lay.ring), slot);
  else
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
    launches += pl->tensor ? 3 : 2;
  }
  double *out = reinterpret_cast<double *>(pl->ws + pl->lay.stage);
  if (P.precision == BSDE_FP32C) {
    const float4 *r32 = reinterpret_cast<const float4 *>(pl->ws + pl->lay.ring);
    k2_readout32<<<1, 32, 0, s>>>(P, r32, 0, st);
    k2_export32<<<eb, 256, 0, s>>>(P, r32, 0, out);
  } else {
    k2_readout<<<1, 32, 0, s>>>(P, ring, 0, st);
    // level 0 into the staging area (its first 3 planes)
    k2_export<<<eb, 256, 0, s>>>(P, ring, 0, out);
  }
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
  pl->tensor = tensor_form2(*p);
  if (pl->tensor) build_tp2(*p, pl->P, tab, pl->tpd, pl->tpf);
  cudaError_t e;
  if (p->precision == BSDE_FP32C) {
    std::vector<Node2f> t32;
    build_pairs2f(pl->P, tab, t32);
    e = cudaMemcpy(pl->ws + lay.table, t32.data(), sizeof(Node2f) * t32.size(),
                   cudaMemcpyHostToDevice);
    pl->tab_param = t32.size() <= size_t(kPairTab2Cap);
    if (pl->tab_param) std::memcpy(pl->tab.e, t32.data(), sizeof(Node2f) * t32.size());
    const size_t sm = step32_2d_smem(pl->P);
    if (e == cudaSuccess && sm > 48 * 1024)
      e = cudaFuncSetAttribute(k2_step32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  } else {
    e = cudaMemcpy(pl->ws + lay.table, tab.data(), sizeof(Node2) * tab.size(),
                   cudaMemcpyHostToDevice);
  }
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
  if ((parts & 12) && !pl->tensor) return fail(BSDE_EINVAL, "pass parts need the TENSOR form");
  if (parts & 1) launch2_step(pl, s, n);
  if (parts & 4) launch2_tp(pl, s, n, 1);
  if (parts & 8) launch2_tp(pl, s, n, 2);
  if (parts & 2) launch2_deriv(pl, s, n % pl->P.nslot);
  BSDE_CUDA_TRY(cudaGetLastError());
  return BSDE_OK;
}

int64_t bsde2_plan_launches(const bsde2_plan_t *pl) {
  if (!pl) return 0;
  const bsde::Params2 &P = pl->P;
  return 1 + 2 * int64_t(P.k) + (pl->tensor ? 3 : 2) * int64_t(P.N - P.k + 1) + 2;
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
