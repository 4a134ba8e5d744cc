// Device code of the multistep BSDE solver (sm_103a).  Included once, by
// bsde_cuda.cu.
#pragma once

#include <cuda_runtime.h>

#include "bsde_internal.h"

namespace bsde {

// ---------------------------------------------------------------------------
// Drivers f(t, y, z) (Eq. 22, 24, 29 and the 1-D analogue of Eq. 34).
// Coefficients are precomputed per problem: for BS and LB
// f = -(ca y + cb z) [+ cc min(y - cis z, 0)].
// ---------------------------------------------------------------------------
template <typename T>
struct DrvC {
  T ca, cb, cc, cis;
};

// Every product and sum is spelled out with an explicit rounding intrinsic,
// so no kernel that inlines a driver can contract it differently from
// another: the single-problem, batched and served solves give bitwise equal
// results.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <int DRV, typename T>
__device__ __forceinline__ T driver(const DrvC<T> &c, T t, T et, T emt, T y, T z) {
  // et = exp(t^2), emt = exp(-t^2): per-level constants of Example 2
  if constexpr (DRV == BSDE_DRIVER_LIN_SIN) {
    return rsub(rmul(T(0.5), y), z);
  } else if constexpr (DRV == BSDE_DRIVER_BS) {
    return -rfma(c.ca, y, rmul(c.cb, z));
  } else if constexpr (DRV == BSDE_DRIVER_LB) {
    T m = rsub(y, rmul(z, c.cis));
    m = m < T(0) ? m : T(0);
    return rfma(c.cc, m, -rfma(c.ca, y, rmul(c.cb, z)));
  } else if constexpr (DRV == BSDE_DRIVER_EX1) {
    const T y2 = rmul(y, y);
    return rfma(T(-1.5), y, rfma(T(2.5), y2, -rmul(y2, y)));
  } else {
    const T e = exp(rsub(rmul(t, t), rmul(y, emt)));
    const T s = rfma(rmul(z, z), emt, rsub(et, rfma(T(3), e, rmul(rmul(T(4), t), y))));
    return rmul(T(0.5), s);
  }
}

// ---------------------------------------------------------------------------
// Closed-form solutions for the k initial levels (Section 3.1 step 2, read as
// the exact start) and the cell-averaged call payoff (Section 5, Example 3).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ncdf(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }

__device__ void closed_form(const Params &P, double t, double x, bool smooth_level,
                            double &u, double &z) {
  double ux = 0.0;
  if (P.terminal == BSDE_TERMINAL_SIN) {
    u = sin(x + t);
    ux = cos(x + t);
  } else if (P.terminal == BSDE_TERMINAL_CALL_LOG) {
    const double K = P.strike;
    if (smooth_level) {
      // averages over [x - dx/2, x + dx/2] of (e^s - K)^+ and of its derivative
      const double a = x - 0.5 * P.dx, b = x + 0.5 * P.dx, kap = log(K);
      if (b <= kap) {
        u = 0.0;
        ux = 0.0;
      } else if (a >= kap) {
        const double ea = exp(a) * expm1(b - a) / P.dx;
        u = ea - K;
        ux = ea;
      } else {
        const double d = b - kap;
        u = K * (expm1(d) - d) / P.dx;
        ux = K * expm1(d) / P.dx;
      }
    } else {
      double r = P.r, dl = P.delta;
      if (P.driver == BSDE_DRIVER_LB) {
        r = P.r - P.lb_sign * (P.R - P.r);
        dl = 0.0;
      }
      // rounded separately (no contraction with the caller's t = n dt): at
      // the terminal level tau is exactly 0 and the payoff branch is taken
      const double S = exp(x), tau = __dsub_rn(P.T, t);
      if (tau <= 0.0) {
        u = S > K ? S - K : 0.0;
        ux = S > K ? S : 0.0;
      } else {
        const double sq = P.sigma * sqrt(tau);
        const double d1 = (log(S / K) + (r - dl + 0.5 * P.sigma * P.sigma) * tau) / sq;
        const double d2 = d1 - sq;
        const double a = S * exp(-dl * tau) * ncdf(d1);
        u = a - K * exp(-r * tau) * ncdf(d2);
        ux = a;
      }
    }
  } else if (P.terminal == BSDE_TERMINAL_LOGISTIC) {
    const double e = exp(x + t);
    u = e / (e + 1.0);
    ux = e / ((e + 1.0) * (e + 1.0));
  } else if (P.terminal == BSDE_TERMINAL_LNSIN) {
    const double e = exp(t * t);
    u = log(sin(x) + 3.0) * e;
    ux = e * cos(x) / (sin(x) + 3.0);
  } else if (P.terminal == BSDE_TERMINAL_ONE) {
    // the Vasicek bond: kappa = -a_1, theta = a_x / kappa, sigma = b_x
    const double tau = __dsub_rn(P.T, t);
    if (tau <= 0.0) {
      u = 1.0;
      ux = 0.0;
    } else {
      const double kap = -P.a_1, th = P.a_x / kap, sg = P.b_x;
      const double B = -expm1(-kap * tau) / kap;
      const double lnA = (th - sg * sg / (2.0 * kap * kap)) * (B - tau) - sg * sg * B * B / (4.0 * kap);
      u = exp(lnA - B * x);
      ux = -B * u;
    }
  } else {
    // call in the price x = S under geometric Brownian motion (volatility b_1)
    const double K = P.strike, tau = __dsub_rn(P.T, t), sg = P.b_1;
    double r = P.r, dl = P.delta;
    if (P.driver == BSDE_DRIVER_LB) {
      r = P.r - P.lb_sign * (P.R - P.r);
      dl = 0.0;
    }
    if (smooth_level) {
      // averages over [x - dx/2, x + dx/2] of (s - K)^+ and of b(s) 1{s > K}
      const double a = x - 0.5 * P.dx, b = x + 0.5 * P.dx;
      if (b <= K) {
        u = 0.0;
        z = 0.0;
      } else {
        const double lo = a > K ? a : K;
        u = 0.5 * ((b - K) * (b - K) - (lo - K) * (lo - K)) / P.dx;
        z = (P.b_x * (b - lo) + 0.5 * P.b_1 * (b * b - lo * lo)) / P.dx;
      }
      return;
    }
    if (x <= 0.0) {
      u = 0.0;
      ux = 0.0;
    } else if (tau <= 0.0) {
      u = x > K ? x - K : 0.0;
      ux = x > K ? 1.0 : 0.0;
    } else {
      const double sq = sg * sqrt(tau);
      const double d1 = (log(x / K) + (r - dl + 0.5 * sg * sg) * tau) / sq, d2 = d1 - sq;
      u = x * exp(-dl * tau) * ncdf(d1) - K * exp(-r * tau) * ncdf(d2);
      ux = exp(-dl * tau) * ncdf(d1);
    }
  }
  // z = b(x) u_x (b constant unless the forward process is AFFINE)
  z = (P.b_x + P.b_1 * x) * ux;
}

// ---------------------------------------------------------------------------
// Level storage.  FP64: double4_32a (y, M_y, z, M_z) per node.  FP32C: float4
// (y_hi, z_hi, y_lo, z_lo) plus float2 (M_y, M_z) per node, value = hi + lo;
// the (y, z) lane pairs feed packed FP32x2 arithmetic directly.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_store(float4 *A, int64_t i, double y, double z) {
  const float yh = __double2float_rn(y), zh = __double2float_rn(z);
  const float yl = __double2float_rn(__dsub_rn(y, (double)yh));
  const float zl = __double2float_rn(__dsub_rn(z, (double)zh));
  A[i] = make_float4(yh, zh, yl, zl);
}

// Level loads: plain loads through L1.  Within one launch of the per-level
// kernels the levels they read are constant.  The persistent batch and
// serving kernels rewrite ring slots between levels from other SMs of a
// cluster; the cluster barrier between those phases (barrier.cluster.arrive
// with release and barrier.cluster.wait with acquire semantics, at cluster
// scope) orders the writes before the next phase's loads, so these loads see
// them without bypassing L1.
template <typename T>
__device__ __forceinline__ T ldl(const T *p) {
  return *p;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor on the stream finishes; it
// waits here, before touching anything the predecessor wrote.  (A no-op for
// an ordinary launch.)
__device__ __forceinline__ void wait_predecessor() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

struct Ring64 {
  double4_32a *ring;
};
// FP32C level slots, per node: A = (y_hi, z_hi, y_lo, z_lo) (value = hi + lo)
// and M = (M_y, M_z), the natural spline's second derivatives.  The spline
// value at x_c + theta dx is v_c + theta d + kappa (P + theta Q),
// kappa = -theta (1 - theta) dx^2 / 6, with d = v_{c+1} - v_c,
// P = 2 M_c + M_{c+1}, Q = M_{c+1} - M_c formed from nodes c and c + 1
// (node_value): 24 bytes per node.
struct Ring32 {
  float4 *A;
  float2 *M;
};
__host__ __device__ inline Ring32 ring32(void *A, void *M, const Params &) {
  return Ring32{static_cast<float4 *>(A), static_cast<float2 *>(M)};
}

__global__ void k_reset_stats(Stats *s) {
  if (threadIdx.x == 0) {
    s->y0 = 0.0;
    s->z0 = 0.0;
    s->resid_bits = 0ull;
    s->iters_max = 0;
    s->nonconv = 0;
    s->timeout = 0;
  }
}

// initial level N - m from the closed form
// point i of initial level N - m from the closed form
template <int PREC>
__device__ __forceinline__ void init_point(const Params &P, Ring64 r64, Ring32 r32, int m,
                                           int64_t i) {
  const int level = P.N - m;
  const int64_t off = int64_t(level % P.nslot) * P.Nx;
  const double t = __dmul_rn(double(level), P.dt);
  const bool smooth = (m == 0) && P.smoothing &&
                      (P.terminal == BSDE_TERMINAL_CALL_LOG ||
                       P.terminal == BSDE_TERMINAL_CALL_PRICE);
  const double x = P.x_min + double(i) * P.dx;
  double u, z;
  closed_form(P, t, x, smooth, u, z);
  if (PREC == BSDE_FP64) {
    r64.ring[off + i] = make_double4_32a(u, 0.0, z, 0.0);
  } else {
    split_store(r32.A + off, i, u, z);
  }
}

template <int PREC>
__global__ void k_init_closed(const Params P, Ring64 r64, Ring32 r32, int m) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < P.Nx;
       i += int64_t(gridDim.x) * blockDim.x)
    init_point<PREC>(P, r64, r32, m, i);
}

// initial level N - m imported from the staging area (row m of y, row m of z)
template <int PREC>
__global__ void k_import(const Params P, Ring64 r64, Ring32 r32, const double *sy,
                         const double *sz, int m) {
  const int level = P.N - m;
  const int64_t off = int64_t(level % P.nslot) * P.Nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < P.Nx;
       i += int64_t(gridDim.x) * blockDim.x) {
    const double u = sy[int64_t(m) * P.Nx + i], z = sz[int64_t(m) * P.Nx + i];
    if (PREC == BSDE_FP64) {
      r64.ring[off + i] = make_double4_32a(u, 0.0, z, 0.0);
    } else {
      split_store(r32.A + off, i, u, z);
    }
  }
}

// level in `slot` exported to the staging area as doubles
template <int PREC>
__global__ void k_export(const Params P, Ring64 r64, Ring32 r32, double *sy, double *sz,
                         int slot) {
  const int64_t off = int64_t(slot) * P.Nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < P.Nx;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (PREC == BSDE_FP64) {
      const double4_32a v = r64.ring[off + i];
      sy[i] = v.x;
      sz[i] = v.z;
    } else {
      const float4 v = r32.A[off + i];
      sy[i] = double(v.x) + double(v.z);
      sz[i] = double(v.y) + double(v.w);
    }
  }
}

// ---------------------------------------------------------------------------
// S2: natural cubic spline second derivatives of the level in `slot`
// (Section 3.3; the paper solves the tridiagonal system iteratively, here it
// is solved exactly).  Unknowns u_m = M_{m+1}, m = 0..Nx-3:
//   u_{m-1} + 4 u_m + u_{m+1} = r_m = 6 (v_m - 2 v_{m+1} + v_{m+2}) / dx^2,
// M_0 = M_{Nx-1} = 0.  LU of tridiag(1, 4, 1): forward g_m = r_m - g_{m-1}/d_{m-1},
// backward u_m = (g_m - u_{m+1})/d_m.  Both recurrences contract by 2 - sqrt 3
// per step, so a chunk of unknowns started W steps early from zero is exact
// to (2 - sqrt 3)^{W+1}: W = 32 (1.4e-19) in FP64; W = 12 (3.7e-8) in FP32C,
// where M enters a value at weight |kappa| <= dx^2/24, so the truncation is a
// few 1e-12 of the value at most (below the FP32C resolution of the sums).
// One CTA owns a tile of kSplineTile unknowns: it loads the level values of
// the tile and its halo, forms r in shared memory, runs the forward sweep of
// each thread's chunk (warm-up from the left), then the backward sweep
// (warm-up from the right over the neighbouring chunks' g), all on chip.  In
// FP32C it then writes the second derivatives M of its nodes.
// ---------------------------------------------------------------------------
template <int PREC>
struct SplineT;
template <>
struct SplineT<BSDE_FP64> {
  using T = double;
  static constexpr int W = 32;
};
template <>
struct SplineT<BSDE_FP32C> {
  using T = float;
  static constexpr int W = 12;
};

// Shared-memory span of a spline tile of TS unknowns: the tile, W on the
// left and W + 2 on the right, and room for the FP32C sums' register windows
// to read up to kSplineChunkMax - 2 values past the last one they use.
constexpr int kSplineChunkMax = 8;
template <int PREC>
__host__ __device__ constexpr int spline_span(int TS) {
  return TS + 2 * SplineT<PREC>::W + kSplineChunkMax;
}

// One tile of TS unknowns of the level in `slot`, by the threads tid < nt of
// the CTA (all threads of the CTA must call it: it holds barriers); NT is the
// compile-time thread count the right-hand sides are spread over (nt >= NT).
// sr, sg: [2][spline_span(TS)] and sid: [kInvPivots] in shared memory;
// sid must hold the pivots 1/d_m in T before the call.
// Unknown m is M_{m+1}; the tile is unknowns [a, b), the forward sweep runs
// over [a, rb) and the backward one over [a, min(b + 1, u)) (one more on the
// right: FP32C cell b needs M_{b+1}).
template <int PREC, int TS, int NT>
__device__ __forceinline__ void spline_tile(const Params &P, Ring64 r64, Ring32 r32, int slot,
                                            int tile, int nt,
                                            typename SplineT<PREC>::T (*sr)[spline_span<PREC>(TS)],
                                            typename SplineT<PREC>::T (*sg)[spline_span<PREC>(TS)],
                                            const typename SplineT<PREC>::T *sid) {
  using T = typename SplineT<PREC>::T;
  constexpr int W = SplineT<PREC>::W;
  constexpr int C = kSplineChunk;
  const int u = int(P.Nx - 2);
  const int a = tile * TS;
  const int b = a + TS < u ? a + TS : u;
  const int ra = a - W > 0 ? a - W : 0;
  const int rb = b + W + 1 < u ? b + W + 1 : u;
  const int bx = b + 1 < u ? b + 1 : u;
  const int base = a - W;
  const int64_t off = int64_t(slot) * P.Nx;
  const int tid = threadIdx.x;
  if (a >= u) return;  // uniform over the CTA
  auto bar_sync = [] { __syncthreads(); };

  // right-hand sides r_m (m in [ra, rb)), in FP32C from the first
  // differences d_m = v_{m+1} - v_m, RC consecutive m per thread: the RC + 2
  // level values of a chunk are loaded together
  constexpr int RC = (TS + 2 * W + 2 + NT - 1) / NT;
  {
    const int m0 = ra + tid * RC;
    if (tid < NT && m0 <= rb) {
      if constexpr (PREC == BSDE_FP64) {
        double vy[RC + 2], vz[RC + 2];
#pragma unroll
        for (int q = 0; q < RC + 2; ++q) {
          const double4_32a v = m0 + q < rb + 2 ? ldl(r64.ring + off + m0 + q)
                                                : make_double4_32a(0.0, 0.0, 0.0, 0.0);
          vy[q] = v.x;
          vz[q] = v.z;
        }
#pragma unroll
        for (int q = 0; q < RC; ++q) {
          if (m0 + q < rb) {
            sr[0][m0 + q - base] = P.inv_dx2_6 * (vy[q] - 2.0 * vy[q + 1] + vy[q + 2]);
            sr[1][m0 + q - base] = P.inv_dx2_6 * (vz[q] - 2.0 * vz[q + 1] + vz[q + 2]);
          }
        }
      } else {
        // (hi, lo) pairs: neighbouring hi values differ exactly (Sterbenz)
        // away from sign changes, so the differences keep the pair precision
        float4 v[RC + 2];
#pragma unroll
        for (int q = 0; q < RC + 2; ++q)
          v[q] = m0 + q < rb + 2 ? ldl(r32.A + off + m0 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float inv6 = float(P.inv_dx2_6);
        float dy[RC + 1], dz[RC + 1];
#pragma unroll
        for (int q = 0; q < RC + 1; ++q) {
          dy[q] = __fadd_rn(__fsub_rn(v[q + 1].x, v[q].x), __fsub_rn(v[q + 1].z, v[q].z));
          dz[q] = __fadd_rn(__fsub_rn(v[q + 1].y, v[q].y), __fsub_rn(v[q + 1].w, v[q].w));
        }
#pragma unroll
        for (int q = 0; q < RC; ++q) {
          if (m0 + q < rb) {
            sr[0][m0 + q - base] = inv6 * __fsub_rn(dy[q + 1], dy[q]);
            sr[1][m0 + q - base] = inv6 * __fsub_rn(dz[q + 1], dz[q]);
          }
        }
      }
    }
  }
  __syncthreads();

  if constexpr (PREC == BSDE_FP64) {
    // forward sweep over the chunks of [a, rb): the tile and its right halo
    for (int s0 = a + tid * C; s0 < rb && tid < nt; s0 += nt * C) {
      const int e = s0 + C < rb ? s0 + C : rb;
      const int st = s0 - W > 0 ? s0 - W : 0;
      T gy = T(0), gz = T(0);
      for (int m = st; m < e; ++m) {
        const T id = m > 0 ? sid[m - 1 < kInvPivots ? m - 1 : kInvPivots - 1] : T(0);
        gy = sr[0][m - base] - gy * id;
        gz = sr[1][m - base] - gz * id;
        if (m >= s0) {
          sg[0][m - base] = gy;
          sg[1][m - base] = gz;
        }
      }
    }
    bar_sync();

    // backward sweep over the chunks of the tile, warm-up from the right
    for (int s0 = a + tid * C; s0 < b && tid < nt; s0 += nt * C) {
      const int e = s0 + C < b ? s0 + C : b;
      const int top = e + W < u ? e + W : u;
      T my = T(0), mz = T(0);
      for (int m = top - 1; m >= s0; --m) {
        const T id = sid[m < kInvPivots ? m : kInvPivots - 1];
        my = (sg[0][m - base] - my) * id;
        mz = (sg[1][m - base] - mz) * id;
        if (m < e) {
          r64.ring[off + m + 1].y = my;
          r64.ring[off + m + 1].w = mz;
        }
      }
    }
  } else {
    // FP32C: beyond the first kSplineHead unknowns the pivots are 2 + sqrt 3
    // to FP32 precision, and both recurrences become sums over W + 1 terms
    // with weights rho^q (rho = 1 / (2 + sqrt 3)), the same truncation as
    // the warm-up of a serial chunk but with no serial chain:
    //   g_m = sum_q (-rho)^q r_{m-q},     u_m = sum_q rho (-rho)^q g_{m+q}
    // (the backward sum stops at the last unknown, where u = rho g exactly).
    // The first tile runs its head (forward, m < H + W) and tail (backward,
    // m < H) serially with the exact pivots.
    constexpr int H = kSplineHead;
    constexpr int F0 = H + W;
    const T rho = sid[H];
    if (a < F0 && tid == 0) {
      T gy = T(0), gz = T(0);
      const int e = F0 < rb ? F0 : rb;
      for (int m = 0; m < e; ++m) {
        const T id = m > 0 ? sid[m - 1] : T(0);
        gy = sr[0][m - base] - gy * id;
        gz = sr[1][m - base] - gz * id;
        sg[0][m - base] = gy;
        sg[1][m - base] = gz;
      }
    }
    // Each thread takes CP consecutive unknowns and keeps the W + CP values
    // its sums read in registers, so a value is read from shared memory once
    // per thread instead of once per sum.  Every unknown's sum keeps its
    // terms and their order, so the results do not depend on CP or the
    // tiling.
    constexpr int CP = (TS + W + 1 + NT - 1) / NT;
    static_assert(CP <= kSplineChunkMax, "spline chunk wider than the shared-memory span allows");
    const int c0 = a + tid * CP;
    {
      const int lo = a > F0 ? a : F0;
      if (tid < nt && c0 < rb && c0 + CP > lo) {
        T wy[W + CP], wz[W + CP];  // r_{c0-W} .. r_{c0+CP-1}
#pragma unroll
        for (int t = 0; t < W + CP; ++t) {
          wy[t] = sr[0][c0 - W + t - base];
          wz[t] = sr[1][c0 - W + t - base];
        }
        T gy[CP], gz[CP];
#pragma unroll
        for (int t = 0; t < CP; ++t) {
          gy[t] = wy[W + t];
          gz[t] = wz[W + t];
        }
        T c = T(1);
#pragma unroll
        for (int q = 1; q <= W; ++q) {
          c = -c * rho;
#pragma unroll
          for (int t = 0; t < CP; ++t) {
            gy[t] = __fmaf_rn(c, wy[W + t - q], gy[t]);
            gz[t] = __fmaf_rn(c, wz[W + t - q], gz[t]);
          }
        }
#pragma unroll
        for (int t = 0; t < CP; ++t) {
          const int m = c0 + t;
          if (m >= lo && m < rb) {
            sg[0][m - base] = gy[t];
            sg[1][m - base] = gz[t];
          }
        }
      }
    }
    bar_sync();
    // backward: M of unknowns [a, bx) into sr (r is no longer needed)
    {
      const int lo = a > H ? a : H;
      if (tid < nt && c0 < bx && c0 + CP > lo) {
        T wy[W + CP], wz[W + CP];  // g_{c0} .. g_{c0+CP-1+W}
#pragma unroll
        for (int t = 0; t < W + CP; ++t) {
          wy[t] = sg[0][c0 + t - base];
          wz[t] = sg[1][c0 + t - base];
        }
        T my[CP], mz[CP];
#pragma unroll
        for (int t = 0; t < CP; ++t) my[t] = mz[t] = T(0);
        if (c0 + CP - 1 + W <= u - 1) {
          // every sum of the chunk has its W + 1 terms
          T c = rho;
#pragma unroll
          for (int q = 0; q <= W; ++q) {
#pragma unroll
            for (int t = 0; t < CP; ++t) {
              my[t] = __fmaf_rn(c, wy[t + q], my[t]);
              mz[t] = __fmaf_rn(c, wz[t + q], mz[t]);
            }
            c = -c * rho;
          }
        } else {
          // near the last unknown the sums stop there
#pragma unroll
          for (int t = 0; t < CP; ++t) {
            const int qmax = u - 1 - (c0 + t) < W ? u - 1 - (c0 + t) : W;
            T c = rho;
#pragma unroll
            for (int q = 0; q <= W; ++q) {
              if (q <= qmax) {
                my[t] = __fmaf_rn(c, wy[t + q], my[t]);
                mz[t] = __fmaf_rn(c, wz[t + q], mz[t]);
              }
              c = -c * rho;
            }
          }
        }
#pragma unroll
        for (int t = 0; t < CP; ++t) {
          const int m = c0 + t;
          if (m >= lo && m < bx) {
            sr[0][m - base] = my[t];
            sr[1][m - base] = mz[t];
          }
        }
      }
    }
    bar_sync();
    if (a < H && tid == 0) {
      const int e = H < bx ? H : bx;  // unknowns [a, e) serially, from u_e down
      T my = e < u ? sr[0][e - base] : T(0), mz = e < u ? sr[1][e - base] : T(0);
      for (int m = e - 1; m >= a; --m) {
        my = (sg[0][m - base] - my) * sid[m];
        mz = (sg[1][m - base] - mz) * sid[m];
        sr[0][m - base] = my;
        sr[1][m - base] = mz;
      }
    }
  }
  if constexpr (PREC == BSDE_FP64) {
    if (tile == 0 && tid == 0) {
      // natural end conditions M_0 = M_{Nx-1} = 0
      r64.ring[off].y = 0.0;
      r64.ring[off].w = 0.0;
      r64.ring[off + P.Nx - 1].y = 0.0;
      r64.ring[off + P.Nx - 1].w = 0.0;
    }
  } else {
    __syncthreads();
    // second derivatives of nodes a + 1 .. b (M_c is unknown c - 1), and of
    // node 0 for the first tile and node Nx - 1 for the last tile:
    // M_0 = M_{Nx-1} = 0 (natural spline)
    const int c0 = a == 0 ? 0 : a + 1;
    const int c1 = b == u ? u + 1 : b;  // inclusive
    for (int c = c0 + tid; c <= c1 && tid < nt; c += nt) {
      const bool end = c == 0 || c == u + 1;
      r32.M[off + c] = end ? make_float2(0.f, 0.f)
                           : make_float2(sr[0][c - 1 - base], sr[1][c - 1 - base]);
    }
  }
}


// The tiled spline kernel: FP64 runs tiles of kSplineTile unknowns, serial
// chunks of kSplineChunk unknowns per thread; FP32C tiles of 1011 unknowns,
// four consecutive unknowns per thread (its sweeps are sums, not chains),
// the forward sweep covering the tile and its right halo of W + 1 (1024).
// FP32C takes these wide tiles on grids that fill the GPU twice over; on
// smaller grids single solves run the warp-tiled k_spline32w below, and
// batches and the server run spline_tile inside their persistent kernels.
template <int PREC>
struct SplineLaunch {
  static constexpr int TS = PREC == BSDE_FP64 ? kSplineTile : 1011;
  static constexpr int NT = PREC == BSDE_FP64 ? kSplineTile / kSplineChunk : 256;
};

template <int PREC>
__global__ void __launch_bounds__(SplineLaunch<PREC>::NT)
    k_spline(const Params P, Ring64 r64, Ring32 r32, int slot) {
  using T = typename SplineT<PREC>::T;
  constexpr int TS = SplineLaunch<PREC>::TS, NT = SplineLaunch<PREC>::NT;
  constexpr int S = spline_span<PREC>(TS);
  __shared__ T sr[2][S], sg[2][S];
  __shared__ T sid[kInvPivots];
  if (threadIdx.x < kInvPivots) sid[threadIdx.x] = T(P.invd[threadIdx.x]);
  wait_predecessor();
  spline_tile<PREC, TS, NT>(P, r64, r32, slot, blockIdx.x, blockDim.x, sr, sg, sid);
}

// ---------------------------------------------------------------------------
// The FP32C spline of a single solve, warp-tiled.  Beyond the first tile the
// sweeps are the 13-term sums of spline_tile, evaluated without shared memory
// or block barriers: a warp holds 128 consecutive unknowns, 4 per lane (r
// from the lane's own level records), and takes the 12 values each sum needs
// from the neighbouring lanes by shuffles.  It outputs the 104 unknowns whose
// forward sums have their left terms and whose backward sums their right ones
// inside the warp (the first and last 12 are its halo).  Each sum keeps the
// terms, weights and order of spline_tile, so the second derivatives are
// bitwise those of the tiled kernel.  CTA 0 runs the first tile (unknowns
// 0..242: the exact serial head, node 0) with spline_tile itself.
// ---------------------------------------------------------------------------
constexpr int kSplWarpCP = 4;                                      // unknowns per lane
constexpr int kSplWarpOut = 32 * kSplWarpCP - 2 * SplineT<BSDE_FP32C>::W;  // 104
constexpr int kSplHeadTS = 243;                                    // CTA 0's tile
constexpr int kSplWarpThreads = 128;

// One warp tile of the level in `slot`: output unknowns [s0, s0 + 104) with
// s0 = kSplHeadTS + 104 wt (unknowns below kSplHeadTS are the first tile's).
// Called by all 32 lanes of a warp.
__device__ __forceinline__ void spline_warp_tile(const Params &P, Ring32 r32, int slot, int wt) {
  constexpr int W = SplineT<BSDE_FP32C>::W, CP = kSplWarpCP;
  const int u = int(P.Nx - 2);
  const int lane = threadIdx.x & 31;
  const int s0 = kSplHeadTS + wt * kSplWarpOut;  // first output unknown
  if (s0 >= u) return;                           // uniform over the warp
  const int64_t off = int64_t(slot) * P.Nx;
  const int m0 = s0 - W + lane * CP;             // the lane's unknowns m0 .. m0 + 3
  const float inv6 = float(P.inv_dx2_6);
  const float rho = float(P.invd[kSplineHead]);
  // r_m from the (hi, lo) pairs of nodes m, m + 1, m + 2 (as spline_tile)
  float ry[CP], rz[CP];
  {
    float4 v[CP + 2];
#pragma unroll
    for (int q = 0; q < CP + 2; ++q)
      v[q] = m0 + q <= u + 1 ? ldl(r32.A + off + m0 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    float dy[CP + 1], dz[CP + 1];
#pragma unroll
    for (int q = 0; q < CP + 1; ++q) {
      dy[q] = __fadd_rn(__fsub_rn(v[q + 1].x, v[q].x), __fsub_rn(v[q + 1].z, v[q].z));
      dz[q] = __fadd_rn(__fsub_rn(v[q + 1].y, v[q].y), __fsub_rn(v[q + 1].w, v[q].w));
    }
#pragma unroll
    for (int q = 0; q < CP; ++q) {
      const bool in = m0 + q < u;
      ry[q] = in ? __fmul_rn(inv6, __fsub_rn(dy[q + 1], dy[q])) : 0.f;
      rz[q] = in ? __fmul_rn(inv6, __fsub_rn(dz[q + 1], dz[q])) : 0.f;
    }
  }
  // forward: g_m = sum_q (-rho)^q r_{m-q}; the window r_{m0-W} .. r_{m0+3}
  // from lanes lane-3 .. lane (lanes 0..2 hold the halo: their g is unused)
  float gy[CP], gz[CP];
  {
    float wy[W + CP], wz[W + CP];
#pragma unroll
    for (int d = 1; d <= W / CP; ++d) {
#pragma unroll
      for (int t = 0; t < CP; ++t) {
        wy[W - d * CP + t] = __shfl_up_sync(0xffffffffu, ry[t], d);
        wz[W - d * CP + t] = __shfl_up_sync(0xffffffffu, rz[t], d);
      }
    }
#pragma unroll
    for (int t = 0; t < CP; ++t) {
      wy[W + t] = ry[t];
      wz[W + t] = rz[t];
      gy[t] = wy[W + t];
      gz[t] = wz[W + t];
    }
    float c = 1.f;
#pragma unroll
    for (int q = 1; q <= W; ++q) {
      c = -c * rho;
#pragma unroll
      for (int t = 0; t < CP; ++t) {
        gy[t] = __fmaf_rn(c, wy[W + t - q], gy[t]);
        gz[t] = __fmaf_rn(c, wz[W + t - q], gz[t]);
      }
    }
  }
  // backward: M_m = sum_q rho (-rho)^q g_{m+q}, stopping at the last
  // unknown; the window g_{m0} .. g_{m0+3+W} from lanes lane .. lane+3
  // (lanes 29..31 hold the halo: their M is not written)
  float wy[W + CP], wz[W + CP];
#pragma unroll
  for (int t = 0; t < CP; ++t) {
    wy[t] = gy[t];
    wz[t] = gz[t];
  }
#pragma unroll
  for (int d = 1; d <= W / CP; ++d) {
#pragma unroll
    for (int t = 0; t < CP; ++t) {
      wy[d * CP + t] = __shfl_down_sync(0xffffffffu, gy[t], d);
      wz[d * CP + t] = __shfl_down_sync(0xffffffffu, gz[t], d);
    }
  }
  const int e = s0 + kSplWarpOut < u ? s0 + kSplWarpOut : u;  // outputs [s0, e)
#pragma unroll
  for (int t = 0; t < CP; ++t) {
    const int m = m0 + t;
    if (m < s0 || m >= e) continue;
    const int qmax = u - 1 - m < W ? u - 1 - m : W;
    float my = 0.f, mz = 0.f, c = rho;
#pragma unroll
    for (int q = 0; q <= W; ++q) {
      if (q <= qmax) {
        my = __fmaf_rn(c, wy[t + q], my);
        mz = __fmaf_rn(c, wz[t + q], mz);
      }
      c = -c * rho;
    }
    r32.M[off + m + 1] = make_float2(my, mz);  // M of node m + 1
  }
  // natural end condition at the last node
  if (lane == 0 && u - 1 >= s0 && u - 1 < e) r32.M[off + u + 1] = make_float2(0.f, 0.f);
}

// Warp tiles of a level: ceil((u - kSplHeadTS) / 104) for u = Nx - 2 unknowns.
__host__ __device__ inline int spline_warp_tiles(int64_t Nx) {
  const int64_t u = Nx - 2;
  return u > kSplHeadTS ? int((u - kSplHeadTS + kSplWarpOut - 1) / kSplWarpOut) : 0;
}

__global__ void __launch_bounds__(kSplWarpThreads)
    k_spline32w(const Params P, Ring32 r32, int slot) {
  __shared__ float sr[2][spline_span<BSDE_FP32C>(kSplHeadTS)];
  __shared__ float sg[2][spline_span<BSDE_FP32C>(kSplHeadTS)];
  __shared__ float sid[kInvPivots];
  if (blockIdx.x == 0) {  // uniform over the CTA
    if (threadIdx.x < kInvPivots) sid[threadIdx.x] = float(P.invd[threadIdx.x]);
    wait_predecessor();
    spline_tile<BSDE_FP32C, kSplHeadTS, kSplWarpThreads>(
        P, Ring64{nullptr}, r32, slot, 0, blockDim.x, sr, sg, sid);
    return;
  }
  wait_predecessor();
  spline_warp_tile(P, r32, slot, (blockIdx.x - 1) * (kSplWarpThreads / 32) + (threadIdx.x >> 5));
}

// ---------------------------------------------------------------------------
// Picard statistics: per-warp maxima folded into the Stats block.  Every
// warp of every CTA reports, so an atomic is issued only when it would change
// the block (the fields only grow; the check reads them from L2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void record_picard(Stats *st, bool active, int it, double d,
                                              double tol) {
  const unsigned full = 0xffffffffu;
  const unsigned itm = __reduce_max_sync(full, active ? unsigned(it) : 0u);
  unsigned long long db = active ? (unsigned long long)__double_as_longlong(d) : 0ull;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(full, db, o);
    db = other > db ? other : db;
  }
  // not <= tol: a NaN step (the level overflowed) is non-convergence too
  const unsigned nc = __reduce_or_sync(full, (active && !(d <= tol)) ? 1u : 0u);
  if ((threadIdx.x & 31) == 0) {
    if (int(itm) > __ldcg(&st->iters_max)) atomicMax(&st->iters_max, int(itm));
    if (db > __ldcg(&st->resid_bits)) atomicMax(&st->resid_bits, db);
    if (nc && !__ldcg(&st->nonconv)) atomicOr(&st->nonconv, 1);
  }
}

// The same statistics from the FP32C tails: the test !(d <= picard_tol_f) is
// exactly !(d <= picard_tol) for a float d, and the maximum of non-negative
// floats (or NaN) is the maximum of their bit patterns, so the warp reduces
// 32-bit words and converts its maximum to double once.
__device__ __forceinline__ void record_picard32(Stats *st, bool active, int it, float d,
                                                float tol_f) {
  const unsigned full = 0xffffffffu;
  const unsigned itm = __reduce_max_sync(full, active ? unsigned(it) : 0u);
  const unsigned db = __reduce_max_sync(full, active ? __float_as_uint(d) : 0u);
  const unsigned nc = __reduce_or_sync(full, (active && !(d <= tol_f)) ? 1u : 0u);
  if ((threadIdx.x & 31) == 0) {
    const unsigned long long dd =
        (unsigned long long)__double_as_longlong(double(__uint_as_float(db)));
    if (int(itm) > __ldcg(&st->iters_max)) atomicMax(&st->iters_max, int(itm));
    if (dd > __ldcg(&st->resid_bits)) atomicMax(&st->resid_bits, dd);
    if (nc && !__ldcg(&st->nonconv)) atomicOr(&st->nonconv, 1);
  }
}

// ---------------------------------------------------------------------------
// S3: the step kernels.  A CTA owns kStepTP consecutive grid points and runs
// G = k S groups of threads over them; group g takes j = g / S + 1 and the
// l-chunk g % S of the Gauss-Hermite nodes (Eq. 21).  For every node a thread
// forms the spline values of y^{n+j} and z^{n+j} at the off-grid point (cell
// i + shift_jl, the same for every i on the uniform grid), evaluates the
// driver there and accumulates the folded sums of Eq. 20 (see NodeF64).  The
// groups' partial sums meet in shared memory; the first group then forms
// z^n, runs the Picard iteration for y^n and writes the new level.
// A warp covers 32 consecutive points of one group, so every node load is a
// coalesced window.  CTAs whose points keep all their nodes of level n+j
// inside [0, Nx-1] skip the boundary clamping (Section 3.2 first remark).
// ---------------------------------------------------------------------------
template <bool CLAMP, typename W4>
__device__ __forceinline__ void node_cells(int ii, int shift, int last, int &c0, int &c1,
                                           W4 &w0, W4 &w1, W4 &w2, W4 &w3) {
  c0 = ii + shift;
  c1 = c0 + 1;
  if (CLAMP) {
    const bool cl = c0 < 0, ch = c0 >= last;
    if (cl | ch) {
      c0 = cl ? 0 : last;
      c1 = c0;
      w0 = W4(1);
      w1 = W4(0);
      w2 = W4(0);
      w3 = W4(0);
    }
  }
}

// yj: this level is n + K_y (E[y^] enters A); zf: the E[y DeltaW] z form's
// y^ term (j = 1).
template <int DRV, bool CLAMP>
__device__ __forceinline__ void nodes64(const DrvC<double> &dc, const double4_32a *__restrict__ lev,
                                        const NodeF64 *row, int l0, int l1, int ii, int last,
                                        double tj, double et, double emt, bool yj, bool zf,
                                        double &Zs, double &Ys) {
#pragma unroll 4
  for (int l = l0; l < l1; ++l) {
    const NodeF64 &e = row[l];
    double w0 = e.w0, w1 = e.w1, w2 = e.w2, w3 = e.w3;
    int c0, c1;
    node_cells<CLAMP>(ii, e.shift, last, c0, c1, w0, w1, w2, w3);
    const double4_32a a = lev[c0], b = lev[c1];
    const double yh = w0 * a.x + w1 * b.x + w2 * a.y + w3 * b.y;
    const double zh = w0 * a.z + w1 * b.z + w2 * a.w + w3 * b.w;
    const double F = driver<DRV>(dc, tj, et, emt, yh, zh);
    Zs += e.cz * zh + e.cfz * F;
    Ys += e.cfy * F;
    if (yj) Ys += e.cy * yh;
    if (zf) Zs += e.cyz * yh;
  }
}

template <int DRV>
__global__ void __launch_bounds__(kStepTP * kMaxGroups)
    k_step64(const Params P, const DrvC<double> dc, double4_32a *__restrict__ ring,
             const NodeF64 *__restrict__ table, int n, Stats *st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int kL = P.k * P.L;
  NodeF64 *tab = reinterpret_cast<NodeF64 *>(smem_raw);
  double *part = reinterpret_cast<double *>(smem_raw + sizeof(NodeF64) * kL);  // [2][G][TP]
  for (int t = threadIdx.x; t < kL; t += blockDim.x) tab[t] = table[t];
  __syncthreads();
  wait_predecessor();

  const int tp = threadIdx.x % kStepTP, g = threadIdx.x / kStepTP;
  const int j = g / P.S + 1, lc = g % P.S;
  const int l0 = lc * P.Lg, l1 = l0 + P.Lg < P.L ? l0 + P.Lg : P.L;
  const int i0 = blockIdx.x * kStepTP, ii = i0 + tp;
  const int last = int(P.Nx - 1);
  double Zs = 0.0, Ys = 0.0;
  if (ii <= last) {
    const double4_32a *lev = ring + int64_t((n + j) % P.nslot) * P.Nx;
    const double tj = (n + j) * P.dt;
    double et = 0.0, emt = 0.0;  // Example 2's driver only
    if constexpr (DRV == BSDE_DRIVER_EX2) {
      et = exp(tj * tj);
      emt = exp(-tj * tj);
    }
    const NodeF64 *row = tab + (j - 1) * P.L;
    const bool interior = i0 + P.smin[j - 1] >= 0 && i0 + kStepTP + P.smax[j - 1] <= last;
    const bool yj = j == P.ky, zf = P.zform && j == 1;
    if (interior)
      nodes64<DRV, false>(dc, lev, row, l0, l1, ii, last, tj, et, emt, yj, zf, Zs, Ys);
    else
      nodes64<DRV, true>(dc, lev, row, l0, l1, ii, last, tj, et, emt, yj, zf, Zs, Ys);
  }
  part[(0 * P.G + g) * kStepTP + tp] = Zs;
  part[(1 * P.G + g) * kStepTP + tp] = Ys;
  __syncthreads();
  if (g != 0) return;

  const bool active = ii <= last;
  int it = 0;
  double d = 0.0;
  if (active) {
    double z = 0.0, A = 0.0;
    for (int q = 0; q < P.G; ++q) {
      z += part[(0 * P.G + q) * kStepTP + tp];
      A += part[(1 * P.G + q) * kStepTP + tp];
    }
    const double tn = n * P.dt;
    const double etn = exp(tn * tn), emtn = exp(-tn * tn);
    double y = ring[int64_t((n + 1) % P.nslot) * P.Nx + ii].x;
    while (it < P.picard_max) {
      const double y1 = A + P.hg0 * driver<DRV>(dc, tn, etn, emtn, y, z);
      d = fabs(y1 - y);
      y = y1;
      ++it;
      if (d <= P.picard_tol || !isfinite(d)) break;  // a non-finite step cannot converge
    }
    ring[int64_t(n % P.nslot) * P.Nx + ii] = make_double4_32a(y, 0.0, z, 0.0);
  }
  record_picard(st, active, it, d, P.picard_tol);
}

// ---------------------------------------------------------------------------
// The general forward path (FP64): the forward process is advanced from the
// grid point by one Euler step, X = x_i + a(x_i) j dt + b(x_i) DeltaW_jl with
// a, b affine in x, so a node's position, cell and spline weights depend on
// the point; the driver may read X (SHORT_RATE).  Otherwise as k_step64:
// same groups, same table weights (cz, cfz, cfy, cy, cyz), same Picard tail.
// ---------------------------------------------------------------------------
template <int DRV, typename T>
__device__ __forceinline__ T driver_x(const DrvC<T> &dc, T t, T et, T emt, T x, T y, T z) {
  if constexpr (DRV == BSDE_DRIVER_SHORT_RATE)
    return -rmul(x, y);
  else
    return driver<DRV>(dc, t, et, emt, y, z);
}

template <int DRV>
__global__ void __launch_bounds__(kStepTP * kMaxGroups)
    k_step64_gen(const Params P, const DrvC<double> dc, double4_32a *__restrict__ ring,
                 const NodeF64 *__restrict__ table, int n, Stats *st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int kL = P.k * P.L;
  NodeF64 *tab = reinterpret_cast<NodeF64 *>(smem_raw);
  double *part = reinterpret_cast<double *>(smem_raw + sizeof(NodeF64) * kL);  // [2][G][TP]
  for (int t = threadIdx.x; t < kL; t += blockDim.x) tab[t] = table[t];
  __syncthreads();
  wait_predecessor();

  const int tp = threadIdx.x % kStepTP, g = threadIdx.x / kStepTP;
  const int j = g / P.S + 1, lc = g % P.S;
  const int l0 = lc * P.Lg, l1 = l0 + P.Lg < P.L ? l0 + P.Lg : P.L;
  const int ii = blockIdx.x * kStepTP + tp;
  const int last = int(P.Nx - 1);
  const double xi = P.x_min + double(ii) * P.dx;
  double Zs = 0.0, Ys = 0.0;
  if (ii <= last) {
    const double4_32a *lev = ring + int64_t((n + j) % P.nslot) * P.Nx;
    const double tj = __dmul_rn(double(n + j), P.dt);
    double et = 0.0, emt = 0.0;
    if constexpr (DRV == BSDE_DRIVER_EX2) {
      et = exp(tj * tj);
      emt = exp(-tj * tj);
    }
    const NodeF64 *row = tab + (j - 1) * P.L;
    const bool yj = j == P.ky, zf = P.zform && j == 1;
    const double ax = P.a_x + P.a_1 * xi, bx = P.b_x + P.b_1 * xi;
    const double drift = ax * double(j) * P.dt;
    const double c6 = P.c6;
#pragma unroll 2
    for (int l = l0; l < l1; ++l) {
      const NodeF64 &e = row[l];
      const double X = xi + drift + bx * e.dW;
      const double s = (X - P.x_min) * P.inv_dx;
      double yh, zh;
      if (s <= 0.0) {  // off the grid: the end values (Section 3.2)
        const double4_32a a = lev[0];
        yh = a.x;
        zh = a.z;
      } else if (s >= double(last)) {
        const double4_32a a = lev[last];
        yh = a.x;
        zh = a.z;
      } else {
        int c = int(floor(s));
        c = c > last - 1 ? last - 1 : c;
        const double th = s - double(c), om = 1.0 - th;
        const double w2 = c6 * (om * om * om - om), w3 = c6 * (th * th * th - th);
        const double4_32a a = lev[c], b = lev[c + 1];
        yh = om * a.x + th * b.x + (w2 * a.y + w3 * b.y);
        zh = om * a.z + th * b.z + (w2 * a.w + w3 * b.w);
      }
      const double F = driver_x<DRV>(dc, tj, et, emt, X, yh, zh);
      Zs += e.cz * zh + e.cfz * F;
      Ys += e.cfy * F;
      if (yj) Ys += e.cy * yh;
      if (zf) Zs += e.cyz * yh;
    }
  }
  part[(0 * P.G + g) * kStepTP + tp] = Zs;
  part[(1 * P.G + g) * kStepTP + tp] = Ys;
  __syncthreads();
  if (g != 0) return;

  const bool active = ii <= last;
  int it = 0;
  double d = 0.0;
  if (active) {
    double z = 0.0, A = 0.0;
    for (int q = 0; q < P.G; ++q) {
      z += part[(0 * P.G + q) * kStepTP + tp];
      A += part[(1 * P.G + q) * kStepTP + tp];
    }
    const double tn = __dmul_rn(double(n), P.dt);
    const double etn = exp(tn * tn), emtn = exp(-tn * tn);
    double y = ring[int64_t((n + 1) % P.nslot) * P.Nx + ii].x;
    while (it < P.picard_max) {
      const double y1 = A + P.hg0 * driver_x<DRV>(dc, tn, etn, emtn, xi, y, z);
      d = fabs(y1 - y);
      y = y1;
      ++it;
      if (d <= P.picard_tol || !isfinite(d)) break;  // a non-finite step cannot converge
    }
    ring[int64_t(n % P.nslot) * P.Nx + ii] = make_double4_32a(y, 0.0, z, 0.0);
  }
  record_picard(st, active, it, d, P.picard_tol);
}

// ---------------------------------------------------------------------------
// FP32C: the spline value at a node is kept as the unevaluated sum hi_c + del,
// del = theta (v_{c+1} - v_c) + lo_c + (spline-curvature part), computed in
// FP32 (|del| ~ dx |y'|, so its rounding is far below that of y).  The z and
// y sums take the exact product of the coefficient's hi part with hi_c (FMA)
// and add it by TwoSum into an (S, C) pair; the driver terms, which carry a
// dt-sized or sqrt(dt)-sized weight, are summed in plain FP32 (the y driver
// terms with their rounding error).  z^n and the explicit part A of y^n are
// formed as normalized float pairs, and the Picard iteration runs in FP32 on
// the increment y^n - A (finish_points32).
// y and z go through the same arithmetic with the same weights, so it runs on
// (y, z) lane pairs with packed FP32x2 instructions (one instruction, two
// correctly rounded results).
// ---------------------------------------------------------------------------
// Packed FP32x2 operations.  Written as inline PTX on 64-bit register pairs
// so that the two lanes stay in one aligned register pair from load to use.
#define BSDE_F2_OP2(name, op)                                                           \
  __device__ __forceinline__ float2 name(float2 a, float2 b) {                         \
    float2 d;                                                                           \
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"  \
        " " op ".rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"                       \
        : "=f"(d.x), "=f"(d.y)                                                          \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                      \
    return d;                                                                           \
  }
BSDE_F2_OP2(f2add, "add")
BSDE_F2_OP2(f2sub, "sub")
BSDE_F2_OP2(f2mul, "mul")
#undef BSDE_F2_OP2
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.x, v.y); }

// s + e = a + b exactly, lane by lane (TwoSum)
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
  s = f2add(a, b);
  const float2 bp = f2sub(s, a);
  e = f2add(f2sub(a, f2sub(s, bp)), f2sub(b, bp));
}

// S += ch*hi exactly (error-free product by FMA, TwoSum), C += the rounding
// errors plus the small terms ch*del + cl*hi; nch = -ch, ncl = -cl.  The
// product error is formed negated (-e = nch*hi + p), which keeps every step a
// plain FMA, add or subtract.
__device__ __forceinline__ void comp_acc2(float2 &S, float2 &C, float2 ch, float2 nch,
                                          float2 ncl, float2 hi, float2 del) {
  const float2 p = f2mul(ch, hi);
  const float2 ne = f2fma(nch, hi, p);
  const float2 sn = f2add(S, p);
  const float2 bp = f2sub(sn, S);
  const float2 err = f2add(f2sub(S, f2sub(sn, bp)), f2sub(p, bp));
  S = sn;
  // -(ch*del + cl*hi + e) = nch*del + (ncl*hi + (-e))
  const float2 nt = f2fma(nch, del, f2fma(ncl, hi, ne));
  C = f2sub(f2add(C, err), nt);
}

// One lane of comp_acc2: S += ch*hi exactly, C += the rounding errors plus
// ch*del + cl*hi.
__device__ __forceinline__ void comp_acc1(float &S, float &C, float ch, float cl, float hi,
                                          float del) {
  const float p = __fmul_rn(ch, hi);
  const float e = __fmaf_rn(ch, hi, -p);
  const float sn = __fadd_rn(S, p);
  const float bp = __fsub_rn(sn, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(sn, bp)), __fsub_rn(p, bp));
  S = sn;
  C = __fadd_rn(C, __fadd_rn(err, __fmaf_rn(ch, del, __fmaf_rn(cl, hi, e))));
}

__device__ __forceinline__ void two_sum_into(float &S, float &C, float x) {
  const float s = __fadd_rn(S, x);
  const float bp = __fsub_rn(s, S);
  C = __fadd_rn(C, __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(x, bp)));
  S = s;
}

// ---------------------------------------------------------------------------
// Device clock for bounded waits (ns).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Cell of one node for point ii.  A node off the grid clamps to the end
// value: the cell becomes the end node and the caller zeroes the weights.
template <bool CLAMP>
__device__ __forceinline__ bool pair_cell(int ii, int shift, int last, int &c) {
  c = ii + shift;
  if (CLAMP) {
    const bool lo = c < 0, hi = c >= last;
    if (lo | hi) {
      c = lo ? 0 : last;
      return true;
    }
  }
  return false;
}

// (y, z) spline value of one node as hi + del from the level data of the
// ends of its cell c: node records a0 = A_c, a1 = A_{c+1} (y_hi, z_hi,
// y_lo, z_lo) and second derivatives m0 = M_c, m1 = M_{c+1} (see Ring32);
// th = (theta, theta), ka = (kappa, kappa).  d = v_{c+1} - v_c is formed
// from exact float differences of the pairs (neighbouring hi values differ
// exactly away from sign changes), as the spline kernel forms its
// right-hand sides.
__device__ __forceinline__ void node_value(const float4 &a0, const float4 &a1, const float2 &m0,
                                           const float2 &m1, float2 th, float2 ka, float2 &hi,
                                           float2 &del) {
  hi = hi2(a0);
  const float2 d = f2add(f2sub(hi2(a1), hi2(a0)), f2sub(lo2(a1), lo2(a0)));
  const float2 Pc = f2fma(make_float2(2.f, 2.f), m0, m1), Qc = f2sub(m1, m0);
  del = f2fma(ka, f2fma(th, Qc, Pc), f2fma(th, d, lo2(a0)));
}

// The arithmetic of one node pair (see PairF32 for the entry e0..e4), given
// the level data of the ends of the two nodes' cells (node a: aa0, aa1,
// ma0, ma1; node b likewise).  S, C: compensated (y, z) sums; Fz, Fy: driver
// terms.  ZF: the E[y DeltaW] z form's term cyz (y^_a - y^_b) joins the z
// sum (compensated, the difference formed exactly by TwoSum).
template <int DRV, bool ZF = false>
__device__ __forceinline__ void pair_math(const DrvC<float> &dc, float tj, float et, float emt,
                                          const float4 &e0, const float4 &e1, const float4 &e2,
                                          const float4 &e3, const float4 &e4, const float4 &aa0,
                                          const float4 &aa1, const float2 &ma0, const float2 &ma1,
                                          const float4 &ba0, const float4 &ba1, const float2 &mb0,
                                          const float2 &mb1, float2 &S, float2 &C, float &Fz,
                                          float &Fy, float &FyC) {
  float2 ha, da, hb, db;
  node_value(aa0, aa1, ma0, ma1, hi2(e1), lo2(e1), ha, da);
  node_value(ba0, ba1, mb0, mb1, hi2(e2), lo2(e2), hb, db);
  const float2 va = f2add(ha, da), vb = f2add(hb, db);
  const float Fa = driver<DRV>(dc, tj, et, emt, va.x, va.y);
  const float Fb = driver<DRV>(dc, tj, et, emt, vb.x, vb.y);
  Fz = __fmaf_rn(e0.z, __fsub_rn(Fa, Fb), Fz);
  // sum of k dt gy_j f: O(k dt |f|), so accumulated with its rounding error
  two_sum_into(Fy, FyC, __fmul_rn(e0.w, __fadd_rn(Fa, Fb)));
  // the pair's hi parts summed exactly, then one compensated product
  float2 hs, he;
  two_sum2(ha, hb, hs, he);
  comp_acc2(S, C, hi2(e3), lo2(e3), hi2(e4), hs, f2add(f2add(da, db), he));
  if constexpr (ZF) {
    float dh = 0.f, dl = 0.f;
    dh = ha.x;
    two_sum_into(dh, dl, -hb.x);
    comp_acc1(S.y, C.y, e4.z, e4.w, dh, __fadd_rn(dl, __fsub_rn(da.x, db.x)));
  }
}

// Accumulators of one point: compensated (y, z) sums and the driver terms.
struct Acc32 {
  float2 S, C;
  float Fz, Fy, FyC;  // Fy + FyC: the y driver terms with their rounding error
};

// One group's node pairs for point ii, level data loaded directly from
// global memory (L1/L2).  With CLAMP false every cell must lie on the grid.
// UNR: pairs unrolled together, so the next pair's loads can be issued
// before the current pair's arithmetic (2 pays in the single-solve flat
// kernel, 2% at config3, whose threads have the registers; the grouped tiles
// and the batch kernel, which would spill, keep 1).
template <int DRV, bool CLAMP, bool ZF = false, int UNR = 1>
__device__ __forceinline__ void pairs32(const DrvC<float> &dc, Ring32 r, int64_t off,
                                        const PairF32 *row, int q0, int q1, int ii, int last,
                                        float tj, float et, float emt, Acc32 &acc) {
  const float4 *A = r.A + off;
  const float2 *M = r.M + off;
#pragma unroll UNR
  for (int q = q0; q < q1; ++q) {
    const float4 *te = reinterpret_cast<const float4 *>(row + q);
    const float4 e0 = te[0], e3 = te[3], e4 = te[4];
    float4 e1 = te[1], e2 = te[2];
    int ca, cb;
    if (pair_cell<CLAMP>(ii, __float_as_int(e0.x), last, ca)) e1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pair_cell<CLAMP>(ii, __float_as_int(e0.y), last, cb)) e2 = make_float4(0.f, 0.f, 0.f, 0.f);
    // the cell's right end (a clamped node sits on an end node with zero
    // weights, so its right end is the node itself)
    const int ca1 = CLAMP && ca == last ? ca : ca + 1, cb1 = CLAMP && cb == last ? cb : cb + 1;
    const float4 aa0 = ldl(A + ca), aa1 = ldl(A + ca1), ba0 = ldl(A + cb), ba1 = ldl(A + cb1);
    const float2 ma0 = ldl(M + ca), ma1 = ldl(M + ca1), mb0 = ldl(M + cb), mb1 = ldl(M + cb1);
    pair_math<DRV, ZF>(dc, tj, et, emt, e0, e1, e2, e3, e4, aa0, aa1, ma0, ma1, ba0, ba1, mb0,
                       mb1, acc.S, acc.C, acc.Fz, acc.Fy, acc.FyC);
  }
}

// Group g of a tile: pairs q0..q1 of level n + j, g = (j - 1) S + chunk.
struct Group32 {
  int j, q0, q1;
  bool interior;  // every node cell of every point of the tile on the grid
};
__device__ __forceinline__ Group32 group32(const Params &P, int g, int i0) {
  Group32 w;
  w.j = g / P.S + 1;
  const int lc = g % P.S;
  w.q0 = lc * P.Lg;
  w.q1 = w.q0 + P.Lg < P.Lp ? w.q0 + P.Lg : P.Lp;
  w.interior = i0 + P.smin[w.j - 1] >= 0 && i0 + kStepTP + P.smax[w.j - 1] <= int(P.Nx - 1);
  return w;
}

// Driver time constants of level m (t, exp(t^2), exp(-t^2) for Example 2).
template <int DRV>
__device__ __forceinline__ void level_time(const Params &P, int m, float &t, float &et,
                                           float &emt) {
  const double td = m * P.dt;
  t = float(td);
  et = emt = 0.f;
  if constexpr (DRV == BSDE_DRIVER_EX2) {
    et = float(exp(td * td));
    emt = float(exp(-td * td));
  }
}

__device__ __forceinline__ void store_partials(float *part, int G, int g, int tp,
                                               const Acc32 &a) {
  // lanes: y (x), z (y); part is [kPartArrays][G][kStepTP]
  const int o = g * kStepTP + tp, gs = G * kStepTP;
  part[0 * gs + o] = a.S.y;
  part[1 * gs + o] = a.C.y;
  part[2 * gs + o] = a.Fz;
  part[3 * gs + o] = a.Fy;
  part[4 * gs + o] = a.S.x;
  part[5 * gs + o] = a.C.x;
  part[6 * gs + o] = a.FyC;
}

// Whether a Picard two-cycle (delta^(p+1) == delta^(p-1)) of step d is the
// rounding of the FP32 iteration and not an oscillation: d within 2^-22 of
// |y| + |delta| (two to four ulps of the larger), y = A + delta being the
// argument the FP32 driver sees and delta the increment it returns.
__device__ __forceinline__ bool picard_cycle_ok(float d, float y, float delta) {
  return d <= __fmul_rn(__fadd_rn(fabsf(y), fabsf(delta)), 2.384185791015625e-7f);
}

// The last part of the step for the kStepTP points of a tile, by the threads
// tid < kStepTP of the CTA (the others pass through; all threads call it):
// the groups' partial sums are added, z^n and the explicit part A of y^n are
// formed as normalized float pairs (hi + lo, ~48 significant bits), y^n is
// found by Picard iteration on the increment delta = y^n - A =
// k dt gy_0 f(t_n, A + delta, z^n), and (y^n, z^n) is stored.
// The driver sees y in FP32, so the iteration runs in FP32; the test
// |delta^(p+1) - delta^(p)| <= tol is exact (near convergence the two
// increments are within a factor two, so their float difference carries no
// rounding; a float is <= tol exactly when it is <= picard_tol_f).  A
// two-cycle whose step is within a couple of ulps of the FP32 argument
// A + delta or of the increment (picard_cycle_ok) is that argument's rounding
// flipping between neighbours, as far as the FP32 driver can resolve, and
// ends it too; a wider cycle is an oscillation of the iteration itself and
// runs on to picard_max, where it is reported as non-convergence.
// The groups' partial sums of one point, folded in group order: compensated
// z and y sums (S, C), the z driver terms and the y driver terms with their
// rounding error.
struct Sums32 {
  float zS, zC, fz, fy, fyC, yS, yC;
};
__device__ __forceinline__ void fold_group(Sums32 &s, float Sy, float Cy, float Fz, float Fy,
                                           float Sx, float Cx, float FyC) {
  two_sum_into(s.zS, s.zC, Sy);
  s.zC = __fadd_rn(s.zC, Cy);
  s.fz = __fadd_rn(s.fz, Fz);
  two_sum_into(s.fy, s.fyC, Fy);
  s.fyC = __fadd_rn(s.fyC, FyC);
  two_sum_into(s.yS, s.yC, Sx);
  s.yC = __fadd_rn(s.yC, Cx);
}

// z^n, A and the Picard iteration for point ii from its folded sums (see
// finish_points32); stores (y^n, z^n), returns the last step and the
// iteration count in it.
template <int DRV>
__device__ __forceinline__ float finish_point32(const Params &P, const DrvC<float> &dc,
                                                float4 *__restrict__ ringA, int n, int ii,
                                                const Sums32 &s, float prev_y, int &it) {
  float d = 0.f;
  // z^n = zS + (zC + fz) and A = yS + (yC + fy) as exact float pairs
  float zh = s.zS, zl = 0.f, Ah = s.yS, Al = 0.f;
  two_sum_into(zh, zl, __fadd_rn(s.zC, s.fz));
  two_sum_into(Ah, Al, s.fy);
  two_sum_into(Ah, Al, __fadd_rn(s.yC, s.fyC));
  float tn, etn, emtn;
  level_time<DRV>(P, n, tn, etn, emtn);
  const float hg0 = P.hg0_f;
  float dl = __fsub_rn(prev_y, Ah), dpp = __int_as_float(0x7fc00000);
  // the forward state at the point, for x-aware drivers only
  float xf = 0.f;
  if constexpr (DRV == BSDE_DRIVER_SHORT_RATE) xf = float(P.x_min + double(ii) * P.dx);
  while (it < P.picard_max) {
    const float dn = hg0 * driver_x<DRV>(dc, tn, etn, emtn, xf, Ah + dl, zh);
    ++it;
    d = fabsf(__fsub_rn(dn, dl));
    const bool cyc = dn == dpp && picard_cycle_ok(d, __fadd_rn(Ah, dl), dn);
    dpp = dl;
    dl = dn;
    if (cyc) d = 0.f;
    if (d <= P.picard_tol_f || !isfinite(d)) break;  // a non-finite step cannot converge
  }
  // y^n = A + delta, renormalized
  float yh = Ah, yl = Al;
  two_sum_into(yh, yl, dl);
  const float sy = __fadd_rn(yh, yl);
  yl = __fsub_rn(yl, __fsub_rn(sy, yh));
  yh = sy;
  const float sz = __fadd_rn(zh, zl);
  zl = __fsub_rn(zl, __fsub_rn(sz, zh));
  zh = sz;
  ringA[int64_t(n % P.nslot) * P.Nx + ii] = make_float4(yh, zh, yl, zl);
  return d;
}

template <int DRV>
__device__ __forceinline__ void finish_points32(const Params &P, const DrvC<float> &dc,
                                                float4 *__restrict__ ringA, const float *part,
                                                int G, int n, int i0, Stats *st, float prev_y) {
  const int tid = threadIdx.x;
  const int ii = i0 + tid;
  const bool active = tid < kStepTP && ii <= int(P.Nx - 1);
  int it = 0;
  float d = 0.f;
  if (active) {
    const int gs = G * kStepTP;
    Sums32 s{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < G; ++q) {
      const int o = q * kStepTP + tid;
      fold_group(s, part[0 * gs + o], part[1 * gs + o], part[2 * gs + o], part[3 * gs + o],
                 part[4 * gs + o], part[5 * gs + o], part[6 * gs + o]);
    }
    d = finish_point32<DRV>(P, dc, ringA, n, ii, s, prev_y, it);
  }
  record_picard32(st, active, it, d, P.picard_tol_f);
}

// One tile of kStepTP points of level n with direct loads, called by every
// thread of the CTA; `tab` is the pair table of the problem (in shared memory
// or in the kernel's parameters) and `part` is in shared memory.  Thread tp
// of group g accumulates the pairs of group g for point i0 + tp; threads of
// groups g >= G idle.  The caller separates consecutive tiles by a barrier
// (part is reused).
template <int DRV>
__device__ __forceinline__ void step_tile32(const Params &P, const DrvC<float> &dc, Ring32 r32,
                                            const PairF32 *tab, float *part, int n, int i0,
                                            Stats *st) {
  const int tp = threadIdx.x % kStepTP, g = threadIdx.x / kStepTP;
  const int G = P.G;
  const int last = int(P.Nx - 1);
  // the Picard start y^{n+1} of the points this thread finishes, loaded early
  float prev_y = 0.f;
  if (threadIdx.x < kStepTP && i0 + int(threadIdx.x) <= last)
    prev_y = ldl(r32.A + int64_t((n + 1) % P.nslot) * P.Nx + i0 + threadIdx.x).x;
  if (g < G) {
    const Group32 w = group32(P, g, i0);
    Acc32 acc{make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f, 0.f, 0.f};
    const int64_t off = int64_t((n + w.j) % P.nslot) * P.Nx;
    float tj, et, emt;
    level_time<DRV>(P, n + w.j, tj, et, emt);
    const PairF32 *row = tab + (w.j - 1) * P.Lp;
    if (P.zform && w.j == 1)  // the E[y DeltaW] z form (clamping always on)
      pairs32<DRV, true, true>(dc, r32, off, row, w.q0, w.q1, i0 + tp, last, tj, et, emt, acc);
    else if (w.interior)
      pairs32<DRV, false>(dc, r32, off, row, w.q0, w.q1, i0 + tp, last, tj, et, emt, acc);
    else  // cells clamp onto the grid, so points past the end are harmless
      pairs32<DRV, true>(dc, r32, off, row, w.q0, w.q1, i0 + tp, last, tj, et, emt, acc);
    store_partials(part, G, g, tp, acc);
  }
  __syncthreads();
  finish_points32<DRV>(P, dc, r32.A, part, G, n, i0, st, prev_y);
}


// ---------------------------------------------------------------------------
// The FP32C step kernel of one level: one CTA per tile of kStepTP points and
// G groups of kStepTP threads, level data loaded through L1 from the
// L2-resident ring.  The pair table is a kernel parameter: every thread of a
// group reads the same entry, so the reads go through the constant cache and
// leave the L1 data path to the level loads (and no CTA copies the table).
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t step32_smem(int G, int kP) {
  return sizeof(PairF32) * size_t(kP) + sizeof(float) * kPartArrays * size_t(G) * kStepTP;
}

// The pair table of a plan (k Lp entries used) as a kernel parameter.
struct PairTab32 {
  PairF32 e[kMaxK * (kMaxL / 2)];
};
// kernel parameters are limited to 32764 bytes
static_assert(sizeof(Params) + sizeof(DrvC<float>) + sizeof(Ring32) + sizeof(PairTab32) + 16 <=
                  32764,
              "k_step32 parameters exceed the kernel parameter limit");

template <int DRV>
__global__ void __launch_bounds__(kStepTP * kMaxGroups, 3)
    k_step32(const Params P, const DrvC<float> dc, Ring32 r32,
             const __grid_constant__ PairTab32 tab, int n, Stats *st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float *part = reinterpret_cast<float *>(smem_raw);  // [kPartArrays][G][kStepTP]
  wait_predecessor();
  step_tile32<DRV>(P, dc, r32, tab.e, part, n, blockIdx.x * kStepTP, st);
}

// ---------------------------------------------------------------------------
// The FP32C step kernel for grids that fill the GPU several times over: one
// thread per grid point runs all G groups of its point, in group order, with
// the grouped kernel's pairs, arithmetic and fold (fold_group), so its
// results are bitwise those of k_step32 with the same work split.  The group
// and pair indices are loop counters, uniform across the CTA, so the pair
// table in the kernel parameters is read by uniform constant loads; there
// are no shared-memory partial sums and no barrier.
// ---------------------------------------------------------------------------
constexpr int kFlatTP = 128;  // grid points (threads) per CTA

// One flat tile: blockDim.x consecutive points from i0, one per thread, all
// groups of a point in turn.  `tab` is the pair table (kernel parameters or
// shared memory: its reads are uniform across the CTA either way).  Needs no
// barrier, before or after.  UNR as for pairs32 (the interior pairs).
template <int DRV, int UNR = 1>
__device__ __forceinline__ void step_tile32f(const Params &P, const DrvC<float> &dc, Ring32 r32,
                                             const PairF32 *tab, int n, int i0, Stats *st) {
  const int ii = i0 + int(threadIdx.x);
  const int last = int(P.Nx - 1);
  const int tw = int(blockDim.x);
  const bool active = ii <= last;
  float prev_y = 0.f;
  if (active) prev_y = ldl(r32.A + int64_t((n + 1) % P.nslot) * P.Nx + ii).x;
  Sums32 s{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int g = 0; g < P.G; ++g) {
    const int j = g / P.S + 1, lc = g % P.S;
    const int q0 = lc * P.Lg, q1 = q0 + P.Lg < P.Lp ? q0 + P.Lg : P.Lp;
    // every node cell of every point of the tile on the grid (points past the
    // end take the clamping path, whose cells stay on the grid)
    const bool interior = i0 + P.smin[j - 1] >= 0 && i0 + tw + P.smax[j - 1] <= last;
    Acc32 acc{make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f, 0.f, 0.f};
    const int64_t off = int64_t((n + j) % P.nslot) * P.Nx;
    float tj, et, emt;
    level_time<DRV>(P, n + j, tj, et, emt);
    const PairF32 *row = tab + (j - 1) * P.Lp;
    if (P.zform && j == 1)
      pairs32<DRV, true, true>(dc, r32, off, row, q0, q1, ii, last, tj, et, emt, acc);
    else if (interior)
      pairs32<DRV, false, false, UNR>(dc, r32, off, row, q0, q1, ii, last, tj, et, emt, acc);
    else
      pairs32<DRV, true>(dc, r32, off, row, q0, q1, ii, last, tj, et, emt, acc);
    fold_group(s, acc.S.y, acc.C.y, acc.Fz, acc.Fy, acc.S.x, acc.C.x, acc.FyC);
  }
  int it = 0;
  float d = 0.f;
  if (active) d = finish_point32<DRV>(P, dc, r32.A, n, ii, s, prev_y, it);
  record_picard32(st, active, it, d, P.picard_tol_f);
}

template <int DRV>
__global__ void __launch_bounds__(kFlatTP, 8)
    k_step32f(const Params P, const DrvC<float> dc, Ring32 r32,
              const __grid_constant__ PairTab32 tab, int n, Stats *st) {
  wait_predecessor();
  step_tile32f<DRV, 2>(P, dc, r32, tab.e, n, blockIdx.x * kFlatTP, st);
}

// ---------------------------------------------------------------------------
// The FP32C general forward path: as k_step32, but a node's position is
// computed per point.  Node q of a pair sits at the offset
// o = A_j + B_j a_q cells from its grid point (node L-1-q at A_j - B_j a_q),
// A_j = a(x_i) j dt / dx and B_j = b(x_i) sqrt(2 j dt) / dx formed once per
// thread as float pairs from the plan's affine coefficients and x_i (itself
// a float pair; pair_affine, no FP64), a_q a float pair, so the offset is a
// float pair accurate to ~1e-9 cells (a plain float would lose 1e-3 cells at
// offsets of thousands of cells); its floor is the cell shift and the
// remainder theta.  The spline value, the pair arithmetic, the
// compensated sums and the Picard tail are those of k_step32, with the
// driver reading the node's position.
// ---------------------------------------------------------------------------
// c0 + c1 x for float pairs c0, c1, x, as a float pair to ~2^-44 relative:
// the exact product of the hi parts (FMA error term) and the exact sum of
// the large terms (TwoSum), the small cross terms in FP32.
__device__ __forceinline__ void pair_affine(float c0h, float c0l, float c1h, float c1l, float xh,
                                            float xl, float &h, float &l) {
  const float p = __fmul_rn(c1h, xh);
  const float pl = __fmaf_rn(c1h, xl, __fmaf_rn(c1l, xh, __fmaf_rn(c1h, xh, -p)));
  const float s = __fadd_rn(c0h, p);
  const float bp = __fsub_rn(s, c0h);
  const float err = __fadd_rn(__fsub_rn(c0h, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  h = s;
  l = __fadd_rn(err, __fadd_rn(c0l, pl));
}

// o = A + s B a (s = +1 or -1) as a float pair; the cell shift (floor) and
// theta in [0, 1)
__device__ __forceinline__ void gen_offset(float Ah, float Al, float Bh, float Bl, float ah,
                                           float al, float &fl, float &th, float &ol_out) {
  const float p = __fmul_rn(Bh, ah);
  const float pe = __fmaf_rn(Bh, ah, -p);                 // exact product error
  const float t = __fmaf_rn(Bh, al, __fmul_rn(Bl, ah));   // the small cross terms
  const float s = __fadd_rn(Ah, p);
  const float bp = __fsub_rn(s, Ah);
  const float err = __fadd_rn(__fsub_rn(Ah, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  const float ol = __fadd_rn(err, __fadd_rn(Al, __fadd_rn(pe, t)));
  fl = floorf(s);
  float r = __fadd_rn(__fsub_rn(s, fl), ol);  // s - fl is exact
  if (r < 0.f) {
    fl = __fsub_rn(fl, 1.f);
    r = __fadd_rn(r, 1.f);
  } else if (r >= 1.f) {
    fl = __fadd_rn(fl, 1.f);
    r = __fsub_rn(r, 1.f);
  }
  th = r;
  ol_out = __fadd_rn(s, ol);  // the offset, rounded (for the node's position)
}

template <int DRV>
__global__ void __launch_bounds__(kStepTP * kMaxGroups, 3)
    k_step32_gen(const Params P, const DrvC<float> dc, Ring32 r32,
                 const PairF32 *__restrict__ table, int n, Stats *st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int kP = P.k * P.Lp;
  PairF32 *tab = reinterpret_cast<PairF32 *>(smem_raw);
  float *part = reinterpret_cast<float *>(tab + kP);  // [kPartArrays][G][kStepTP]
  {
    const float4 *src = reinterpret_cast<const float4 *>(table);
    float4 *dst = reinterpret_cast<float4 *>(tab);
    for (int t = threadIdx.x; t < kP * kPairVec; t += blockDim.x) dst[t] = src[t];
  }
  __syncthreads();
  wait_predecessor();
  const int i0 = blockIdx.x * kStepTP;
  const int tp = threadIdx.x % kStepTP, g = threadIdx.x / kStepTP;
  const int G = P.G;
  const int last = int(P.Nx - 1);
  const int ii = i0 + tp;
  float prev_y = 0.f;
  if (threadIdx.x < kStepTP && i0 + int(threadIdx.x) <= last)
    prev_y = r32.A[int64_t((n + 1) % P.nslot) * P.Nx + i0 + threadIdx.x].x;
  if (g < G) {
    const Group32 w = group32(P, g, i0);
    Acc32 acc{make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f, 0.f, 0.f};
    if (ii <= last) {
      const int64_t off = int64_t((n + w.j) % P.nslot) * P.Nx;
      const float4 *A = r32.A + off;
      const float2 *M = r32.M + off;
      float tj, et, emt;
      level_time<DRV>(P, n + w.j, tj, et, emt);
      const PairF32 *row = tab + (w.j - 1) * P.Lp;
      // x_i = x_min + i dx as a float pair (i < 2^24 is exact in FP32)
      float xh, xl;
      pair_affine(P.xmin_f[0], P.xmin_f[1], P.dx_f[0], P.dx_f[1], float(ii), 0.f, xh, xl);
      const float *gf = P.gen_f[w.j - 1];
      float Ah, Al, Bh, Bl;
      pair_affine(gf[0], gf[1], gf[2], gf[3], xh, xl, Ah, Al);
      pair_affine(gf[4], gf[5], gf[6], gf[7], xh, xl, Bh, Bl);
      const float xf = __fadd_rn(xh, xl), dxf = P.dx_f[0];
      const float c6 = P.c6_f;
#pragma unroll 1
      for (int q = w.q0; q < w.q1; ++q) {
        const float4 *te = reinterpret_cast<const float4 *>(row + q);
        const float4 e0 = te[0], e3 = te[3], e4 = te[4];
        const float ah = P.gh_hi[q], al = P.gh_lo[q];
        float fla, tha, oa, flb, thb, ob;
        gen_offset(Ah, Al, Bh, Bl, ah, al, fla, tha, oa);
        gen_offset(Ah, Al, Bh, Bl, -ah, -al, flb, thb, ob);
        int ca = ii + int(fla), cb = ii + int(flb);
        float kaa = -tha * (1.f - tha) * c6, kab = -thb * (1.f - thb) * c6;
        // off the grid: the end value (theta = kappa = 0 on the end node)
        if (ca < 0 || ca >= last) {
          ca = ca < 0 ? 0 : last;
          tha = kaa = 0.f;
        }
        if (cb < 0 || cb >= last) {
          cb = cb < 0 ? 0 : last;
          thb = kab = 0.f;
        }
        const int ca1 = ca == last ? ca : ca + 1, cb1 = cb == last ? cb : cb + 1;
        float2 ha, da, hb, db;
        node_value(A[ca], A[ca1], M[ca], M[ca1], make_float2(tha, tha), make_float2(kaa, kaa),
                   ha, da);
        node_value(A[cb], A[cb1], M[cb], M[cb1], make_float2(thb, thb), make_float2(kab, kab),
                   hb, db);
        const float2 va = f2add(ha, da), vb = f2add(hb, db);
        const float Xa = __fmaf_rn(oa, dxf, xf), Xb = __fmaf_rn(ob, dxf, xf);
        const float Fa = driver_x<DRV>(dc, tj, et, emt, Xa, va.x, va.y);
        const float Fb = driver_x<DRV>(dc, tj, et, emt, Xb, vb.x, vb.y);
        acc.Fz = __fmaf_rn(e0.z, __fsub_rn(Fa, Fb), acc.Fz);
        two_sum_into(acc.Fy, acc.FyC, __fmul_rn(e0.w, __fadd_rn(Fa, Fb)));
        float2 hs, he;
        two_sum2(ha, hb, hs, he);
        comp_acc2(acc.S, acc.C, hi2(e3), lo2(e3), hi2(e4), hs, f2add(f2add(da, db), he));
        if (P.zform && w.j == 1) {
          // E[y DeltaW] z form: cyz (y^_a - y^_b) into the z lane
          float dh = ha.x, dl2 = 0.f;
          two_sum_into(dh, dl2, -hb.x);
          comp_acc1(acc.S.y, acc.C.y, e4.z, e4.w, dh, __fadd_rn(dl2, __fsub_rn(da.x, db.x)));
        }
      }
    }
    store_partials(part, G, g, tp, acc);
  }
  __syncthreads();
  finish_points32<DRV>(P, dc, r32.A, part, G, n, i0, st, prev_y);
}

// ---------------------------------------------------------------------------
// Measurement helper: every CTA streams its contiguous slice of `n` float4
// `reps` times with coalesced 16-byte loads through L2 (up to four in
// flight per thread) and adds a sum into sink[CTA] so no load is dropped.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_l2_read(const float4 *__restrict__ buf, size_t n,
                                                 int reps, float *sink) {
  const size_t per = n / gridDim.x;
  const float4 *p = buf + per * blockIdx.x;
  float acc = 0.f;
  for (int r = 0; r < reps; ++r) {
    size_t i = threadIdx.x;
    for (; i + 3 * 256 < per; i += 4 * 256) {
      const float4 a = __ldcg(p + i), b = __ldcg(p + i + 256), c = __ldcg(p + i + 512),
                   d = __ldcg(p + i + 768);
      acc += (a.x + b.y) + (c.z + d.w);
    }
    for (; i < per; i += 256) acc += __ldcg(p + i).x;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sink + blockIdx.x, acc);
}

// ---------------------------------------------------------------------------
// Measurement helper: the FMA pipe's rate.  Every thread runs kFmaChains
// independent chains a = a * m + c, kFmaUnroll steps each per iteration, and
// stores the chains' sum into sink (so none is dropped).  T = double (the
// FP64 pipe), float (scalar FP32) or float2 (packed fma.rn.f32x2, two FP32
// FMAs per instruction).
// ---------------------------------------------------------------------------
constexpr int kFmaChains = 8, kFmaUnroll = 16;
template <typename T>
struct FmaProbe;
template <>
struct FmaProbe<double> {
  static __device__ __forceinline__ double fma(double a, double m, double c) { return __fma_rn(a, m, c); }
  static __device__ __forceinline__ double val(float v) { return double(v); }
  static __device__ __forceinline__ double sum(double v) { return v; }
};
template <>
struct FmaProbe<float> {
  static __device__ __forceinline__ float fma(float a, float m, float c) { return __fmaf_rn(a, m, c); }
  static __device__ __forceinline__ float val(float v) { return v; }
  static __device__ __forceinline__ double sum(float v) { return double(v); }
};
template <>
struct FmaProbe<float2> {
  static __device__ __forceinline__ float2 fma(float2 a, float2 m, float2 c) { return f2fma(a, m, c); }
  static __device__ __forceinline__ float2 val(float v) { return make_float2(v, 0.5f * v); }
  static __device__ __forceinline__ double sum(float2 v) { return double(v.x) + double(v.y); }
};

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, double *sink) {
  using F = FmaProbe<T>;
  T a[kFmaChains];
#pragma unroll
  for (int q = 0; q < kFmaChains; ++q) a[q] = F::val(float(threadIdx.x + q) * 1e-3f);
  const T m = F::val(0.9999f), c = F::val(1e-4f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kFmaUnroll; ++u) {
#pragma unroll
      for (int q = 0; q < kFmaChains; ++q) a[q] = F::fma(a[q], m, c);
    }
  }
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < kFmaChains; ++q) acc += F::sum(a[q]);
  sink[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = acc;
}

// ---------------------------------------------------------------------------
// S4: readout of y^0, z^0 at x0 by the spline (Section 3.1 step 3).
// ---------------------------------------------------------------------------
template <int PREC>
__device__ void readout_values(const Params &P, Ring64 r64, Ring32 r32, int slot, double &ay,
                               double &az) {
  const int64_t off = int64_t(slot) * P.Nx;
  const double s = (P.x0 - P.x_min) / P.dx;
  int64_t c = (int64_t)floor(s);
  double v[2][2], M[2][2];  // [y|z][c|c+1]
  double th;
  if (s <= 0.0) {
    c = 0;
    th = 0.0;
  } else if (s >= double(P.Nx - 1)) {
    c = P.Nx - 2;
    th = 1.0;
  } else {
    if (c > P.Nx - 2) c = P.Nx - 2;
    th = s - double(c);
  }
  for (int q = 0; q < 2; ++q) {
    if constexpr (PREC == BSDE_FP64) {
      const double4_32a a = ldl(r64.ring + off + c + q);
      v[0][q] = a.x; M[0][q] = a.y; v[1][q] = a.z; M[1][q] = a.w;
    } else {
      const float4 a = ldl(r32.A + off + c + q);
      v[0][q] = double(a.x) + double(a.z);
      v[1][q] = double(a.y) + double(a.w);
    }
  }
  const double om = 1.0 - th, c6 = P.dx * P.dx / 6.0;
  if constexpr (PREC == BSDE_FP64) {
    ay = om * v[0][0] + th * v[0][1] +
         c6 * ((om * om * om - om) * M[0][0] + (th * th * th - th) * M[0][1]);
    az = om * v[1][0] + th * v[1][1] +
         c6 * ((om * om * om - om) * M[1][0] + (th * th * th - th) * M[1][1]);
  } else {
    // curvature part kappa (P + theta Q), P and Q formed in FP32 from the
    // nodes' second derivatives as the step kernels form them
    const float2 m0 = ldl(r32.M + off + c), m1 = ldl(r32.M + off + c + 1);
    const float Py = __fmaf_rn(2.f, m0.x, m1.x), Pz = __fmaf_rn(2.f, m0.y, m1.y);
    const float Qy = __fsub_rn(m1.x, m0.x), Qz = __fsub_rn(m1.y, m0.y);
    const double ka = -c6 * th * om;
    ay = om * v[0][0] + th * v[0][1] + ka * (double(Py) + th * double(Qy));
    az = om * v[1][0] + th * v[1][1] + ka * (double(Pz) + th * double(Qz));
  }
}

template <int PREC>
__global__ void k_readout(const Params P, Ring64 r64, Ring32 r32, int slot, Stats *st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double ay, az;
  readout_values<PREC>(P, r64, r32, slot, ay, az);
  st->y0 = ay;
  st->z0 = az;
}

}  // namespace bsde
