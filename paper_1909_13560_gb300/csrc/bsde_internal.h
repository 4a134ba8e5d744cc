// Internal definitions shared by the host planning code (bsde_host.cpp) and
// the CUDA kernels (bsde_cuda.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/bsde.h"

namespace bsde {

constexpr int kMaxK = 6;
constexpr int kMaxL = 64;
constexpr int kInvPivots = 64;   // exact 1/d_m of the spline LU for m < 64
constexpr int kStepTP = 64;      // grid points per CTA in the step kernels
constexpr int kMaxGroups = 6;    // (j, l-chunk) groups per point
constexpr int kPartArrays = 7;   // FP32C per-group partial sums: z (S, C, F), y (S, C, F, F err)
constexpr int kSplineTile = 512;  // unknowns per CTA in the FP64 spline kernel
constexpr int kSplineChunk = 4;   // unknowns per thread (serial recurrence, FP64)
constexpr int kSplineHead = 16;   // FP32C: pivots of the spline LU are constant beyond this

// Per (j, l) entry of the node tables.  The off-grid point
// x_i + a_x j dt + b_x sqrt(2 j dt) a_l sits in cell i + shift at relative
// position theta; w0..w3 are the spline weights of v_c, v_{c+1}, M_c, M_{c+1}.
// The expectations of Eq. 20 are folded into per-node coefficients, so that
// a thread keeps two sums per point (j = 1..K, K = max(K_y, K_z)):
//   z^n = sum_jl cz_jl z^_jl + sum_jl cfz_jl F_jl [+ sum_l cyz_l y^_1l]
//   A   = sum_l  cy_l  y^_{K_y}l + sum_jl cfy_jl F_jl  (y^n = A + K_y dt gy_0 f(t_n, y^n, z^n))
// with wt = omega_l / sqrt(pi) (Eq. 21), DeltaW_jl = sqrt(2 j dt) a_l,
// gy from Table 1 row K_y and gz from Table 2 row K_z (zero beyond them),
// cz = wt (delta_{j1} - gz_j) / gz_0, cfz = gz_j wt DeltaW_jl / gz_0,
// cy = wt (j = K_y only), cfy = K_y dt gy_j wt.  In the E[y DeltaW] z form
// the delta_{j1} term moves from z^ to y^: cz = -wt gz_j / gz_0 and
// cyz = wt DeltaW_1l / (dt gz_0) at j = 1 (zero otherwise).
struct NodeF64 {
  int32_t shift, pad;
  double w0, w1, w2, w3, cz, cfz, cfy, cy, cyz;
  double dW;  // DeltaW_jl (the general forward path places its nodes per point)
};

// FP32C entry: the same coefficients, with cz and cy split into float
// hi + lo parts for the compensated sums.
struct NodeF32 {
  int32_t shift;
  float w0, w1, w2, w3;
  float czh, czl, cfz, cfy, cyh, cyl, cyzh, cyzl;
};

// FP32C pair entry: Gauss-Hermite nodes l and L-1-l (a_{L-1-l} = -a_l) share
// |DeltaW| and the weight, so cz, cy and cfy are equal for the pair and cfz
// is opposite.  A pair is processed together: the two spline values are
// added exactly (TwoSum) before one compensated product, and the driver
// terms enter as cfz (F_a - F_b) and cfy (F_a + F_b).  For odd L the middle
// node (a = 0, DeltaW = 0) is a pair with itself and halved coefficients.
// The arithmetic runs on (y, z) lane pairs (packed FP32x2), so every weight
// is stored twice, once per lane, and the compensated-sum coefficients are
// lane pairs (cy, cz): hi parts, and negated hi and lo parts, which let the
// error terms be formed by fused multiply-adds alone.  Five float4:
// (shift_a, shift_b, cfz, cfy), (th_a, th_a, ka_a, ka_a),
// (th_b, th_b, ka_b, ka_b), (cyh, czh, -cyh, -czh), (-cyl, -czl, cyzh, cyzl);
// th = theta, ka = -theta (1 - theta) dx^2 / 6 (the spline value is
// v_c + theta d + ka (P + theta Q), see Ring32).  cy is zero for
// j != K_y.  cyz (hi, lo) is node a's weight of y^ in the z sum (E[y DeltaW]
// z form, j = 1; node b's is -cyz): the pair adds cyz (y^_a - y^_b).
struct PairF32 {
  int32_t shift_a, shift_b;
  float cfz, cfy;
  float tha[2], kaa[2], thb[2], kab[2];
  float ch[2], nch[2], ncl[2], cyz[2];
};
constexpr int kPairVec = int(sizeof(PairF32) / 16);  // float4 per entry

// K_z of a problem (0 in the struct means K_z = k) and K = max(K_y, K_z),
// the number of later levels one backward step reads (Eq. 16).
inline int problem_kz(const bsde_problem &p) { return p.k_z > 0 ? p.k_z : p.k; }
inline int problem_K(const bsde_problem &p) {
  return p.k > problem_kz(p) ? p.k : problem_kz(p);
}
// The general forward path: node positions per point (affine a, b) or a
// driver that reads the forward state.
inline bool problem_general(const bsde_problem &p) {
  return p.forward == BSDE_FORWARD_AFFINE || p.driver == BSDE_DRIVER_SHORT_RATE;
}

// Everything a kernel needs to know about one problem.  k is K (levels per
// step, ring of k + 1 slots); ky, kz the steps of the y and z lines.
struct Params {
  int64_t Nx;
  int32_t N, k, L, driver, terminal, precision, smoothing, picard_max, nslot;
  int32_t ky, kz, zform, general;  // general: per-point node positions (AFFINE
                                   // forward or an x-dependent driver)
  double a_1, b_1;                 // AFFINE slopes of a(x), b(x)
  double T, dt, dx, x_min, x_max, x0, a_x, b_x;
  double r, mu, sigma, R, delta, lb_sign, strike;
  double picard_tol;
  float picard_tol_f;  // the largest float <= picard_tol (FP32 Picard test)
  float hg0_f;         // float(hg0), the FP32 Picard weight
  double gy[kMaxK + 1], gz[kMaxK + 1];
  double h;       // K_y dt
  double hg0;     // K_y dt gy_0 (weight of the implicit term)
  double inv_gz0; // 1 / gz_0
  double inv_dx2_6; // 6 / dx^2
  double inv_dx;    // 1 / dx (the general path's cell position: a multiply, not
                    // a divide; it may move a node that lands within rounding
                    // of a grid node to the neighbouring cell, where the spline
                    // has the same value to rounding)
  double c6;        // dx^2 / 6 (the spline's curvature weight scale)
  float c6_f;       // float(c6)
  // general forward path: per step j the node offset in cells,
  // o = A_j(x) + B_j(x) a_l, as affine functions of the point's x:
  // A_j = a0 + a1 x = a(x) j dt / dx, B_j = b0 + b1 x = b(x) sqrt(2 j dt) / dx,
  // formed once on the host; the FP32C kernel takes them as float pairs
  // gen_f[j - 1] = (a0, a1, b0, b1) x (hi, lo) and the point's x from the
  // float pairs xmin_f, dx_f, so it forms its offsets without FP64
  float gen_f[kMaxK][8];
  float xmin_f[2], dx_f[2];
  double invd[kInvPivots];
  // work split of the step kernels: S l-chunks of Lg nodes per j, G = k S
  // groups per point; shift range per j (for the clamp-free fast path)
  int32_t S, Lg, G, Lp;  // Lp = ceil(L/2) pairs; in FP32C the chunks hold Lg pairs
  int32_t wide_spline;   // FP32C: the spline's wide tiles (grids that fill the GPU
                         // twice over, whatever step kernel was asked for)
  int32_t flat;          // FP32C constant-shift step: one thread runs all G groups of
                         // its point (k_step32f), for grids of at least two waves
  int32_t smin[kMaxK], smax[kMaxK];
  // the Gauss-Hermite node of pair q (node q; node L-1-q is its negative) as
  // a float pair hi + lo, for the FP32C general path's per-point positions
  float gh_hi[kMaxL / 2], gh_lo[kMaxL / 2];
};

// Device workspace layout (byte offsets from the workspace base).
struct Layout {
  size_t ring64;   // FP64: double4 (y, M_y, z, M_z) x nslot x Nx
  size_t ringA;    // FP32C: float4 (y_hi, z_hi, y_lo, z_lo) x nslot x Nx
  size_t ringB;    // FP32C: float2 (M_y, M_z) x nslot x Nx
  size_t table;    // node table (K L entries)
  size_t ptable;   // FP32C pair table (K ceil(L/2) entries)
  size_t stage;    // 2 x K x Nx doubles: imported initial levels / exported level 0
  // one-step start-up (init_mode ONESTEP, K > 1): a ring of two slots and the
  // node tables of the 1-step scheme; unused otherwise
  size_t sub_ring64, sub_ringA, sub_ringB, sub_table, sub_ptable;
  size_t stats;    // Stats
  size_t total;
};

struct Stats {
  double y0, z0;
  unsigned long long resid_bits; // max |dy| as the bits of a non-negative double
  int32_t iters_max;
  int32_t nonconv;
  int32_t timeout;  // a bounded device-side wait gave up
  int32_t pad;
};

// Host-side planning (bsde_host.cpp).
int validate(const bsde_problem &p);
int fill_params(const bsde_problem &p, Params &P);
// Whether a solve of p without caller levels runs the one-step start-up, and
// the Params of that start-up: K_y = K_z = 1, N S steps of dt / S on the same
// grid and nodes (Section 3.1 step 2).
bool has_startup(const bsde_problem &p);
Params startup_params(const Params &P, int substeps);
Layout layout_for(const bsde_problem &p);
int gauss_hermite(int L, double *nodes, double *weights);
int gamma_tables(int k, double *gy, double *gz);
void build_tables(Params &P, NodeF64 *t64, NodeF32 *t32, PairF32 *tp = nullptr,
                  int target_groups = 4, int max_groups = kMaxGroups,
                  long resident_threads = 0);

}  // namespace bsde
