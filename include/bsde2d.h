/*
 * bsde2d.h -- C ABI of the two-dimensional solver (GB300, sm_103a) for the
 * multistep BSDE scheme of Kapllani & Teng (arXiv:1909.13560), d = 2.
 *
 * What is solved (Eq. 20-21 with d = 2; Section 3.3; Examples 4 and 5):
 *   the decoupled FBSDE  dX = a dt + B dW (X, a in R^2, B = [[b11, 0],
 *   [b21, b22]] constant), -dy = f(y, z) dt - z dW with the row vector
 *   z = (z1, z2) and the linear driver f = alpha y + beta1 z1 + beta2 z2,
 *   y_T = g(X_T), on the uniform grid x = (x1_min + i1 dx1, x2_min + i2 dx2),
 *   i1 < Nx1, i2 < Nx2, with N time steps dt = T/N and K_y = K_z = k.
 *   Every level n = N-k..0 is computed at every grid point from the k later
 *   levels:
 *     - Gauss-Hermite tensor estimates (Eq. 21, L nodes per dimension, L^2 in
 *       all) of E[z^], E[f], E[f DeltaW^T], E[y^] over the off-grid points
 *       x + a j dt + B sqrt(2 j dt) (a_l1, a_l2), j = 1..k, where y^, z^ are
 *       bicubic Hermite interpolants of the level values whose first and
 *       mixed derivatives come from fourth-order finite differences (central;
 *       forward at the first two and backward at the last two nodes of a
 *       line); a point off the box takes the value at its projection onto it
 *       (Section 3.2);
 *     - z^n explicitly from the second line of Eq. 20, per component;
 *     - y^n from the first line by Picard iteration on f(y^n, z^n).
 *   Initial levels N..N-k+1: the closed form of the terminal id (or the
 *   caller's levels).
 *
 * Memory model, streams and errors: as in bsde.h (caller-owned workspace of
 * bsde2_workspace_bytes, 256-byte aligned; BSDE_* return codes; detail in
 * bsde_last_error()).
 */
#ifndef BSDE2D_H
#define BSDE2D_H

#include "bsde.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BSDE2_DRIVER_LINEAR = 0 /* f = alpha y + beta1 z1 + beta2 z2 (Examples 4 and 5)   */
};

enum {
  BSDE2_TERMINAL_SIN_SUM = 0,   /* g = sin(x1 + x2 + T); u = sin(x1 + x2 + t)
                                   (Eq. 35; the exact solution for X = W and
                                   f = y - (z1 + z2)/2, Example 4)                   */
  BSDE2_TERMINAL_SPREAD_LOG = 1 /* g = (e^{x1} - e^{x2})^+ in log prices; u by
                                   Margrabe's formula (Eq. 37) with sigma1 = b11,
                                   sigma2 = |(b21, b22)|, rho sigma1 sigma2 =
                                   b11 b21 (Example 5)                               */
};

/* Form of the step kernels (bsde2_problem.step_form). */
enum {
  BSDE2_STEP_AUTO = 0,     /* TENSOR when b21 == 0, NODEWISE otherwise              */
  BSDE2_STEP_NODEWISE = 1, /* one kernel over the L^2 tensor nodes of every step j:
                              per node the bicubic values of the three fields      */
  BSDE2_STEP_TENSOR = 2    /* two kernels per level (b21 == 0 only, else
                              BSDE_EINVAL): the node shifts and the quadrature
                              weights then factor per dimension, and the L^2-node
                              sums are taken as an x2 pass of L nodes into a
                              per-step buffer, then an x1 pass of L nodes.  Same
                              values as NODEWISE up to rounding order             */
};

typedef struct bsde2_problem {
  int32_t driver, terminal;
  int32_t precision;  /* BSDE_FP64, or BSDE_FP32C: level values as float pairs,
                         derivatives as floats, the bicubic increment over the
                         cell's corner value in FP32, compensated sums, Picard
                         on the increment in FP32 (derivatives: the finite
                         differences in FP32 over the float pairs' increments) */
  int32_t picard_max; /* Picard iteration cap (paper: 30)                         */
  int32_t N, k, L;    /* time steps, steps of the scheme (1..min(6, N)), GH nodes
                         per dimension (1..16)                                    */
  int32_t step_form;  /* BSDE2_STEP_* (0: AUTO)                                  */
  int64_t Nx1, Nx2;   /* grid points per dimension, >= 6 each (the one-sided
                         stencil at the second node reaches five nodes on)      */
  double T, x1_min, x1_max, x2_min, x2_max, x01, x02; /* horizon, box, readout */
  double a1, a2, b11, b21, b22; /* forward process                                */
  double alpha, beta1, beta2;   /* linear driver                                  */
  double picard_tol;  /* stop when |y^(p+1) - y^(p)| <= picard_tol                */
} bsde2_problem;

typedef struct bsde2_result {
  double y0, z0[2];        /* interpolated y^0, z^0 at (x01, x02)                 */
  double picard_resid_max; /* max over points and levels of the last |dy|         */
  int32_t status;          /* BSDE_OK or BSDE_WARN_NOCONV                         */
  int32_t picard_iters_max;
  int64_t levels_done;     /* N - k + 1                                           */
} bsde2_result;

typedef struct bsde2_plan_s bsde2_plan_t;

/* Device workspace a plan for *p needs, in bytes: a ring of k + 1 levels of
 * 3 fields x (value, dx1 d/dx1, dx2 d/dx2, dx1 dx2 d2/dx1dx2) doubles per
 * grid point (96 B), one plane of new values (24 B per point), the node
 * table, a staging area of 3 k planes and the statistics; the TENSOR form
 * adds the x2 pass's buffer of k records per point (96 B FP64, 64 B FP32C).
 * BSDE_EINVAL for a bad problem (k outside 1..min(6, N), Nx1 or Nx2 < 6, L
 * outside 1..16, x0 outside the box, unknown id, precision or step form,
 * TENSOR with b21 != 0, T <= 0).  FP32C keeps one 64-byte record per point
 * and level instead of 96 bytes. */
BSDE_API int bsde2_workspace_bytes(const bsde2_problem *p, size_t *bytes);

/* Validate *p, build the node table on the host (per (j, l1, l2): the cell
 * shift and the Hermite basis values of the position inside the cell in each
 * dimension, the quadrature and multistep weights) and copy it into
 * dev_workspace (device memory of at least bsde2_workspace_bytes bytes,
 * 256-byte aligned, owned by the caller and reserved for this plan until
 * bsde2_free).  The plan records the current CUDA device. */
BSDE_API int bsde2_plan(const bsde2_problem *p, void *dev_workspace, size_t bytes,
                        bsde2_plan_t **out);

/* Run the whole backward loop on `stream` (one CUDA graph).
 *   init_y, init_z1, init_z2: NULL (closed-form start) or k Nx2 Nx1 doubles
 *                   each (row m = level N - m, i1 fastest); host memory if
 *                   init_on_host != 0, device memory otherwise.
 *   out_y, out_z1, out_z2: NULL or Nx2 Nx1 doubles each, receiving level 0;
 *                   host memory if out_on_host != 0, device memory otherwise.
 *   result:         NULL or host struct; when non-NULL, or when any pointer is
 *                   a host pointer, the call waits for the stream.
 * Returns BSDE_OK, BSDE_WARN_NOCONV (only when result is non-NULL) or an
 * error. */
BSDE_API int bsde2_solve(bsde2_plan_t *plan, void *stream, const double *init_y,
                         const double *init_z1, const double *init_z2, int init_on_host,
                         double *out_y, double *out_z1, double *out_z2, int out_on_host,
                         bsde2_result *result);

/* The result of the last bsde2_solve on this plan, waiting for `stream`. */
BSDE_API int bsde2_result_fetch(bsde2_plan_t *plan, void *stream, bsde2_result *result);

/* Enqueue the kernels of backward level n (0 <= n <= N-k) outside the graph:
 * parts & 1 = the step kernel (the TENSOR form: both passes), parts & 4 = the
 * x2 pass alone, parts & 8 = the x1 pass alone (TENSOR only; the x1 pass
 * reads the buffer the x2 pass of the same level wrote), parts & 2 = the
 * derivative kernel.  Used to time the kernels one by one (meaningful after
 * a completed solve). */
BSDE_API int bsde2_enqueue_level(bsde2_plan_t *plan, void *stream, int n, int parts);

/* Kernel launches in one bsde2_solve: 1 + 2 k + (2 or 3 with TENSOR)
 * (N - k + 1) + 2. */
BSDE_API int64_t bsde2_plan_launches(const bsde2_plan_t *plan);

/* Release the plan's host resources and graphs (not the workspace). */
BSDE_API void bsde2_free(bsde2_plan_t *plan);

#ifdef __cplusplus
}
#endif

#endif /* BSDE2D_H */
