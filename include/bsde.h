/*
 * bsde.h -- C ABI of the GB300 (sm_103a) solver for the multistep BSDE scheme
 * of Kapllani & Teng, "Multistep schemes for solving backward stochastic
 * differential equations on GPU" (arXiv:1909.13560).
 *
 * What is solved (Section 2.2, Eq. 20-21; Section 3.1):
 *   the decoupled FBSDE  dX = a_x dt + b_x dW,  -dy = f(t, y, z) dt - z dW,
 *   y_T = g(X_T), on a uniform grid x_i = x_min + i*dx (i = 0..Nx-1),
 *   dx = (x_max - x_min)/(Nx-1), with N time steps dt = T/N.  With K_y = k
 *   steps for y, K_z = k_z steps for z and K = max(K_y, K_z) (Eq. 16), going
 *   backward from the K initial levels N, N-1, ..., N-K+1, every level
 *   n = N-K..0 is computed at every grid point from the K later levels:
 *     - Gauss-Hermite estimates (Eq. 21, L nodes) of E[z^], E[f], E[f dW],
 *       E[y^], E[y^ dW] over the off-grid points
 *       x_i + a_x j dt + b_x sqrt(2 j dt) a_l, j = 1..K, l = 1..L, where y^
 *       and z^ are natural cubic splines of the level values (Section 3.3),
 *       constant outside [x_min, x_max] (Section 3.2);
 *     - z^n explicitly from the second line of Eq. 20 (K_z steps);
 *     - y^n from the first line of Eq. 20 (K_y steps) by Picard iteration on
 *       the implicit term f(t_n, y^n, z^n) (Section 3.1 step 3).
 *   gamma coefficients: Tables 1 and 2 (K_y, K_z <= 6).
 *
 * Memory model: the caller owns every device buffer (one workspace per
 * plan, sized by bsde_workspace_bytes) and every stream.  A plan owns host
 * metadata, CUDA graphs and a small pinned host buffer only; bsde_free never
 * frees caller memory.  Pointers passed as "host" must stay valid until the
 * call returns (calls that take host pointers synchronise the stream).
 * Streams are passed as void* (a cudaStream_t; NULL = the legacy default
 * stream).
 *
 * Errors: every int-returning call returns BSDE_OK (0), a positive warning
 * or a negative error; bsde_strerror() describes a code and bsde_last_error()
 * gives the detail of the last failure on the calling thread.
 */
#ifndef BSDE_H
#define BSDE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BSDE_API __attribute__((visibility("default")))
#else
#define BSDE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* driver ids: f(t, y, z) */
enum {
  BSDE_DRIVER_LIN_SIN = 0, /* f = y/2 - z (1-D analogue of Example 4, Eq. 34)     */
  BSDE_DRIVER_BS = 1,      /* f = -(r y + (mu - r + delta) z / sigma)   (Eq. 29)     */
  BSDE_DRIVER_LB = 2,      /* f = -(r y + (mu - r) z / sigma)
                              + lb_sign (R - r) min(y - z/sigma, 0): borrowing rate */
  BSDE_DRIVER_EX1 = 3,     /* f = -y^3 + 5/2 y^2 - 3/2 y                (Eq. 22)     */
  BSDE_DRIVER_EX2 = 4,     /* f = (e^{t^2} - 4ty - 3e^{t^2 - y e^{-t^2}}
                              + z^2 e^{-t^2}) / 2                       (Eq. 24)     */
  BSDE_DRIVER_SHORT_RATE = 5 /* f = -x y: discounting at the short rate x, the
                              forward state where f is evaluated (the zero-coupon
                              bond; general forward path only)                     */
};

/* forward process: a(x) dt + b(x) dW, advanced from the grid point by one
 * Euler step over j dt (the general Markovian X of Section 1) */
enum {
  BSDE_FORWARD_CONST = 0, /* a = a_x, b = b_x (exact; the constant-shift kernels)  */
  BSDE_FORWARD_AFFINE = 1 /* a = a_x + a_1 x, b = b_x + b_1 x (the node
                             positions are computed per point; FP32C keeps
                             each node's offset as a float pair).  With an
                             x-dependent a or b only z_form = EYDW with k_z = 1
                             is consistent: Eq. 20's E[z^{n+1}] relies on the
                             identity E[y DeltaW] = dt E[z] of constant
                             coefficients, and its z misses the drift's slope   */
};

/* terminal ids: g and, for the closed-form start, the exact solution u(t, x)
 * with z = b(x) u_x */
enum {
  BSDE_TERMINAL_SIN = 0,      /* g = sin(x + T); u = sin(x + t)             (Eq. 35) */
  BSDE_TERMINAL_CALL_LOG = 1, /* g = (e^x - strike)^+, x = ln S; u = Black-Scholes
                                 call with dividend yield delta (Eq. 31; for LB
                                 the rate r - lb_sign (R - r), no dividend)          */
  BSDE_TERMINAL_LOGISTIC = 2, /* g = e^{x+T}/(e^{x+T}+1)                    (Eq. 23) */
  BSDE_TERMINAL_LNSIN = 3,    /* g = ln(sin x + 3) e^{T^2}                  (Eq. 25) */
  BSDE_TERMINAL_ONE = 4,      /* g = 1; u = the Vasicek bond price A e^{-B x} for
                                 SHORT_RATE with AFFINE a_1 < 0, b_1 = 0
                                 (kappa = -a_1, theta = a_x / kappa, sigma = b_x)   */
  BSDE_TERMINAL_CALL_PRICE = 5 /* g = (x - strike)^+ in the price x = S; u =
                                 Black-Scholes with volatility b_1 for AFFINE
                                 a_x = b_x = 0 (geometric Brownian motion)          */
};

/* arithmetic of the bulk (interpolation, driver at the nodes, quadrature) */
enum {
  BSDE_FP64 = 0,  /* everything in IEEE double                                     */
  BSDE_FP32C = 1  /* levels as float (hi, lo) pairs, FP32 interpolation and driver,
                     compensated (error-free product and sum) accumulation of the
                     y and z expectations, z^n and the explicit part of y^n as
                     normalized float pairs, Picard in FP32 on the increment
                     with an exact convergence test; spline second derivatives
                     from exact float differences of the pairs                   */
};

/* first term of the z line of Eq. 20 */
enum {
  BSDE_ZFORM_EZ = 0,   /* E[z^{n+1}], as Eq. 20 prints it                          */
  BSDE_ZFORM_EYDW = 1  /* E[y^{n+1} DeltaW_1] / dt, the term it replaces (Eq. 12
                          with l = 1).  Stable for K_z = 1 only, where it is the
                          second-order theta = 1/2 scheme: for K_z >= 2 the z
                          recurrence has a root of modulus > 1 and the solution
                          grows without bound as dt -> 0                          */
};

/* initial levels N-1, ..., N-K+1 (level N is always the terminal condition) */
enum {
  BSDE_INIT_EXACT = 0,   /* the closed form of the terminal id at t_{N-m}         */
  BSDE_INIT_ONESTEP = 1  /* the 1-step scheme (K_y = K_z = 1) run backward from
                            t_N with step dt / init_substeps on the same grid,
                            nodes and z form (Section 3.1 step 2)                */
};

/* FP32C step kernel of a single solve with a constant forward process.  Both
 * forms run the same node pairs in the same order of operations, so their
 * results are bitwise equal; they differ in how threads share a point. */
enum {
  BSDE_STEP_AUTO = 0,    /* flat when the grid alone fills the GPU's resident
                            threads twice, grouped otherwise                     */
  BSDE_STEP_GROUPED = 1, /* a CTA of 64 points x G groups of threads (j, pair
                            chunk), partial sums combined in shared memory       */
  BSDE_STEP_FLAT = 2     /* one thread per point runs all G groups in turn       */
};

/* return codes */
enum {
  BSDE_OK = 0,
  BSDE_WARN_NOCONV = 1, /* Picard stopped at picard_max somewhere; results written */
  BSDE_BUSY = 2,        /* server: no free slot or pool memory now; try again later */
  BSDE_EINVAL = -1,     /* bad problem: k or k_z outside 1..6, max(k, k_z) > N,
                           Nx < 4, L outside 1..64, x0 outside [x_min, x_max],
                           unknown id or mode, T <= 0, init_substeps < 1 or
                           N init_substeps > 2^30 with ONESTEP, or a terminal
                           whose closed form needs a forward process the
                           problem does not have (ONE, CALL_PRICE)              */
  BSDE_ENOSPC = -2,     /* workspace smaller than bsde_workspace_bytes()          */
  BSDE_ECUDA = -3,      /* a CUDA call failed (detail in bsde_last_error())       */
  BSDE_ENOMEM = -4,     /* host allocation failed                                 */
  BSDE_ETIMEOUT = -5    /* a bounded device-side wait expired (the server's idle
                           wait; single solves and batches have no device waits) */
};

/* Problem description (all fields read by bsde_plan; nothing is kept by
 * reference).  Initial levels: unless the caller passes them to bsde_solve,
 * level N is the terminal condition and levels N-1..N-K+1 come from
 * init_mode: the closed form of the terminal id at t_{N-m} (EXACT) or the
 * one-step start-up (ONESTEP, Section 3.1 step 2); when smoothing = 1 and
 * the terminal is CALL_LOG, level N holds the cell averages of the payoff and
 * of b_x times its derivative over [x_i - dx/2, x_i + dx/2] (Section 5,
 * Example 3).  Callers may instead pass their own K initial levels to
 * bsde_solve.  A zero-filled tail (k_z, z_form, init_mode, init_substeps all
 * 0) is the scheme of Eq. 20 with K_y = K_z = k and the closed-form start. */
typedef struct bsde_problem {
  int32_t driver, terminal, precision, smoothing;
  int32_t picard_max; /* Picard iteration cap (paper: 30)                     */
  int32_t N, k, L;    /* time steps, steps of the y line (K_y), GH nodes      */
  int64_t Nx;         /* grid points                                          */
  double T, x_min, x_max, x0; /* horizon, grid ends, readout point            */
  double a_x, b_x;    /* forward process dX = a_x dt + b_x dW                 */
  double r, mu, sigma, R, delta, lb_sign, strike; /* driver/payoff parameters */
  double picard_tol;  /* stop when |y^(p+1) - y^(p)| <= picard_tol            */
  int32_t k_z;        /* K_z, 1..6; 0: K_z = k                                 */
  int32_t z_form;     /* BSDE_ZFORM_*                                          */
  int32_t init_mode;  /* BSDE_INIT_*                                           */
  int32_t init_substeps; /* ONESTEP: 1-step scheme steps per dt, >= 1          */
  int32_t forward;    /* BSDE_FORWARD_*                                        */
  int32_t step_kernel; /* BSDE_STEP_*: the FP32C constant-shift step kernel    */
  double a_1, b_1;    /* AFFINE: slopes of a(x) and b(x)                       */
} bsde_problem;

typedef struct bsde_result {
  double y0, z0;           /* spline values of y^0, z^0 at x0 (Section 3.1 step 3) */
  double picard_resid_max; /* max over points and levels of the last |dy|          */
  int32_t status;          /* BSDE_OK or BSDE_WARN_NOCONV                          */
  int32_t picard_iters_max;
  int64_t levels_done;     /* N - K + 1, K = max(k, k_z) (start-up not counted)    */
} bsde_result;

typedef struct bsde_plan_s bsde_plan_t;

/* Device workspace a plan for *p needs, in bytes (ring of k+1 levels, the
 * spline scratch, node tables, output staging).  Used for admission by
 * footprint.  Returns BSDE_EINVAL for a bad problem. */
BSDE_API int bsde_workspace_bytes(const bsde_problem *p, size_t *bytes);

/* Validate *p, compute the plan constants on the host (Gauss-Hermite rule,
 * gamma tables, per-(j, l) cell shift and spline weights), copy the node
 * table into dev_workspace (device memory of at least bsde_workspace_bytes
 * bytes, 256-byte aligned, owned by the caller and reserved for this plan
 * until bsde_free) and return the plan in *out.  The plan records the
 * current CUDA device.  Solves on one plan must be ordered (one stream, or
 * synchronised streams): they share the workspace. */
BSDE_API int bsde_plan(const bsde_problem *p, void *dev_workspace, size_t bytes,
              bsde_plan_t **out);

/* Run the whole backward loop on `stream`.
 *   init_y, init_z: NULL (the start init_mode names) or K*Nx doubles each, row m
 *                   holding level N-m; host memory if init_on_host != 0,
 *                   device memory otherwise.
 *   out_y, out_z:   NULL or Nx doubles each, receiving level 0; host memory
 *                   if out_on_host != 0, device memory otherwise.
 *   result:         NULL or host struct receiving y0, z0 and the Picard
 *                   statistics; when non-NULL, or when any pointer is a host
 *                   pointer, the call waits for the stream.
 * Without host pointers and with result == NULL the call only enqueues work;
 * bsde_result_fetch() then reads the result.  Returns BSDE_OK,
 * BSDE_WARN_NOCONV (only when result is non-NULL) or an error. */
BSDE_API int bsde_solve(bsde_plan_t *plan, void *stream, const double *init_y,
               const double *init_z, int init_on_host, double *out_y,
               double *out_z, int out_on_host, bsde_result *result);

/* Copy the result of the last bsde_solve on this plan to the host, waiting
 * for `stream`. */
BSDE_API int bsde_result_fetch(bsde_plan_t *plan, void *stream, bsde_result *result);

/* Enqueue on `stream`, outside the captured graph, the kernels of backward
 * level n (0 <= n <= N-K): parts & 1 = the step kernel (Gauss-Hermite
 * expectations, z^n, Picard y^n), parts & 2 = the two spline sweeps of level
 * n.  The ring must hold levels n+1..n+K for meaningful values (after a
 * completed bsde_solve it does for n = 0, and re-running level 0 then
 * rewrites the same values); every index stays inside the workspace either
 * way.  Used to time the kernels one by one. */
BSDE_API int bsde_enqueue_level(bsde_plan_t *plan, void *stream, int n, int parts);

/* Level-by-level driving, for a grid decomposed over several plans (each
 * plan one slab of the grid with a halo; see the package's decomposition
 * driver).  A solve is then:
 *   bsde_enqueue_start(plan, stream, init_y, init_z, init_on_host);
 *   for n = N-K down to 0:
 *     bsde_enqueue_level(plan, stream, n, 1);   -- the step writes level n
 *     (replace the halo part of level n's value records)
 *     bsde_enqueue_level(plan, stream, n, 2);   -- the spline of level n
 *   bsde_enqueue_finish(plan, stream, out_y, out_z, out_on_host);
 *   bsde_result_fetch(plan, stream, &result);
 * bsde_enqueue_start: the stats reset, the start-up if any and the K initial
 *   levels with their splines; init_y/init_z as in bsde_solve (the call waits
 *   for the stream when they are host memory).
 * bsde_enqueue_finish: readout of level 0 at x0, its export (to out_y/out_z
 *   if given, host or device memory as out_on_host says; the call waits for
 *   host copies) and the statistics for bsde_result_fetch. */
BSDE_API int bsde_enqueue_start(bsde_plan_t *plan, void *stream, const double *init_y,
                                const double *init_z, int init_on_host);
BSDE_API int bsde_enqueue_finish(bsde_plan_t *plan, void *stream, double *out_y,
                                 double *out_z, int out_on_host);

/* Device address of level n's per-point value records in the plan's ring
 * (valid for the levels the ring holds at the time of use) and their size:
 * FP64 32-byte records (y, M_y, z, M_z) as doubles, FP32C 16-byte records
 * (y_hi, z_hi, y_lo, z_lo) as floats, value = hi + lo; record i belongs to
 * grid point i.  The spline part (M, in FP32C a separate array) is
 * recomputed by the spline launch, so a halo exchange copies these records
 * between the step and the spline launches of a level. */
BSDE_API int bsde_level_records(bsde_plan_t *plan, int n, void **records, size_t *record_bytes);

/* Release the plan's host resources and graphs (not the workspace). */
BSDE_API void bsde_free(bsde_plan_t *plan);

/* Number of kernel launches one bsde_solve without caller levels issues (for
 * launch accounting); with caller levels the start-up's launches, if any,
 * are left out. */
BSDE_API int64_t bsde_plan_launches(const bsde_plan_t *plan);

BSDE_API const char *bsde_strerror(int code);
BSDE_API const char *bsde_last_error(void);

/* Host-side plan constants, exposed for inspection and tests: the Gauss-
 * Hermite rule used by the kernels (nodes ascending, weights for exp(-a^2)),
 * and the gamma tables (Table 1 into gy[0..k], Table 2 into gz[0..k]). */
BSDE_API int bsde_gauss_hermite(int L, double *nodes, double *weights);
BSDE_API int bsde_gamma(int k, double *gy, double *gz);

/* Measurement helper (no counterpart in the paper): enqueue on `stream` one
 * launch that reads the `bytes` of device buffer `buf` `reps` times with
 * 16-byte loads from every SM (each CTA a contiguous slice, again and again)
 * and adds a float per CTA into `sink` (grid floats, device memory).
 * With a buffer that fits in L2 this times the L2 -> SM read bandwidth the
 * step kernels' level loads draw on.  `buf` 16-byte aligned, bytes a
 * multiple of 16 and at least 16 * grid * 256, grid <= 65535.  Returns
 * BSDE_EINVAL for bad arguments, BSDE_ECUDA if the launch fails. */
BSDE_API int bsde_l2_read_probe(const void *buf, size_t bytes, int reps, int grid, void *sink,
                                void *stream);

/* Measurement helper (no counterpart in the paper): enqueue on `stream` one
 * launch of `grid` CTAs of 256 threads in which every thread runs 8
 * independent fused multiply-add chains, 16 x `iters` steps each, and writes
 * one double into sink[grid * 256] (device memory).  kind 0: FP64 FMA;
 * 1: FP32 FMA; 2: packed FP32x2 FMA (two FP32 FMAs per instruction).  The
 * launch's flop count (2 per FMA) goes to *flops (may be NULL).  Timed with
 * CUDA events, this is the FMA pipe's rate that the step kernels' arithmetic
 * is measured against.  BSDE_EINVAL for bad arguments (kind outside 0..2,
 * iters < 1, grid outside 1..65535), BSDE_ECUDA if the launch fails. */
BSDE_API int bsde_fma_probe(int kind, int iters, int grid, void *sink, void *stream,
                            int64_t *flops);

/* ---- batched solves ------------------------------------------------------
 * Many independent problems (uneven Nx, N, k, driver, parameters; all
 * precision BSDE_FP32C, closed-form start) solved by one persistent launch:
 * a cluster of CTAs takes the next problem from a device queue (largest work
 * first) and shares its levels; the launch and its queue reset are one CUDA
 * graph.  Results are those of one bsde_solve per problem (same kernels per
 * tile, same order of operations), whatever the composition of the batch. */
typedef struct bsde_batch_s bsde_batch_t;

typedef struct bsde_batch_config {
  int32_t cluster;       /* CTAs that share one problem: 1, 2, 4 or 8            */
  int32_t target_groups; /* thread groups per grid point in the step tiles, 1..6 */
  int32_t flat_tiles;    /* step-tile form: 0 = grouped tiles of 64 points x the
                            groups (partial sums in shared memory, a barrier per
                            tile; CTAs of 384 threads, 2 per SM); 1 = flat
                            tiles of one point per thread (CTAs of 256 points, 3
                            per SM), each thread running its point's groups in
                            turn with no barrier                                 */
  int32_t reserved[5];
} bsde_batch_config;

/* Workspace for the n problems ps[0..n-1] (rings, tables, descriptors,
 * queue, per-problem statistics).  BSDE_EINVAL if any problem is invalid,
 * not BSDE_FP32C, asks for the one-step start-up or takes the general
 * forward path (AFFINE or SHORT_RATE): batches run the constant-shift
 * kernels from the closed form; K_z and the z form are free. */
BSDE_API int bsde_batch_workspace_bytes(int n, const bsde_problem *ps, size_t *bytes);

/* Plan the batch on dev_workspace (caller-owned, >= bsde_batch_workspace_bytes,
 * 256-byte aligned): host constants per problem, descriptors and tables copied
 * to the device.  The default configuration is cluster 2, 4 target groups,
 * grouped tiles. */
BSDE_API int bsde_plan_batch(int n, const bsde_problem *ps, void *dev_workspace,
                             size_t bytes, bsde_batch_t **out);

BSDE_API int bsde_batch_set_config(bsde_batch_t *b, const bsde_batch_config *cfg);
BSDE_API int bsde_batch_get_config(const bsde_batch_t *b, bsde_batch_config *cfg);

/* Time every candidate configuration (cluster in {1, 2, 4, 8} x step-tile
 * form in {grouped with 2, 4 or 6 target groups, flat}) on this batch with
 * CUDA events on `stream`, keep the fastest and return it in *best (may be
 * NULL).  Solves the batch 2 x 16 times; waits for the stream. */
BSDE_API int bsde_batch_autotune(bsde_batch_t *b, void *stream, bsde_batch_config *best);

/* Solve all problems; results (NULL or n host structs, in the order of ps)
 * receive y0, z0 and the Picard statistics of each.  Waits for the stream
 * when results is non-NULL. */
BSDE_API int bsde_solve_batch(bsde_batch_t *b, void *stream, bsde_result *results);

BSDE_API void bsde_batch_free(bsde_batch_t *b);

/* ---- continuous-batching server ---------------------------------------------
 * A persistent kernel solves pricing requests as they are submitted: each
 * request is admitted when a slot and enough of the device pool for its
 * level ring are free (admission by footprint), runs on the next free
 * cluster while others are in flight, and frees its slot and memory when
 * polled.  Problems must be BSDE_FP32C with the closed-form start and a
 * constant forward process (as for batches).  Requests run flat step tiles
 * (one point per thread; the same results as grouped tiles at the same group
 * split; step_kernel is not consulted).  A request gives the same result
 * alone and in any mix (same kernels per tile, same order of operations).  The server's waits for new requests are bounded: a
 * cluster that finds no request for idle_ms milliseconds stops the whole
 * server (every cluster leaves after its current request).  From then on
 * bsde_server_submit returns BSDE_ETIMEOUT, bsde_server_poll hands back the
 * requests no cluster will serve with status BSDE_ETIMEOUT and NaN values,
 * and bsde_server_stop returns BSDE_ETIMEOUT; after stop and a poll of every
 * request, bsde_server_start may launch it again. */
typedef struct bsde_server_s bsde_server_t;

/* Device bytes a request for *p occupies in the pool (its level ring). */
BSDE_API int bsde_request_bytes(const bsde_problem *p, size_t *bytes);

/* Workspace for a server with `slots` request slots (1..65536) and a pool
 * of pool_bytes for level rings. */
BSDE_API int bsde_server_workspace_bytes(int slots, size_t pool_bytes, size_t *bytes);

/* Bind a server to dev_workspace (caller-owned device memory); allocates its
 * host-mapped control block and slots (pinned). */
BSDE_API int bsde_server_create(void *dev_workspace, size_t bytes, int slots,
                                size_t pool_bytes, bsde_server_t **out);

/* Launch the persistent kernel on `stream` (clusters of `cluster` CTAs, as
 * many as fit on the GPU at once).  The kernel holds the stream until
 * bsde_server_stop; give it a stream of its own.  BSDE_EINVAL while a
 * request of an earlier run is still unpolled. */
BSDE_API int bsde_server_start(bsde_server_t *s, void *stream, int cluster, int idle_ms);

/* Admit a request: BSDE_OK with *slot set, BSDE_BUSY when no slot or pool
 * memory is free now, BSDE_EINVAL for a bad problem (as for batches: FP32C,
 * closed-form start), BSDE_ETIMEOUT once the
 * server has stopped itself.  Non-blocking. */
BSDE_API int bsde_server_submit(bsde_server_t *s, const bsde_problem *p, int *slot);

/* Collect up to max finished requests: their slots and results; frees their
 * slots and pool memory.  Returns the number collected (>= 0) or an error. */
BSDE_API int bsde_server_poll(bsde_server_t *s, int max, int *slots, bsde_result *results);

/* Ask the kernel to finish (requests already published are still solved)
 * and wait for it.  BSDE_ETIMEOUT if a cluster gave up waiting. */
BSDE_API int bsde_server_stop(bsde_server_t *s);

BSDE_API void bsde_server_free(bsde_server_t *s);

/* Solve without allocating anything (no counterpart in the paper; this is a
 * service for callers of this library).
 *
 * Some callers must not allocate device or pinned memory at solve time: a
 * host application that owns the whole device through its own allocator and
 * forbids others from calling cudaMalloc, a latency-critical pricing loop
 * where an allocation would synchronise the device in the middle of a
 * trading cycle, or a plug-in loaded into a process whose memory budget is
 * fixed.  This entry point serves them.  It runs the same kernels as
 * bsde_solve, with the workspace in a fixed array that the library reserves
 * in device memory (BSDE_NOALLOC_MAX_BYTES per GPU, held by every GPU that
 * loads the library until the process exits).  It launches the kernels one
 * by one and calls no cudaMalloc, cudaMallocHost, cudaFree or any other
 * allocating routine.  The plan constants and node tables (about 130 KB)
 * live in a file-scope host buffer, not on the caller's stack; a library
 * mutex guards it, so calls from several host threads run one at a time.
 *
 * Arguments are those of bsde_plan and bsde_solve (the caller still passes
 * the initial levels, if any, and the output buffers).  The call waits for
 * `stream` before returning.  A problem whose workspace
 * (bsde_workspace_bytes) exceeds BSDE_NOALLOC_MAX_BYTES is rejected with
 * BSDE_ENOSPC and a message naming both sizes.
 *
 * The first call on each device looks up that device's copy of the array
 * (cudaGetSymbolAddress, with the device current) and caches the address;
 * make that first call before any stream capture on the device.  The cached
 * address belongs to the device's primary context: after cudaDeviceReset (or
 * any reset of that context) this entry point must not be called again in
 * the same process.  All calls
 * on a device share the one array, which keeps the contents of the last
 * call; every call rewrites what it reads before reading it.  Calls whose GPU
 * work overlaps (different streams, or different host threads, on the same
 * device) race on the array: order them. */
#define BSDE_NOALLOC_MAX_BYTES ((size_t)32 << 20)
BSDE_API int bsde_solve_noalloc(const bsde_problem *p, void *stream,
                                const double *init_y, const double *init_z,
                                int init_on_host, double *out_y, double *out_z,
                                int out_on_host, bsde_result *result);

#ifdef __cplusplus
}
#endif
#endif /* BSDE_H */
