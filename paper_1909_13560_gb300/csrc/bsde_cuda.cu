// C ABI of the multistep BSDE solver: plans, CUDA-graph capture of the whole
// backward loop, solve and result transfer.  Kernels: bsde_kernels.cuh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "bsde_internal.h"
#include "bsde_kernels.cuh"
#include "bsde_batch.cuh"
#include "bsde_server.cuh"

namespace bsde {

static thread_local std::string g_last_error;

static int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

#define BSDE_CUDA_TRY(expr)                                                              \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return fail(BSDE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));       \
  } while (0)

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = dev;  // then nothing to restore
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
  }
  ~DeviceGuard() {
    if (prev_ != dev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = 0, dev_ = 0;
};

}  // namespace bsde

using namespace bsde;

namespace bsde {
// One backward run on the workspace: its constants, level ring and node
// tables.  A plan has the main run and, for the one-step start-up, the run of
// the 1-step scheme.
struct Run {
  Params P;
  Ring64 r64;
  Ring32 r32;
  const NodeF64 *t64;
  const PairF32 *tp;   // FP32C pair table in the workspace
  PairTab32 tab;       // the same table, passed to k_step32 by value
};
}  // namespace bsde

struct bsde_plan_s {
  bsde_problem prob;
  Params P;
  Layout lay;
  bsde::Run run, sub;  // main loop; start-up (valid when has_startup(prob))
  int device;
  unsigned char *ws;
  size_t ws_bytes;
  DrvC<double> dc64;
  DrvC<float> dc32;
  cudaGraphExec_t graph[2];  // [closed-form start, imported start]
  int64_t launches[2];
  Stats *host_stats;         // pinned
};

namespace bsde {

// Threads of the step kernels the GPU holds at once (36 warps per SM at the
// kernels' register use), or 0 if the device cannot be queried.
static long resident_step_threads(int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  return long(sms) * 36 * 32;
}

static void driver_coefs(const Params &P, DrvC<double> &c64, DrvC<float> &c32) {
  c64 = DrvC<double>{0.0, 0.0, 0.0, 0.0};
  if (P.driver == BSDE_DRIVER_BS) {
    c64.ca = P.r;
    c64.cb = (P.mu - P.r + P.delta) / P.sigma;
  } else if (P.driver == BSDE_DRIVER_LB) {
    c64.ca = P.r;
    c64.cb = (P.mu - P.r) / P.sigma;
    c64.cc = P.lb_sign * (P.R - P.r);
    c64.cis = 1.0 / P.sigma;
  }
  c32 = DrvC<float>{float(c64.ca), float(c64.cb), float(c64.cc), float(c64.cis)};
}

// Launch with programmatic stream serialization: the kernel may begin (and
// stage what it owns) while its predecessor on the stream finishes; it waits
// (griddepcontrol.wait) before reading anything the predecessor wrote.
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t lc{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.gridDim = dim3(grid, 1, 1);
  lc.blockDim = dim3(block, 1, 1);
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaLaunchKernelEx(&lc, kernel, std::forward<Args>(args)...);
}

template <int PREC, int DRV>
static void launch_step(bsde_plan_t *pl, const Run &R, cudaStream_t s, int n) {
  const Params &P = R.P;
  const unsigned threads = unsigned(kStepTP * P.G);
  const unsigned blocks = unsigned((P.Nx + kStepTP - 1) / kStepTP);
  const int kL = P.k * P.L;
  Stats *st = reinterpret_cast<Stats *>(pl->ws + pl->lay.stats);
  if (PREC == BSDE_FP64) {
    const size_t sm = sizeof(NodeF64) * kL + sizeof(double) * 2 * P.G * kStepTP;
    if (P.general)
      launch_pdl(k_step64_gen<DRV>, blocks, threads, sm, s, P, pl->dc64, R.r64.ring, R.t64, n,
                 st);
    else if constexpr (DRV != BSDE_DRIVER_SHORT_RATE)
      launch_pdl(k_step64<DRV>, blocks, threads, sm, s, P, pl->dc64, R.r64.ring, R.t64, n, st);
  } else {
    if (P.general)
      launch_pdl(k_step32_gen<DRV>, blocks, threads, step32_smem(P.G, P.k * P.Lp), s, P,
                 pl->dc32, R.r32, R.tp, n, st);
    else if constexpr (DRV != BSDE_DRIVER_SHORT_RATE) {
      if (P.flat)
        launch_pdl(k_step32f<DRV>, unsigned((P.Nx + kFlatTP - 1) / kFlatTP), unsigned(kFlatTP),
                   0, s, P, pl->dc32, R.r32, R.tab, n, st);
      else
        launch_pdl(k_step32<DRV>, blocks, threads, step32_smem(P.G, 0), s, P, pl->dc32, R.r32,
                   R.tab, n, st);
    }
  }
}

template <int PREC>
static void launch_step_any(bsde_plan_t *pl, const Run &R, cudaStream_t s, int n) {
  switch (R.P.driver) {
    case BSDE_DRIVER_LIN_SIN: launch_step<PREC, BSDE_DRIVER_LIN_SIN>(pl, R, s, n); break;
    case BSDE_DRIVER_BS: launch_step<PREC, BSDE_DRIVER_BS>(pl, R, s, n); break;
    case BSDE_DRIVER_LB: launch_step<PREC, BSDE_DRIVER_LB>(pl, R, s, n); break;
    case BSDE_DRIVER_EX1: launch_step<PREC, BSDE_DRIVER_EX1>(pl, R, s, n); break;
    case BSDE_DRIVER_SHORT_RATE: launch_step<PREC, BSDE_DRIVER_SHORT_RATE>(pl, R, s, n); break;
    default: launch_step<PREC, BSDE_DRIVER_EX2>(pl, R, s, n); break;
  }
}

template <int PREC>
static void launch_spline(const Run &R, cudaStream_t s, int slot) {
  const Params &P = R.P;
  constexpr int TS = SplineLaunch<PREC>::TS;
  const unsigned blocks = unsigned((P.Nx - 2 + TS - 1) / TS);
  launch_pdl(k_spline<PREC>, blocks, unsigned(SplineLaunch<PREC>::NT), 0, s, P, R.r64, R.r32,
             slot);
}

// The spline of a single solve.  FP32C: on grids that fill the GPU twice
// over the wide tiles (fewer CTAs, which leave room to other solves' work
// running beside them), else the warp-tiled kernel (CTA 0 the first tile,
// then 104 unknowns per warp, 4 warps per CTA); both give the same M
// bitwise.  FP64: the tiled kernel.
template <int PREC>
static int64_t enqueue_spline(const Run &R, cudaStream_t s, int slot) {
  if constexpr (PREC == BSDE_FP32C) {
    if (R.P.wide_spline) {
      launch_spline<PREC>(R, s, slot);
      return 1;
    }
    const int64_t nw = spline_warp_tiles(R.P.Nx);
    const int per = kSplWarpThreads / 32;
    launch_pdl(k_spline32w, unsigned(1 + (nw + per - 1) / per), unsigned(kSplWarpThreads), 0, s,
               R.P, R.r32, slot);
  } else {
    launch_spline<PREC>(R, s, slot);
  }
  return 1;
}

// Views of the workspace for the main run and the start-up run (their
// Params as upload_tables left them).
static void bind_runs(bsde_plan_t *pl) {
  unsigned char *ws = pl->ws;
  const Layout &L = pl->lay;
  Run &R = pl->run;
  R.P = pl->P;
  R.r64 = Ring64{reinterpret_cast<double4_32a *>(ws + L.ring64)};
  R.r32 = ring32(ws + L.ringA, ws + L.ringB, R.P);
  R.t64 = reinterpret_cast<const NodeF64 *>(ws + L.table);
  R.tp = reinterpret_cast<const PairF32 *>(ws + L.ptable);
  Run &Q = pl->sub;
  if (has_startup(pl->prob)) {
    Q.r64 = Ring64{reinterpret_cast<double4_32a *>(ws + L.sub_ring64)};
    Q.r32 = ring32(ws + L.sub_ringA, ws + L.sub_ringB, Q.P);
    Q.t64 = reinterpret_cast<const NodeF64 *>(ws + L.sub_table);
    Q.tp = reinterpret_cast<const PairF32 *>(ws + L.sub_ptable);
  }
}

// Node tables of the plan's runs, built on the host (the work split needs the
// device's resident thread count) into host_buf and copied to the workspace
// on `s`; the caller keeps host_buf alive until the copies are done.
struct HostTables {
  NodeF64 t64[kMaxK * kMaxL], s64[kMaxL];
  NodeF32 t32[kMaxK * kMaxL], s32[kMaxL];
  PairF32 tp[kMaxK * kMaxL], sp[kMaxL];
};
static int upload_tables(bsde_plan_t *pl, HostTables &h, cudaStream_t s) {
  const long resident = resident_step_threads(pl->device);
  build_tables(pl->P, h.t64, h.t32, h.tp, 4, kMaxGroups, resident);
  const bool sub = has_startup(pl->prob);
  if (sub) {
    pl->sub.P = startup_params(pl->P, pl->prob.init_substeps);
    build_tables(pl->sub.P, h.s64, h.s32, h.sp, 4, kMaxGroups, resident);
  }
  pl->run.P = pl->P;
  const Params &P = pl->P;
  const Layout &L = pl->lay;
  if (P.precision == BSDE_FP64) {
    BSDE_CUDA_TRY(cudaMemcpyAsync(pl->ws + L.table, h.t64, sizeof(NodeF64) * P.k * P.L,
                                  cudaMemcpyHostToDevice, s));
    if (sub)
      BSDE_CUDA_TRY(cudaMemcpyAsync(pl->ws + L.sub_table, h.s64, sizeof(NodeF64) * P.L,
                                    cudaMemcpyHostToDevice, s));
  } else {
    BSDE_CUDA_TRY(cudaMemcpyAsync(pl->ws + L.ptable, h.tp, sizeof(PairF32) * P.k * P.Lp,
                                  cudaMemcpyHostToDevice, s));
    std::memcpy(pl->run.tab.e, h.tp, sizeof(PairF32) * P.k * P.Lp);
    if (sub) std::memcpy(pl->sub.tab.e, h.sp, sizeof(PairF32) * pl->sub.P.Lp);
    if (sub)
      BSDE_CUDA_TRY(cudaMemcpyAsync(pl->ws + L.sub_ptable, h.sp,
                                    sizeof(PairF32) * pl->sub.P.Lp, cudaMemcpyHostToDevice, s));
  }
  return BSDE_OK;
}

// The one-step start-up (Section 3.1 step 2): the 1-step scheme from the
// closed-form level N down K-1 levels of the main grid, S of its steps each;
// level N and every S-th level after it go to row m of the staging area, from
// which the main loop imports its K initial levels.
template <int PREC>
static int64_t enqueue_startup(bsde_plan_t *pl, cudaStream_t s, double *sy, double *sz) {
  const Run &Q = pl->sub;
  const Params &P1 = Q.P;
  const int64_t nx = P1.Nx;
  const int S = pl->prob.init_substeps, K = pl->P.k;
  const unsigned eb = unsigned((nx + 255) / 256 < 4096 ? (nx + 255) / 256 : 4096);
  int64_t launches = 0;
  k_init_closed<PREC><<<eb, 256, 0, s>>>(P1, Q.r64, Q.r32, 0);
  launches += 1 + enqueue_spline<PREC>(Q, s, P1.N % P1.nslot);
  k_export<PREC><<<eb, 256, 0, s>>>(P1, Q.r64, Q.r32, sy, sz, P1.N % P1.nslot);
  ++launches;
  for (int q = 1; q <= (K - 1) * S; ++q) {
    const int n1 = P1.N - q;
    launch_step_any<PREC>(pl, Q, s, n1);
    launches += 1 + enqueue_spline<PREC>(Q, s, n1 % P1.nslot);
    if (q % S == 0) {
      const int m = q / S;
      k_export<PREC><<<eb, 256, 0, s>>>(P1, Q.r64, Q.r32, sy + m * nx, sz + m * nx,
                                        n1 % P1.nslot);
      ++launches;
    }
  }
  return launches;
}

template <int PREC>
static int64_t enqueue_start(bsde_plan_t *pl, cudaStream_t s, bool imported) {
  // stats reset, the start-up if any, the K initial levels and their splines
  const Params &P = pl->P;
  const Run &R = pl->run;
  Stats *st = reinterpret_cast<Stats *>(pl->ws + pl->lay.stats);
  double *sy = reinterpret_cast<double *>(pl->ws + pl->lay.stage);
  double *sz = sy + int64_t(P.k) * P.Nx;
  int64_t launches = 0;
  k_reset_stats<<<1, 32, 0, s>>>(st);
  ++launches;
  if (!imported && has_startup(pl->prob)) {
    launches += enqueue_startup<PREC>(pl, s, sy, sz);
    imported = true;
  }
  const unsigned eb = unsigned((P.Nx + 255) / 256 < 4096 ? (P.Nx + 255) / 256 : 4096);
  for (int m = 0; m < P.k; ++m) {
    if (imported)
      k_import<PREC><<<eb, 256, 0, s>>>(P, R.r64, R.r32, sy, sz, m);
    else
      k_init_closed<PREC><<<eb, 256, 0, s>>>(P, R.r64, R.r32, m);
    ++launches;
    launches += enqueue_spline<PREC>(R, s, (P.N - m) % P.nslot);
  }
  return launches;
}

template <int PREC>
static int64_t enqueue_finish(bsde_plan_t *pl, cudaStream_t s) {
  // readout of level 0 at x0 and its export to the staging area
  const Params &P = pl->P;
  const Run &R = pl->run;
  Stats *st = reinterpret_cast<Stats *>(pl->ws + pl->lay.stats);
  double *sy = reinterpret_cast<double *>(pl->ws + pl->lay.stage);
  const unsigned eb = unsigned((P.Nx + 255) / 256 < 4096 ? (P.Nx + 255) / 256 : 4096);
  k_readout<PREC><<<1, 32, 0, s>>>(P, R.r64, R.r32, 0, st);
  k_export<PREC><<<eb, 256, 0, s>>>(P, R.r64, R.r32, sy, sy + P.Nx, 0);
  return 2;
}

// The whole solve as one stream-ordered sequence (captured into a graph).
template <int PREC>
static int64_t enqueue_solve(bsde_plan_t *pl, cudaStream_t s, bool imported) {
  const Params &P = pl->P;
  const Run &R = pl->run;
  int64_t launches = enqueue_start<PREC>(pl, s, imported);
  for (int n = P.N - P.k; n >= 0; --n) {
    launch_step_any<PREC>(pl, R, s, n);
    ++launches;
    launches += enqueue_spline<PREC>(R, s, n % P.nslot);
  }
  return launches + enqueue_finish<PREC>(pl, s);
}

static int build_graph(bsde_plan_t *pl, int which) {
  cudaStream_t cs;
  BSDE_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(BSDE_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  }
  int64_t n = pl->P.precision == BSDE_FP64 ? enqueue_solve<BSDE_FP64>(pl, cs, which == 1)
                                           : enqueue_solve<BSDE_FP32C>(pl, cs, which == 1);
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(BSDE_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&pl->graph[which], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return fail(BSDE_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  pl->launches[which] = n;
  return BSDE_OK;
}

}  // namespace bsde

extern "C" {

int bsde_workspace_bytes(const bsde_problem *p, size_t *bytes) {
  if (!p || !bytes) return fail(BSDE_EINVAL, "null argument");
  if (validate(*p)) return fail(BSDE_EINVAL, "invalid problem");
  *bytes = layout_for(*p).total;
  return BSDE_OK;
}

int bsde_plan(const bsde_problem *p, void *dev_workspace, size_t bytes, bsde_plan_t **out) {
  if (!p || !out) return fail(BSDE_EINVAL, "null argument");
  *out = nullptr;
  Params P;
  if (fill_params(*p, P)) return fail(BSDE_EINVAL, "invalid problem");
  const Layout lay = layout_for(*p);
  if (!dev_workspace || bytes < lay.total)
    return fail(BSDE_ENOSPC, "workspace smaller than bsde_workspace_bytes()");
  if (reinterpret_cast<uintptr_t>(dev_workspace) % 256)
    return fail(BSDE_EINVAL, "workspace must be 256-byte aligned");
  int device = 0;
  BSDE_CUDA_TRY(cudaGetDevice(&device));
  bsde_plan_t *pl = new (std::nothrow) bsde_plan_t();
  if (!pl) return fail(BSDE_ENOMEM, "plan allocation");
  pl->prob = *p;
  pl->P = P;
  pl->lay = lay;
  pl->device = device;
  pl->ws = static_cast<unsigned char *>(dev_workspace);
  pl->ws_bytes = bytes;
  driver_coefs(P, pl->dc64, pl->dc32);
  // node tables: built on the host, copied once into the workspace
  HostTables *h = new (std::nothrow) HostTables;
  if (!h) {
    delete pl;
    return fail(BSDE_ENOMEM, "table allocation");
  }
  int rc = upload_tables(pl, *h, nullptr);
  cudaError_t e = rc ? cudaErrorUnknown : cudaStreamSynchronize(nullptr);
  delete h;
  if (rc) {
    delete pl;
    return rc;
  }
  bind_runs(pl);
  if (e == cudaSuccess) e = cudaMallocHost(&pl->host_stats, sizeof(Stats));
  if (e != cudaSuccess) {
    delete pl;
    return fail(BSDE_ECUDA, std::string("plan: ") + cudaGetErrorString(e));
  }
  *out = pl;
  return BSDE_OK;
}

static int fill_result(bsde_plan_t *pl, bsde_result *r) {
  const Stats &s = *pl->host_stats;
  r->y0 = s.y0;
  r->z0 = s.z0;
  double d;
  unsigned long long b = s.resid_bits;
  std::memcpy(&d, &b, sizeof(d));
  r->picard_resid_max = d;
  r->picard_iters_max = s.iters_max;
  r->levels_done = pl->P.N - pl->P.k + 1;
  // single solves have no device-side waits (only the server's bounded idle
  // wait sets Stats::timeout), so the status is convergence alone
  r->status = s.nonconv ? BSDE_WARN_NOCONV : BSDE_OK;
  return r->status;
}

int bsde_solve(bsde_plan_t *pl, void *stream, const double *init_y, const double *init_z,
               int init_on_host, double *out_y, double *out_z, int out_on_host,
               bsde_result *result) {
  if (!pl) return fail(BSDE_EINVAL, "null plan");
  if ((init_y == nullptr) != (init_z == nullptr))
    return fail(BSDE_EINVAL, "init_y and init_z must both be given or both be NULL");
  DeviceGuard guard(pl->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Params &P = pl->P;
  const int which = init_y ? 1 : 0;
  if (!pl->graph[which]) {
    int rc = build_graph(pl, which);
    if (rc) return rc;
  }
  double *sy = reinterpret_cast<double *>(pl->ws + pl->lay.stage);
  double *sz = sy + int64_t(P.k) * P.Nx;
  const size_t lev_bytes = size_t(P.k) * size_t(P.Nx) * sizeof(double);
  if (init_y) {
    const cudaMemcpyKind kind = init_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    BSDE_CUDA_TRY(cudaMemcpyAsync(sy, init_y, lev_bytes, kind, s));
    BSDE_CUDA_TRY(cudaMemcpyAsync(sz, init_z, lev_bytes, kind, s));
  }
  BSDE_CUDA_TRY(cudaGraphLaunch(pl->graph[which], s));
  const size_t out_bytes = size_t(P.Nx) * sizeof(double);
  const cudaMemcpyKind okind = out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (out_y) BSDE_CUDA_TRY(cudaMemcpyAsync(out_y, sy, out_bytes, okind, s));
  if (out_z) BSDE_CUDA_TRY(cudaMemcpyAsync(out_z, sy + P.Nx, out_bytes, okind, s));
  BSDE_CUDA_TRY(cudaMemcpyAsync(pl->host_stats, pl->ws + pl->lay.stats, sizeof(Stats),
                                cudaMemcpyDeviceToHost, s));
  const bool host_ptrs = (init_y && init_on_host) || ((out_y || out_z) && out_on_host);
  if (result || host_ptrs) BSDE_CUDA_TRY(cudaStreamSynchronize(s));
  if (result) return fill_result(pl, result);
  return BSDE_OK;
}

int bsde_result_fetch(bsde_plan_t *pl, void *stream, bsde_result *result) {
  if (!pl || !result) return fail(BSDE_EINVAL, "null argument");
  DeviceGuard guard(pl->device);
  BSDE_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return fill_result(pl, result);
}

int bsde_enqueue_level(bsde_plan_t *pl, void *stream, int n, int parts) {
  if (!pl) return fail(BSDE_EINVAL, "null plan");
  if (n < 0 || n > pl->P.N - pl->P.k) return fail(BSDE_EINVAL, "level out of range");
  DeviceGuard guard(pl->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (parts & 1) {
    if (pl->P.precision == BSDE_FP64) launch_step_any<BSDE_FP64>(pl, pl->run, s, n);
    else launch_step_any<BSDE_FP32C>(pl, pl->run, s, n);
  }
  if (parts & 2) {
    if (pl->P.precision == BSDE_FP64) enqueue_spline<BSDE_FP64>(pl->run, s, n % pl->P.nslot);
    else enqueue_spline<BSDE_FP32C>(pl->run, s, n % pl->P.nslot);
  }
  BSDE_CUDA_TRY(cudaGetLastError());
  return BSDE_OK;
}

int bsde_enqueue_start(bsde_plan_t *pl, void *stream, const double *init_y, const double *init_z,
                       int init_on_host) {
  if (!pl) return fail(BSDE_EINVAL, "null plan");
  if ((init_y == nullptr) != (init_z == nullptr))
    return fail(BSDE_EINVAL, "init_y and init_z must both be given or both be NULL");
  DeviceGuard guard(pl->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Params &P = pl->P;
  if (init_y) {
    double *sy = reinterpret_cast<double *>(pl->ws + pl->lay.stage);
    double *sz = sy + int64_t(P.k) * P.Nx;
    const size_t lev_bytes = size_t(P.k) * size_t(P.Nx) * sizeof(double);
    const cudaMemcpyKind kind = init_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    BSDE_CUDA_TRY(cudaMemcpyAsync(sy, init_y, lev_bytes, kind, s));
    BSDE_CUDA_TRY(cudaMemcpyAsync(sz, init_z, lev_bytes, kind, s));
  }
  if (P.precision == BSDE_FP64)
    enqueue_start<BSDE_FP64>(pl, s, init_y != nullptr);
  else
    enqueue_start<BSDE_FP32C>(pl, s, init_y != nullptr);
  BSDE_CUDA_TRY(cudaGetLastError());
  if (init_y && init_on_host) BSDE_CUDA_TRY(cudaStreamSynchronize(s));
  return BSDE_OK;
}

int bsde_enqueue_finish(bsde_plan_t *pl, void *stream, double *out_y, double *out_z,
                        int out_on_host) {
  if (!pl) return fail(BSDE_EINVAL, "null plan");
  DeviceGuard guard(pl->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Params &P = pl->P;
  if (P.precision == BSDE_FP64)
    enqueue_finish<BSDE_FP64>(pl, s);
  else
    enqueue_finish<BSDE_FP32C>(pl, s);
  BSDE_CUDA_TRY(cudaGetLastError());
  const double *sy = reinterpret_cast<const double *>(pl->ws + pl->lay.stage);
  const size_t out_bytes = size_t(P.Nx) * sizeof(double);
  const cudaMemcpyKind okind = out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (out_y) BSDE_CUDA_TRY(cudaMemcpyAsync(out_y, sy, out_bytes, okind, s));
  if (out_z) BSDE_CUDA_TRY(cudaMemcpyAsync(out_z, sy + P.Nx, out_bytes, okind, s));
  BSDE_CUDA_TRY(cudaMemcpyAsync(pl->host_stats, pl->ws + pl->lay.stats, sizeof(Stats),
                                cudaMemcpyDeviceToHost, s));
  if ((out_y || out_z) && out_on_host) BSDE_CUDA_TRY(cudaStreamSynchronize(s));
  return BSDE_OK;
}

int bsde_level_records(bsde_plan_t *pl, int n, void **records, size_t *record_bytes) {
  if (!pl || !records || !record_bytes) return fail(BSDE_EINVAL, "null argument");
  const Params &P = pl->P;
  if (n < 0 || n > P.N) return fail(BSDE_EINVAL, "level out of range");
  const size_t slot = size_t(n % P.nslot);
  if (P.precision == BSDE_FP64) {
    *records = pl->ws + pl->lay.ring64 + slot * size_t(P.Nx) * 32;
    *record_bytes = 32;
  } else {
    *records = pl->ws + pl->lay.ringA + slot * size_t(P.Nx) * 16;
    *record_bytes = 16;
  }
  return BSDE_OK;
}

void bsde_free(bsde_plan_t *pl) {
  if (!pl) return;
  DeviceGuard guard(pl->device);
  for (int w = 0; w < 2; ++w)
    if (pl->graph[w]) cudaGraphExecDestroy(pl->graph[w]);
  if (pl->host_stats) cudaFreeHost(pl->host_stats);
  delete pl;
}

int64_t bsde_plan_launches(const bsde_plan_t *pl) {
  if (!pl) return 0;
  // kernels in one solve without caller levels (with them the start-up, if
  // any, is not run; the rest is the same)
  const Params &P = pl->P;
  int64_t n = 1 + int64_t(P.k) * 2 + int64_t(P.N - P.k + 1) * 2 + 2;
  if (has_startup(pl->prob)) {
    const int64_t steps = int64_t(P.k - 1) * pl->prob.init_substeps;
    n += 3 + 2 * steps + (P.k - 1);
  }
  return n;
}

const char *bsde_strerror(int code) {
  switch (code) {
    case BSDE_OK: return "ok";
    case BSDE_WARN_NOCONV: return "Picard iteration reached picard_max without converging";
    case BSDE_EINVAL: return "invalid argument or problem";
    case BSDE_ENOSPC: return "workspace too small";
    case BSDE_ECUDA: return "CUDA error";
    case BSDE_ENOMEM: return "host allocation failed";
    case BSDE_ETIMEOUT: return "bounded device-side wait expired";
    default: return "unknown code";
  }
}

const char *bsde_last_error(void) { return g_last_error.c_str(); }

int bsde_gauss_hermite(int L, double *nodes, double *weights) {
  if (!nodes || !weights) return BSDE_EINVAL;
  return gauss_hermite(L, nodes, weights);
}

int bsde_gamma(int k, double *gy, double *gz) {
  if (!gy || !gz) return BSDE_EINVAL;
  return gamma_tables(k, gy, gz);
}

int bsde_l2_read_probe(const void *buf, size_t bytes, int reps, int grid, void *sink,
                       void *stream) {
  if (!buf || !sink || reps < 1 || grid < 1 || grid > 65535 || bytes % 16 ||
      reinterpret_cast<uintptr_t>(buf) % 16 || bytes < size_t(16) * 256 * size_t(grid))
    return fail(BSDE_EINVAL, "bad probe arguments");
  k_l2_read<<<unsigned(grid), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const float4 *>(buf), bytes / 16, reps, static_cast<float *>(sink));
  BSDE_CUDA_TRY(cudaGetLastError());
  return BSDE_OK;
}

int bsde_fma_probe(int kind, int iters, int grid, void *sink, void *stream, int64_t *flops) {
  if (!sink || kind < 0 || kind > 2 || iters < 1 || grid < 1 || grid > 65535)
    return fail(BSDE_EINVAL, "bad probe arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *out = static_cast<double *>(sink);
  const unsigned g = unsigned(grid);
  if (kind == 0) k_fma_probe<double><<<g, 256, 0, s>>>(iters, out);
  else if (kind == 1) k_fma_probe<float><<<g, 256, 0, s>>>(iters, out);
  else k_fma_probe<float2><<<g, 256, 0, s>>>(iters, out);
  BSDE_CUDA_TRY(cudaGetLastError());
  if (flops)
    *flops = int64_t(grid) * 256 * kFmaChains * kFmaUnroll * int64_t(iters) * 2 * (kind == 2 ? 2 : 1);
  return BSDE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Solve without allocating: the workspace is a fixed array in device memory
// reserved when the library is loaded.  Host code never touches `noalloc_ws`
// by name as a device address (in host code the symbol is a host-side
// stand-in); it asks the runtime for each device's address once and caches
// it.
// ---------------------------------------------------------------------------
namespace bsde {

static __device__ __align__(256) unsigned char noalloc_ws[BSDE_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
static unsigned char *g_noalloc_addr[kMaxDevices];
static std::mutex g_noalloc_mu;

// The host side of a no-allocation solve: the plan and its node tables
// (about 130 KB), kept in this file-scope buffer rather than on the caller's
// stack, which may be small (a plug-in thread, a musl thread's 128 KB).
// Guarded by g_noalloc_mu for the whole call.
struct NoallocHost {
  bsde_plan_t pl;
  HostTables tabs;
  Stats st;
};
static NoallocHost g_noalloc_host;

// Called with g_noalloc_mu held.
static int noalloc_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(BSDE_EINVAL, "device ordinal out of range");
  if (!g_noalloc_addr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, noalloc_ws);
    if (e != cudaSuccess || ptr == nullptr)
      return fail(BSDE_ECUDA, std::string("cudaGetSymbolAddress(noalloc workspace): ") +
                                  cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<unsigned char *>(ptr);
  }
  *out = g_noalloc_addr[dev];
  return BSDE_OK;
}

}  // namespace bsde

extern "C" int bsde_solve_noalloc(const bsde_problem *p, void *stream, const double *init_y,
                                  const double *init_z, int init_on_host, double *out_y,
                                  double *out_z, int out_on_host, bsde_result *result) {
  if (!p) return fail(BSDE_EINVAL, "null problem");
  if ((init_y == nullptr) != (init_z == nullptr))
    return fail(BSDE_EINVAL, "init_y and init_z must both be given or both be NULL");
  // the plan and its tables live in a file-scope buffer: no host or device
  // allocation, and little of the caller's stack; one call at a time
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoallocHost &H = g_noalloc_host;
  bsde_plan_t &pl = H.pl;
  pl = bsde_plan_t{};
  if (fill_params(*p, pl.P)) return fail(BSDE_EINVAL, "invalid problem");
  pl.lay = layout_for(*p);
  if (pl.lay.total > BSDE_NOALLOC_MAX_BYTES)
    return fail(BSDE_ENOSPC, "problem needs " + std::to_string(pl.lay.total) +
                                 " bytes of workspace; the no-allocation workspace holds " +
                                 std::to_string(size_t(BSDE_NOALLOC_MAX_BYTES)));
  pl.prob = *p;
  BSDE_CUDA_TRY(cudaGetDevice(&pl.device));
  int rc = noalloc_address(pl.device, &pl.ws);
  if (rc) return rc;
  pl.ws_bytes = BSDE_NOALLOC_MAX_BYTES;
  driver_coefs(pl.P, pl.dc64, pl.dc32);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc2 = upload_tables(&pl, H.tabs, s);
  if (rc2) return rc2;
  bind_runs(&pl);
  const Params &P = pl.P;
  // the next call rewrites the host tables: wait for their copies
  BSDE_CUDA_TRY(cudaStreamSynchronize(s));
  double *sy = reinterpret_cast<double *>(pl.ws + pl.lay.stage);
  double *sz = sy + int64_t(P.k) * P.Nx;
  const size_t lev_bytes = size_t(P.k) * size_t(P.Nx) * sizeof(double);
  if (init_y) {
    const cudaMemcpyKind kind = init_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    BSDE_CUDA_TRY(cudaMemcpyAsync(sy, init_y, lev_bytes, kind, s));
    BSDE_CUDA_TRY(cudaMemcpyAsync(sz, init_z, lev_bytes, kind, s));
  }
  if (P.precision == BSDE_FP64)
    enqueue_solve<BSDE_FP64>(&pl, s, init_y != nullptr);
  else
    enqueue_solve<BSDE_FP32C>(&pl, s, init_y != nullptr);
  BSDE_CUDA_TRY(cudaGetLastError());
  const size_t out_bytes = size_t(P.Nx) * sizeof(double);
  const cudaMemcpyKind okind = out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (out_y) BSDE_CUDA_TRY(cudaMemcpyAsync(out_y, sy, out_bytes, okind, s));
  if (out_z) BSDE_CUDA_TRY(cudaMemcpyAsync(out_z, sy + P.Nx, out_bytes, okind, s));
  H.st = Stats{};
  BSDE_CUDA_TRY(cudaMemcpyAsync(&H.st, pl.ws + pl.lay.stats, sizeof(Stats),
                                cudaMemcpyDeviceToHost, s));
  BSDE_CUDA_TRY(cudaStreamSynchronize(s));
  if (!result) return BSDE_OK;
  pl.host_stats = &H.st;
  return fill_result(&pl, result);
}

// ---------------------------------------------------------------------------
// Batched solves: host side
// ---------------------------------------------------------------------------
struct bsde_batch_s {
  int n = 0, device = 0;
  unsigned char *ws = nullptr;
  size_t ws_bytes = 0;
  size_t off_desc = 0, off_order = 0, off_queue = 0, off_stats = 0;
  std::vector<bsde_problem> probs;
  std::vector<size_t> off_ptable, off_ringA, off_ringB;
  bsde_batch_config cfg{};
  int desc_groups = 0;  // target_groups the device descriptors were built with
  int desc_flat = -1;   // and their step-tile form (flat_tiles)
  cudaGraphExec_t graph = nullptr;
  int graph_cluster = 0, graph_groups = 0, graph_flat = -1;
  Stats *host_stats = nullptr;
};

namespace bsde {

struct BatchLayout {
  size_t off_desc, off_order, off_queue, off_stats, total;
  std::vector<size_t> ptable, ringA, ringB;
};

static int batch_layout(int n, const bsde_problem *ps, BatchLayout &L) {
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  size_t off = 0;
  L.off_desc = off; off = up(off + size_t(n) * sizeof(InstDesc));
  L.off_order = off; off = up(off + size_t(n) * sizeof(int));
  L.off_queue = off; off = up(off + 16);
  L.off_stats = off; off = up(off + size_t(n) * sizeof(Stats));
  L.ptable.resize(n);
  L.ringA.resize(n);
  L.ringB.resize(n);
  for (int i = 0; i < n; ++i) {
    const bsde_problem &p = ps[i];
    // batches start from the closed form (no one-step start-up)
    if (validate(p) || p.precision != BSDE_FP32C || has_startup(p) || problem_general(p))
      return BSDE_EINVAL;
    const size_t K = size_t(problem_K(p));
    const size_t nx = size_t(p.Nx), ns = K + 1;
    L.ptable[i] = off; off = up(off + K * ((p.L + 1) / 2) * sizeof(PairF32));
    L.ringA[i] = off; off = up(off + ns * nx * 16);
    L.ringB[i] = off; off = up(off + ns * nx * 8);
  }
  L.total = off;
  return BSDE_OK;
}

// Descriptors, pair tables and the largest-first order, copied to the device.
// Every problem takes the batch's step-tile form (flat or grouped).
static int batch_upload(bsde_batch_t *b, int target_groups, int flat) {
  const int n = b->n;
  std::vector<InstDesc> descs(n);
  std::vector<double> work(n);
  std::vector<NodeF32> t32(kMaxK * kMaxL);
  std::vector<PairF32> tp(kMaxK * kMaxL);
  for (int i = 0; i < n; ++i) {
    InstDesc &D = descs[i];
    std::memset(&D, 0, sizeof(D));
    fill_params(b->probs[i], D.P);
    build_tables(D.P, nullptr, t32.data(), tp.data(), target_groups, 6);
    D.P.flat = flat;
    DrvC<double> c64;
    driver_coefs(D.P, c64, D.dc32);
    D.ringA = int64_t(b->off_ringA[i]);
    D.ringB = int64_t(b->off_ringB[i]);
    D.ptable = int64_t(b->off_ptable[i]);
    BSDE_CUDA_TRY(cudaMemcpy(b->ws + b->off_ptable[i], tp.data(),
                             sizeof(PairF32) * D.P.k * D.P.Lp, cudaMemcpyHostToDevice));
    work[i] = double(D.P.Nx) * double(D.P.N - D.P.k + 1) * double(D.P.k) * double(D.P.L);
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
  BSDE_CUDA_TRY(cudaMemcpy(b->ws + b->off_desc, descs.data(), sizeof(InstDesc) * n,
                           cudaMemcpyHostToDevice));
  BSDE_CUDA_TRY(cudaMemcpy(b->ws + b->off_order, order.data(), sizeof(int) * n,
                           cudaMemcpyHostToDevice));
  b->desc_groups = target_groups;
  b->desc_flat = flat;
  return BSDE_OK;
}

static int batch_enqueue(bsde_batch_t *b, cudaStream_t s) {
  const int n = b->n;
  int *queue = reinterpret_cast<int *>(b->ws + b->off_queue);
  Stats *stats = reinterpret_cast<Stats *>(b->ws + b->off_stats);
  k_batch_reset<<<(n + 255) / 256, 256, 0, s>>>(queue, stats, n);
  const size_t smem = sizeof(BatchSmem);
  auto *kern = b->cfg.flat_tiles ? k_batch32<true> : k_batch32<false>;
  BSDE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem)));
  const int cl = b->cfg.cluster;
  cudaLaunchConfig_t lc{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(cl);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(b->cfg.flat_tiles ? kBatchFlatThreads : kBatchThreads, 1, 1);
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  lc.attrs = attr;
  lc.numAttrs = 1;
  lc.gridDim = dim3(unsigned(cl), 1, 1);
  int active = 0;
  BSDE_CUDA_TRY(cudaOccupancyMaxActiveClusters(&active, kern, &lc));
  if (active < 1) return fail(BSDE_ECUDA, "batch kernel: no cluster fits on the device");
  const int clusters = std::min(active, n);
  lc.gridDim = dim3(unsigned(clusters * cl), 1, 1);
  const InstDesc *descs = reinterpret_cast<const InstDesc *>(b->ws + b->off_desc);
  const int *order = reinterpret_cast<const int *>(b->ws + b->off_order);
  BSDE_CUDA_TRY(cudaLaunchKernelEx(&lc, kern, descs, order, n, queue, b->ws, stats));
  return BSDE_OK;
}

static int batch_graph(bsde_batch_t *b) {
  const int flat = b->cfg.flat_tiles;
  if (b->graph && b->graph_cluster == b->cfg.cluster && b->graph_groups == b->cfg.target_groups &&
      b->graph_flat == flat)
    return BSDE_OK;
  if (b->desc_groups != b->cfg.target_groups || b->desc_flat != flat) {
    int rc = batch_upload(b, b->cfg.target_groups, flat);
    if (rc) return rc;
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaStream_t cs;
  BSDE_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = BSDE_OK;
  if (e == cudaSuccess) {
    rc = batch_enqueue(b, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  cudaStreamDestroy(cs);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(BSDE_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return fail(BSDE_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  b->graph_cluster = b->cfg.cluster;
  b->graph_groups = b->cfg.target_groups;
  b->graph_flat = flat;
  return BSDE_OK;
}

static bool valid_config(const bsde_batch_config &c) {
  return (c.cluster == 1 || c.cluster == 2 || c.cluster == 4 || c.cluster == 8) &&
         c.target_groups >= 1 && c.target_groups <= 6 && (c.flat_tiles == 0 || c.flat_tiles == 1);
}

}  // namespace bsde

extern "C" {

int bsde_batch_workspace_bytes(int n, const bsde_problem *ps, size_t *bytes) {
  if (n < 1 || !ps || !bytes) return fail(BSDE_EINVAL, "bad batch arguments");
  BatchLayout L;
  if (batch_layout(n, ps, L)) return fail(BSDE_EINVAL, "invalid problem in batch (FP32C only)");
  *bytes = L.total;
  return BSDE_OK;
}

int bsde_plan_batch(int n, const bsde_problem *ps, void *dev_workspace, size_t bytes,
                    bsde_batch_t **out) {
  if (!out) return fail(BSDE_EINVAL, "null argument");
  *out = nullptr;
  if (n < 1 || !ps) return fail(BSDE_EINVAL, "bad batch arguments");
  BatchLayout L;
  if (batch_layout(n, ps, L)) return fail(BSDE_EINVAL, "invalid problem in batch (FP32C only)");
  if (!dev_workspace || bytes < L.total)
    return fail(BSDE_ENOSPC, "workspace smaller than bsde_batch_workspace_bytes()");
  if (reinterpret_cast<uintptr_t>(dev_workspace) % 256)
    return fail(BSDE_EINVAL, "workspace must be 256-byte aligned");
  int device = 0;
  BSDE_CUDA_TRY(cudaGetDevice(&device));
  bsde_batch_t *b = new (std::nothrow) bsde_batch_t();
  if (!b) return fail(BSDE_ENOMEM, "batch allocation");
  b->n = n;
  b->device = device;
  b->ws = static_cast<unsigned char *>(dev_workspace);
  b->ws_bytes = bytes;
  b->off_desc = L.off_desc;
  b->off_order = L.off_order;
  b->off_queue = L.off_queue;
  b->off_stats = L.off_stats;
  b->off_ptable = L.ptable;
  b->off_ringA = L.ringA;
  b->off_ringB = L.ringB;
  b->probs.assign(ps, ps + n);
  b->cfg.cluster = 2;
  b->cfg.target_groups = 4;
  b->cfg.flat_tiles = 0;
  int rc = batch_upload(b, b->cfg.target_groups, b->cfg.flat_tiles);
  if (rc == BSDE_OK && cudaMallocHost(&b->host_stats, sizeof(Stats) * size_t(n)) != cudaSuccess)
    rc = fail(BSDE_ECUDA, "pinned result buffer");
  if (rc) {
    delete b;
    return rc;
  }
  *out = b;
  return BSDE_OK;
}

int bsde_batch_set_config(bsde_batch_t *b, const bsde_batch_config *cfg) {
  if (!b || !cfg || !valid_config(*cfg)) return fail(BSDE_EINVAL, "bad batch configuration");
  b->cfg = *cfg;
  return BSDE_OK;
}

int bsde_batch_get_config(const bsde_batch_t *b, bsde_batch_config *cfg) {
  if (!b || !cfg) return fail(BSDE_EINVAL, "null argument");
  *cfg = b->cfg;
  return BSDE_OK;
}

int bsde_solve_batch(bsde_batch_t *b, void *stream, bsde_result *results) {
  if (!b) return fail(BSDE_EINVAL, "null batch");
  DeviceGuard guard(b->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = batch_graph(b);
  if (rc) return rc;
  BSDE_CUDA_TRY(cudaGraphLaunch(b->graph, s));
  if (!results) return BSDE_OK;
  BSDE_CUDA_TRY(cudaMemcpyAsync(b->host_stats, b->ws + b->off_stats, sizeof(Stats) * b->n,
                                cudaMemcpyDeviceToHost, s));
  BSDE_CUDA_TRY(cudaStreamSynchronize(s));
  int worst = BSDE_OK;
  for (int i = 0; i < b->n; ++i) {
    const Stats &st = b->host_stats[i];
    bsde_result &r = results[i];
    r.y0 = st.y0;
    r.z0 = st.z0;
    double d;
    unsigned long long bits = st.resid_bits;
    std::memcpy(&d, &bits, sizeof(d));
    r.picard_resid_max = d;
    r.picard_iters_max = st.iters_max;
    r.levels_done = b->probs[i].N - problem_K(b->probs[i]) + 1;
    r.status = st.nonconv ? BSDE_WARN_NOCONV : BSDE_OK;
    if (r.status != BSDE_OK) worst = r.status;
  }
  return worst;
}

int bsde_batch_autotune(bsde_batch_t *b, void *stream, bsde_batch_config *best) {
  if (!b) return fail(BSDE_EINVAL, "null batch");
  DeviceGuard guard(b->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bsde_batch_config keep = b->cfg;
  bsde_batch_config win = keep;
  float win_ms = -1.f;
  cudaEvent_t e0, e1;
  BSDE_CUDA_TRY(cudaEventCreate(&e0));
  BSDE_CUDA_TRY(cudaEventCreate(&e1));
  // the step-tile forms: grouped tiles with 2, 4 or 6 groups of threads per
  // point, and flat tiles (one point per thread, its groups in turn; one
  // group per step j)
  const int clusters[4] = {1, 2, 4, 8};
  const int forms[4][2] = {{2, 0}, {4, 0}, {6, 0}, {1, 1}};  // {target_groups, flat_tiles}
  int rc = BSDE_OK;
  for (int fi = 0; fi < 4 && rc == BSDE_OK; ++fi) {
    for (int ci = 0; ci < 4 && rc == BSDE_OK; ++ci) {
      b->cfg.cluster = clusters[ci];
      b->cfg.target_groups = forms[fi][0];
      b->cfg.flat_tiles = forms[fi][1];
      rc = batch_graph(b);
      if (rc) break;
      if (cudaGraphLaunch(b->graph, s) != cudaSuccess) { rc = fail(BSDE_ECUDA, "autotune launch"); break; }
      cudaEventRecord(e0, s);
      cudaGraphLaunch(b->graph, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(BSDE_ECUDA, "autotune timing"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (win_ms < 0.f || ms < win_ms) {
        win_ms = ms;
        win = b->cfg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cfg = rc ? keep : win;
  if (rc) return rc;
  if (best) *best = win;
  return BSDE_OK;
}

void bsde_batch_free(bsde_batch_t *b) {
  if (!b) return;
  DeviceGuard guard(b->device);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->host_stats) cudaFreeHost(b->host_stats);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Continuous-batching server: host side
// ---------------------------------------------------------------------------
struct bsde_server_s {
  int device = 0, nslots = 0;
  unsigned char *ws = nullptr;
  size_t ws_bytes = 0, off_dev = 0, off_stats = 0, off_pool = 0, pool_bytes = 0;
  ServerCtl *ctl = nullptr;   // host view of the mapped control block
  ServerCtl *ctl_d = nullptr; // device view
  ServerSlot *slots = nullptr, *slots_d = nullptr;
  std::vector<int> free_slots;
  std::vector<size_t> slot_off, slot_size;
  std::vector<char> busy;
  std::map<size_t, size_t> free_blocks;  // pool offset -> bytes
  uint32_t tail = 0;
  bool running = false;
  cudaStream_t stream = nullptr;
};

namespace bsde {

static size_t request_bytes(const bsde_problem &p) {
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t nx = size_t(p.Nx), ns = size_t(problem_K(p) + 1);
  return up(ns * nx * 16) + up(ns * nx * 8);
}

static bool pool_alloc(bsde_server_t *s, size_t bytes, size_t &off) {
  for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      off = it->first;
      const size_t rest = it->second - bytes;
      s->free_blocks.erase(it);
      if (rest) s->free_blocks[off + bytes] = rest;
      return true;
    }
  }
  return false;
}

static void pool_free(bsde_server_t *s, size_t off, size_t bytes) {
  auto it = s->free_blocks.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_blocks.erase(nx);
  }
  if (it != s->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_blocks.erase(it);
    }
  }
}

}  // namespace bsde

extern "C" {

int bsde_request_bytes(const bsde_problem *p, size_t *bytes) {
  if (!p || !bytes) return fail(BSDE_EINVAL, "null argument");
  if (validate(*p) || p->precision != BSDE_FP32C || has_startup(*p) || problem_general(*p))
    return fail(BSDE_EINVAL, "invalid request");
  *bytes = request_bytes(*p);
  return BSDE_OK;
}

int bsde_server_workspace_bytes(int slots, size_t pool_bytes, size_t *bytes) {
  // at most one unread ring entry per slot: slots <= ring positions
  if (slots < 1 || slots > kServerRing || !bytes) return fail(BSDE_EINVAL, "bad server arguments");
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  *bytes = up(sizeof(ServerDev)) + up(sizeof(Stats) * size_t(slots)) + up(pool_bytes);
  return BSDE_OK;
}

int bsde_server_create(void *dev_workspace, size_t bytes, int slots, size_t pool_bytes,
                       bsde_server_t **out) {
  if (!out) return fail(BSDE_EINVAL, "null argument");
  *out = nullptr;
  size_t need = 0;
  int rc = bsde_server_workspace_bytes(slots, pool_bytes, &need);
  if (rc) return rc;
  if (!dev_workspace || bytes < need) return fail(BSDE_ENOSPC, "server workspace too small");
  if (reinterpret_cast<uintptr_t>(dev_workspace) % 256)
    return fail(BSDE_EINVAL, "workspace must be 256-byte aligned");
  int device = 0;
  BSDE_CUDA_TRY(cudaGetDevice(&device));
  bsde_server_t *s = new (std::nothrow) bsde_server_t();
  if (!s) return fail(BSDE_ENOMEM, "server allocation");
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  s->device = device;
  s->nslots = slots;
  s->ws = static_cast<unsigned char *>(dev_workspace);
  s->ws_bytes = bytes;
  s->off_dev = 0;
  s->off_stats = up(sizeof(ServerDev));
  s->off_pool = s->off_stats + up(sizeof(Stats) * size_t(slots));
  s->pool_bytes = pool_bytes;
  cudaError_t e = cudaHostAlloc(&s->ctl, sizeof(ServerCtl), cudaHostAllocMapped);
  if (e == cudaSuccess)
    e = cudaHostAlloc(&s->slots, sizeof(ServerSlot) * size_t(slots), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->ctl_d, s->ctl, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->slots_d, s->slots, 0);
  if (e != cudaSuccess) {
    if (s->ctl) cudaFreeHost(s->ctl);
    if (s->slots) cudaFreeHost(s->slots);
    delete s;
    return fail(BSDE_ECUDA, std::string("server host memory: ") + cudaGetErrorString(e));
  }
  std::memset(s->ctl, 0, sizeof(ServerCtl));
  std::memset(s->slots, 0, sizeof(ServerSlot) * size_t(slots));
  s->free_slots.resize(slots);
  for (int i = 0; i < slots; ++i) s->free_slots[i] = slots - 1 - i;
  s->slot_off.assign(slots, 0);
  s->slot_size.assign(slots, 0);
  s->busy.assign(slots, 0);
  if (pool_bytes) s->free_blocks[0] = pool_bytes;
  *out = s;
  return BSDE_OK;
}

int bsde_server_start(bsde_server_t *s, void *stream, int cluster, int idle_ms) {
  if (!s || s->running) return fail(BSDE_EINVAL, "server missing or already running");
  if (!(cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8) || idle_ms < 1)
    return fail(BSDE_EINVAL, "bad server launch arguments");
  DeviceGuard guard(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < s->nslots; ++i)
    if (s->busy[i]) return fail(BSDE_EINVAL, "poll every request of the last run before a restart");
  // a fresh run: the device claims ring positions from 0 again
  s->tail = 0;
  s->ctl->req_tail = 0;
  s->ctl->shutdown = 0;
  s->ctl->stopped = 0;
  BSDE_CUDA_TRY(cudaMemsetAsync(s->ws + s->off_dev, 0, sizeof(ServerDev), st));
  const size_t smem = sizeof(BatchSmem);
  BSDE_CUDA_TRY(cudaFuncSetAttribute(k_server32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem)));
  cudaLaunchConfig_t lc{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(cluster);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(kBatchFlatThreads, 1, 1);  // requests run flat step tiles
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  lc.attrs = attr;
  lc.numAttrs = 1;
  lc.gridDim = dim3(unsigned(cluster), 1, 1);
  int active = 0;
  BSDE_CUDA_TRY(cudaOccupancyMaxActiveClusters(&active, k_server32, &lc));
  if (active < 1) return fail(BSDE_ECUDA, "server kernel: no cluster fits on the device");
  lc.gridDim = dim3(unsigned(active * cluster), 1, 1);
  BSDE_CUDA_TRY(cudaLaunchKernelEx(&lc, k_server32, s->ctl_d, s->slots_d,
                                   reinterpret_cast<ServerDev *>(s->ws + s->off_dev),
                                   reinterpret_cast<Stats *>(s->ws + s->off_stats),
                                   s->ws + s->off_pool,
                                   (unsigned long long)idle_ms * 1000000ull));
  s->running = true;
  s->stream = st;
  return BSDE_OK;
}

int bsde_server_submit(bsde_server_t *s, const bsde_problem *p, int *slot) {
  if (!s || !p || !slot) return fail(BSDE_EINVAL, "null argument");
  if (!s->running) return fail(BSDE_EINVAL, "server not running");
  if (__atomic_load_n(&s->ctl->stopped, __ATOMIC_ACQUIRE))
    return fail(BSDE_ETIMEOUT, "server stopped: its idle limit passed; poll, stop and start it again");
  if (validate(*p) || p->precision != BSDE_FP32C || has_startup(*p) || problem_general(*p))
    return fail(BSDE_EINVAL, "invalid request");
  if (s->free_slots.empty()) return BSDE_BUSY;
  const size_t need = request_bytes(*p);
  size_t off = 0;
  if (!pool_alloc(s, need, off)) return BSDE_BUSY;
  const int sl = s->free_slots.back();
  s->free_slots.pop_back();
  ServerSlot &S = s->slots[sl];
  InstDesc D;
  std::memset(&D, 0, sizeof(D));
  fill_params(*p, D.P);
  {
    NodeF32 t32[kMaxK * kMaxL];
    PairF32 tp[kMaxK * kMaxL];
    build_tables(D.P, nullptr, t32, tp, 4, 6);
    std::memcpy(S.tab, tp, sizeof(PairF32) * size_t(D.P.k) * size_t(D.P.Lp));
    // the serving kernel runs flat step tiles (bitwise the grouped tiles'
    // results at the same group split)
    D.P.flat = 1;
  }
  DrvC<double> c64;
  driver_coefs(D.P, c64, D.dc32);
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t nx = size_t(p->Nx), ns = size_t(p->k + 1);
  D.ringA = int64_t(off);
  D.ringB = int64_t(off + up(ns * nx * 16));
  D.ptable = 0;
  S.D = D;
  S.done = 0;
  s->slot_off[sl] = off;
  s->slot_size[sl] = need;
  s->busy[sl] = 1;
  // publish: slot data before the ring entry before the tail
  s->ctl->req_slot[s->tail % kServerRing] = sl;
  std::atomic_thread_fence(std::memory_order_release);
  __atomic_store_n(&s->ctl->req_tail, s->tail + 1, __ATOMIC_RELEASE);
  ++s->tail;
  *slot = sl;
  return BSDE_OK;
}

int bsde_server_poll(bsde_server_t *s, int max, int *slots, bsde_result *results) {
  if (!s || max < 0) return fail(BSDE_EINVAL, "bad poll arguments");
  // once the device has stopped itself and its kernel has ended, requests
  // still without a result will never get one: report them as timed out
  bool lost = false;
  if (s->running && __atomic_load_n(&s->ctl->stopped, __ATOMIC_ACQUIRE)) {
    DeviceGuard guard(s->device);
    lost = cudaStreamQuery(s->stream) == cudaSuccess;
  }
  int got = 0;
  for (int sl = 0; sl < s->nslots && got < max; ++sl) {
    if (!s->busy[sl]) continue;
    const bool done = __atomic_load_n(&s->slots[sl].done, __ATOMIC_ACQUIRE) == 1u;
    if (!done && !lost) continue;
    Stats st = s->slots[sl].result;
    if (!done) {
      std::memset(&st, 0, sizeof(st));
      st.y0 = st.z0 = std::nan("");
      st.timeout = 1;
    }
    if (results) {
      bsde_result &r = results[got];
      r.y0 = st.y0;
      r.z0 = st.z0;
      double d;
      unsigned long long bits = st.resid_bits;
      std::memcpy(&d, &bits, sizeof(d));
      r.picard_resid_max = d;
      r.picard_iters_max = st.iters_max;
      r.levels_done = s->slots[sl].D.P.N - s->slots[sl].D.P.k + 1;
      r.status = st.timeout ? BSDE_ETIMEOUT : (st.nonconv ? BSDE_WARN_NOCONV : BSDE_OK);
    }
    if (slots) slots[got] = sl;
    ++got;
    s->busy[sl] = 0;
    pool_free(s, s->slot_off[sl], s->slot_size[sl]);
    s->free_slots.push_back(sl);
  }
  return got;
}

int bsde_server_stop(bsde_server_t *s) {
  if (!s) return fail(BSDE_EINVAL, "null server");
  if (!s->running) return BSDE_OK;
  DeviceGuard guard(s->device);
  __atomic_store_n(&s->ctl->shutdown, 1u, __ATOMIC_RELEASE);
  BSDE_CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->running = false;
  ServerDev dev{};
  BSDE_CUDA_TRY(cudaMemcpy(&dev, s->ws + s->off_dev, sizeof(dev), cudaMemcpyDeviceToHost));
  if (dev.error) return fail(BSDE_ETIMEOUT, "a server cluster waited longer than idle_ms");
  return BSDE_OK;
}

void bsde_server_free(bsde_server_t *s) {
  if (!s) return;
  DeviceGuard guard(s->device);
  if (s->running) bsde_server_stop(s);
  if (s->ctl) cudaFreeHost(s->ctl);
  if (s->slots) cudaFreeHost(s->slots);
  delete s;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Two space dimensions (include/bsde2d.h)
// ---------------------------------------------------------------------------
#include "bsde2d.cuh"
