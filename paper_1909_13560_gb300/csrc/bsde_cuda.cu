// C ABI of the multistep BSDE solver: plans, CUDA-graph capture of the whole
// backward loop, solve and result transfer.  Kernels: bsde_kernels.cuh.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "bsde_internal.h"
#include "bsde_kernels.cuh"

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
    cudaGetDevice(&prev_);
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

struct bsde_plan_s {
  bsde_problem prob;
  Params P;
  Layout lay;
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

template <int PREC, int DRV>
static void launch_step(bsde_plan_t *pl, cudaStream_t s, int n) {
  const Params &P = pl->P;
  const int threads = kStepTP * P.G;
  const unsigned blocks = unsigned((P.Nx + kStepTP - 1) / kStepTP);
  const int kL = P.k * P.L;
  Stats *st = reinterpret_cast<Stats *>(pl->ws + pl->lay.stats);
  if (PREC == BSDE_FP64) {
    const size_t sm = sizeof(NodeF64) * kL + sizeof(double) * 2 * P.G * kStepTP;
    k_step64<DRV><<<blocks, threads, sm, s>>>(
        P, pl->dc64, reinterpret_cast<double4_32a *>(pl->ws + pl->lay.ring64),
        reinterpret_cast<const NodeF64 *>(pl->ws + pl->lay.table), n, st);
  } else {
    const size_t sm = sizeof(NodeF32) * kL + sizeof(float) * 6 * P.G * kStepTP;
    k_step32<DRV><<<blocks, threads, sm, s>>>(
        P, pl->dc32, reinterpret_cast<float4 *>(pl->ws + pl->lay.ringA),
        reinterpret_cast<const float2 *>(pl->ws + pl->lay.ringB),
        reinterpret_cast<const NodeF32 *>(pl->ws + pl->lay.table), n, st);
  }
}

template <int PREC>
static void launch_step_any(bsde_plan_t *pl, cudaStream_t s, int n) {
  switch (pl->P.driver) {
    case BSDE_DRIVER_LIN_SIN: launch_step<PREC, BSDE_DRIVER_LIN_SIN>(pl, s, n); break;
    case BSDE_DRIVER_BS: launch_step<PREC, BSDE_DRIVER_BS>(pl, s, n); break;
    case BSDE_DRIVER_LB: launch_step<PREC, BSDE_DRIVER_LB>(pl, s, n); break;
    case BSDE_DRIVER_EX1: launch_step<PREC, BSDE_DRIVER_EX1>(pl, s, n); break;
    default: launch_step<PREC, BSDE_DRIVER_EX2>(pl, s, n); break;
  }
}

template <int PREC>
static int64_t enqueue_spline(bsde_plan_t *pl, cudaStream_t s, int slot) {
  const Params &P = pl->P;
  Ring64 r64{reinterpret_cast<double4_32a *>(pl->ws + pl->lay.ring64)};
  Ring32 r32{reinterpret_cast<float4 *>(pl->ws + pl->lay.ringA),
             reinterpret_cast<float2 *>(pl->ws + pl->lay.ringB)};
  const unsigned blocks = unsigned((P.Nx - 2 + kSplineTile - 1) / kSplineTile);
  k_spline<PREC><<<blocks, kSplineTile / kSplineChunk, 0, s>>>(P, r64, r32, slot);
  return 1;
}

// The whole solve as one stream-ordered sequence (captured into a graph).
template <int PREC>
static int64_t enqueue_solve(bsde_plan_t *pl, cudaStream_t s, bool imported) {
  const Params &P = pl->P;
  Ring64 r64{reinterpret_cast<double4_32a *>(pl->ws + pl->lay.ring64)};
  Ring32 r32{reinterpret_cast<float4 *>(pl->ws + pl->lay.ringA),
             reinterpret_cast<float2 *>(pl->ws + pl->lay.ringB)};
  Stats *st = reinterpret_cast<Stats *>(pl->ws + pl->lay.stats);
  double *sy = reinterpret_cast<double *>(pl->ws + pl->lay.stage);
  double *sz = sy + int64_t(P.k) * P.Nx;
  int64_t launches = 0;
  k_reset_stats<<<1, 32, 0, s>>>(st);
  ++launches;
  const unsigned eb = unsigned((P.Nx + 255) / 256 < 4096 ? (P.Nx + 255) / 256 : 4096);
  for (int m = 0; m < P.k; ++m) {
    if (imported)
      k_import<PREC><<<eb, 256, 0, s>>>(P, r64, r32, sy, sz, m);
    else
      k_init_closed<PREC><<<eb, 256, 0, s>>>(P, r64, r32, m);
    ++launches;
    launches += enqueue_spline<PREC>(pl, s, (P.N - m) % P.nslot);
  }
  for (int n = P.N - P.k; n >= 0; --n) {
    launch_step_any<PREC>(pl, s, n);
    ++launches;
    launches += enqueue_spline<PREC>(pl, s, n % P.nslot);
  }
  k_readout<PREC><<<1, 32, 0, s>>>(P, r64, r32, 0, st);
  k_export<PREC><<<eb, 256, 0, s>>>(P, r64, r32, sy, sy + P.Nx, 0);
  launches += 2;
  return launches;
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
  bsde_plan_t *pl = new (std::nothrow) bsde_plan_t();
  if (!pl) return fail(BSDE_ENOMEM, "plan allocation");
  pl->prob = *p;
  pl->P = P;
  pl->lay = lay;
  cudaGetDevice(&pl->device);
  pl->ws = static_cast<unsigned char *>(dev_workspace);
  pl->ws_bytes = bytes;
  driver_coefs(P, pl->dc64, pl->dc32);
  // node table: built on the host, copied once into the workspace
  const int kL = P.k * P.L;
  NodeF64 *t64 = new (std::nothrow) NodeF64[kL];
  NodeF32 *t32 = new (std::nothrow) NodeF32[kL];
  if (!t64 || !t32) {
    delete[] t64;
    delete[] t32;
    delete pl;
    return fail(BSDE_ENOMEM, "table allocation");
  }
  build_tables(pl->P, t64, t32);
  cudaError_t e;
  if (P.precision == BSDE_FP64)
    e = cudaMemcpy(pl->ws + lay.table, t64, sizeof(NodeF64) * kL, cudaMemcpyHostToDevice);
  else
    e = cudaMemcpy(pl->ws + lay.table, t32, sizeof(NodeF32) * kL, cudaMemcpyHostToDevice);
  delete[] t64;
  delete[] t32;
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
    if (pl->P.precision == BSDE_FP64) launch_step_any<BSDE_FP64>(pl, s, n);
    else launch_step_any<BSDE_FP32C>(pl, s, n);
  }
  if (parts & 2) {
    if (pl->P.precision == BSDE_FP64) enqueue_spline<BSDE_FP64>(pl, s, n % pl->P.nslot);
    else enqueue_spline<BSDE_FP32C>(pl, s, n % pl->P.nslot);
  }
  BSDE_CUDA_TRY(cudaGetLastError());
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
  // kernels in one solve (identical for both starts)
  const Params &P = pl->P;
  return 1 + int64_t(P.k) * 2 + int64_t(P.N - P.k + 1) * 2 + 2;
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

static int noalloc_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(BSDE_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
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
  // the plan lives on this stack frame: no host or device allocation
  bsde_plan_t pl{};
  if (fill_params(*p, pl.P)) return fail(BSDE_EINVAL, "invalid problem");
  pl.lay = layout_for(*p);
  if (pl.lay.total > BSDE_NOALLOC_MAX_BYTES)
    return fail(BSDE_ENOSPC, "problem needs " + std::to_string(pl.lay.total) +
                                 " bytes of workspace; the no-allocation workspace holds " +
                                 std::to_string(size_t(BSDE_NOALLOC_MAX_BYTES)));
  pl.prob = *p;
  cudaGetDevice(&pl.device);
  int rc = noalloc_address(pl.device, &pl.ws);
  if (rc) return rc;
  pl.ws_bytes = BSDE_NOALLOC_MAX_BYTES;
  driver_coefs(pl.P, pl.dc64, pl.dc32);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Params &P = pl.P;
  const int kL = P.k * P.L;
  NodeF64 t64[kMaxK * kMaxL];
  NodeF32 t32[kMaxK * kMaxL];
  build_tables(pl.P, t64, t32);
  if (P.precision == BSDE_FP64)
    BSDE_CUDA_TRY(cudaMemcpyAsync(pl.ws + pl.lay.table, t64, sizeof(NodeF64) * kL,
                                  cudaMemcpyHostToDevice, s));
  else
    BSDE_CUDA_TRY(cudaMemcpyAsync(pl.ws + pl.lay.table, t32, sizeof(NodeF32) * kL,
                                  cudaMemcpyHostToDevice, s));
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
  Stats st{};
  BSDE_CUDA_TRY(cudaMemcpyAsync(&st, pl.ws + pl.lay.stats, sizeof(Stats),
                                cudaMemcpyDeviceToHost, s));
  BSDE_CUDA_TRY(cudaStreamSynchronize(s));
  if (!result) return BSDE_OK;
  pl.host_stats = &st;
  return fill_result(&pl, result);
}
