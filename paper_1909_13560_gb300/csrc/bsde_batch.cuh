// Batched solves: many independent problems of uneven Nx, N, k and driver in
// one persistent launch (FP32C).  Included once, by bsde_cuda.cu.
//
// A thread-block cluster takes the next problem from a device queue (problems
// ordered by decreasing work, so the longest start first) and its CTAs share
// the problem level by level: the step tiles and spline tiles of a level are
// dealt round-robin over the cluster's CTAs, with a cluster barrier (a
// hardware barrier: no spin loop) between the step phase and the spline phase
// and between levels.  Clusters never wait for one another, so the launch
// needs no co-residency guarantee; the grid is sized to the clusters that fit
// on the GPU at once and they drain the queue.
#pragma once

#include <cooperative_groups.h>

namespace bsde {

namespace cg = cooperative_groups;

// Per-problem descriptor in the batch workspace.
struct alignas(16) InstDesc {
  Params P;
  DrvC<float> dc32;
  int64_t ringA, ringB, ptable;  // byte offsets in the batch workspace
  int64_t pad;
};

constexpr int kBatchThreads = kStepTP * 6;  // grouped tiles: up to six groups per point
// flat tiles (one point per thread): 256-point tiles divide the power-of-two
// grids of a batch evenly, and three such CTAs fit an SM
constexpr int kBatchFlatThreads = 256;

// The spline of a level runs as in a single solve's warp-tiled kernel: the
// cluster's first CTA takes the first tile (the exact serial head; shared
// memory below), and every warp of the cluster takes warp tiles in turn.
struct alignas(16) BatchSmem {
  InstDesc D;
  PairF32 tab[kMaxK * (kMaxL / 2)];
  float part[kPartArrays * kMaxGroups * kStepTP];
  float sr[2][spline_span<BSDE_FP32C>(kSplHeadTS)];
  float sg[2][spline_span<BSDE_FP32C>(kSplHeadTS)];
  float sid[kInvPivots];
  int inst;
};

// The spline of the level in `slot` by the cluster's CTAs (every thread of
// every CTA calls it; the caller separates it from the step phases by a
// cluster barrier).  NT: the first tile's thread count (<= blockDim.x).
template <int NT>
__device__ __forceinline__ void batch_spline(BatchSmem &sm, const Params &P, Ring32 r32,
                                             int slot, int crank, int csize) {
  if (crank == 0)  // uniform over the CTA: the first tile holds CTA barriers
    spline_tile<BSDE_FP32C, kSplHeadTS, NT>(P, Ring64{nullptr}, r32, slot, 0, blockDim.x, sm.sr,
                                            sm.sg, sm.sid);
  const int wpc = int(blockDim.x) / 32, nw = spline_warp_tiles(P.Nx);
  for (int wt = crank * wpc + int(threadIdx.x >> 5); wt < nw; wt += csize * wpc)
    spline_warp_tile(P, r32, slot, wt);
}

__global__ void k_batch_reset(int *queue, Stats *stats, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *queue = 0;
  if (i < count) {
    stats[i].y0 = 0.0;
    stats[i].z0 = 0.0;
    stats[i].resid_bits = 0ull;
    stats[i].iters_max = 0;
    stats[i].nonconv = 0;
    stats[i].timeout = 0;
  }
}

// FLAT: the step-tile form (see below), a template parameter so that each
// form's kernel gets its own register allocation.  Level loads go through L1
// (ldl): the ring slots a CTA reads were written by the cluster's CTAs before
// the cluster barrier that ends the previous phase, whose release/acquire
// semantics make them visible to those loads.  A node's right-end record is
// the neighbouring lane's left-end record, so the loads hit L1.
template <int DRV, bool FLAT>
__device__ void batch_instance(BatchSmem &sm, unsigned char *ws, Stats *st,
                               cg::cluster_group &cl) {
  const Params &P = sm.D.P;
  const int crank = int(cl.block_rank()), csize = int(cl.num_blocks());
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr int kNT = FLAT ? kBatchFlatThreads : kBatchThreads;  // blockDim.x >= kNT
  float4 *ringA = reinterpret_cast<float4 *>(ws + sm.D.ringA);

  Ring64 r64{nullptr};
  const Ring32 r32 = ring32(ringA, ws + sm.D.ringB, P);

  // the k initial levels and their splines
  for (int m = 0; m < P.k; ++m)
    for (int64_t i = int64_t(crank) * nt + tid; i < P.Nx; i += int64_t(csize) * nt)
      init_point<BSDE_FP32C>(P, r64, r32, m, i);
  cl.sync();
  for (int m = 0; m < P.k; ++m) {
    batch_spline<kNT>(sm, P, r32, (P.N - m) % P.nslot, crank, csize);
    __syncthreads();  // CTA 0's shared-memory tile is reused by the next level
  }
  cl.sync();

  // the backward loop: step tiles, barrier, spline tiles, barrier.  Step
  // tiles are grouped (kStepTP points x G groups of threads, partial sums in
  // shared memory, a barrier per tile) or flat (one point per thread, every
  // group in turn, no barrier)
  const int tw = FLAT ? nt : kStepTP;
  const int ntiles = int((P.Nx + tw - 1) / tw);
  for (int n = P.N - P.k; n >= 0; --n) {
    if constexpr (FLAT) {
      for (int t = crank; t < ntiles; t += csize)
        step_tile32f<DRV>(P, sm.D.dc32, r32, sm.tab, n, t * tw, st);
    } else {
      for (int t = crank; t < ntiles; t += csize) {
        step_tile32<DRV>(P, sm.D.dc32, r32, sm.tab, sm.part, n, t * kStepTP, st);
        __syncthreads();
      }
    }
    cl.sync();
    batch_spline<kNT>(sm, P, r32, n % P.nslot, crank, csize);
    cl.sync();
  }
  if (crank == 0 && tid == 0) {
    double ay, az;
    readout_values<BSDE_FP32C>(P, r64, r32, 0, ay, az);
    st->y0 = ay;
    st->z0 = az;
  }
}

template <bool FLAT>
__global__ void __launch_bounds__(FLAT ? kBatchFlatThreads : kBatchThreads, FLAT ? 3 : 2)
    k_batch32(const InstDesc *__restrict__ descs, const int *__restrict__ order, int count,
              int *queue, unsigned char *ws, Stats *stats) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  BatchSmem &sm = *reinterpret_cast<BatchSmem *>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  while (true) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) sm.inst = atomicAdd(queue, 1);
    cl.sync();
    const int q = *cl.map_shared_rank(&sm.inst, 0);
    cl.sync();  // every CTA has read rank 0's value before it changes
    if (q >= count) break;
    const int id = order[q];
    {
      const int4 *src = reinterpret_cast<const int4 *>(descs + id);
      int4 *dst = reinterpret_cast<int4 *>(&sm.D);
      for (int t = threadIdx.x; t < int(sizeof(InstDesc) / 16); t += blockDim.x) dst[t] = src[t];
    }
    __syncthreads();
    {
      const float4 *src = reinterpret_cast<const float4 *>(ws + sm.D.ptable);
      float4 *dst = reinterpret_cast<float4 *>(sm.tab);
      const int n4 = sm.D.P.k * sm.D.P.Lp * kPairVec;
      for (int t = threadIdx.x; t < n4; t += blockDim.x) dst[t] = src[t];
      if (threadIdx.x < kInvPivots) sm.sid[threadIdx.x] = float(sm.D.P.invd[threadIdx.x]);
    }
    __syncthreads();
    switch (sm.D.P.driver) {
      case BSDE_DRIVER_LIN_SIN: batch_instance<BSDE_DRIVER_LIN_SIN, FLAT>(sm, ws, stats + id, cl); break;
      case BSDE_DRIVER_BS: batch_instance<BSDE_DRIVER_BS, FLAT>(sm, ws, stats + id, cl); break;
      case BSDE_DRIVER_LB: batch_instance<BSDE_DRIVER_LB, FLAT>(sm, ws, stats + id, cl); break;
      case BSDE_DRIVER_EX1: batch_instance<BSDE_DRIVER_EX1, FLAT>(sm, ws, stats + id, cl); break;
      default: batch_instance<BSDE_DRIVER_EX2, FLAT>(sm, ws, stats + id, cl); break;
    }
  }
}

}  // namespace bsde
