// Continuous-batching server: a persistent kernel that solves pricing
// requests as the host publishes them.  Included once, by bsde_cuda.cu.
//
// Host side (bsde_cuda.cu): requests are admitted by device-memory footprint
// into a caller-owned pool and a free slot; the slot's descriptor and pair
// table are written into host-mapped memory and the slot index is published
// in a request ring (a release store of the ring tail).  Device side: each
// cluster of the persistent grid claims the next ring position from a device
// counter, waits (bounded) until the host has published it, copies the
// problem into shared memory, solves it with the batch kernel's per-level
// code, writes the result into the slot's mapped result area and raises the
// slot's done flag.  Requests that arrive while others run are picked up by
// the next free cluster, so their work overlaps on the device.
#pragma once

namespace bsde {

constexpr int kServerRing = 1 << 16;  // request ring positions (indices wrap)

// Host-mapped control block.  The first line is written by the host, the
// second by the device.
struct alignas(64) ServerCtl {
  uint32_t req_tail;   // requests published so far
  uint32_t shutdown;   // nonzero: clusters exit once they find no request
  uint32_t pad[14];
  uint32_t stopped;    // set by the device: a cluster's idle limit passed and
                       // every cluster leaves after its current request
  uint32_t pad2[15];
  int32_t req_slot[kServerRing];
};

// Host-mapped per-slot area.
struct alignas(64) ServerSlot {
  InstDesc D;
  PairF32 tab[kMaxK * (kMaxL / 2)];
  Stats result;        // written by the device before done
  uint32_t done;       // 1 once result is written
  uint32_t pad[15];
};

// Device-side state in the workspace.
struct alignas(64) ServerDev {
  uint32_t req_head;   // next ring position to claim
  int32_t error;       // a bounded wait ran out (ms of idle wait exceeded)
  uint32_t pad[14];
};

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t *p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(kBatchFlatThreads, 3)
    k_server32(ServerCtl *ctl, ServerSlot *slots, ServerDev *dev, Stats *dstats,
               unsigned char *pool, unsigned long long idle_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  BatchSmem &sm = *reinterpret_cast<BatchSmem *>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  while (true) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      const uint32_t pos = atomicAdd(&dev->req_head, 1u);
      // wait until the host publishes ring position pos, or shuts down, or
      // the idle limit passes.  A cluster that gives up leaves pos claimed
      // and unserved, so it stops the whole server: the others leave too and
      // the host reports the requests that no cluster will serve.
      int slot = -1;
      const uint64_t t0 = global_ns();
      while (true) {
        if (ld_acquire_sys(&ctl->req_tail) > pos) {
          slot = __ldcv(&ctl->req_slot[pos % kServerRing]);
          break;
        }
        if (ld_acquire_sys(&ctl->shutdown) || ld_acquire_sys(&ctl->stopped)) break;
        if (global_ns() - t0 > idle_ns) {
          atomicExch(&dev->error, 1);
          __threadfence_system();
          st_release_sys(&ctl->stopped, 1u);
          break;
        }
        __nanosleep(2000);
      }
      sm.inst = slot;
    }
    cl.sync();
    const int slot = *cl.map_shared_rank(&sm.inst, 0);
    cl.sync();
    if (slot < 0) break;
    ServerSlot *S = slots + slot;
    // the slot lives in host memory and is rewritten between requests: read
    // it uncached
    {
      const int4 *src = reinterpret_cast<const int4 *>(&S->D);
      int4 *dst = reinterpret_cast<int4 *>(&sm.D);
      for (int t = threadIdx.x; t < int(sizeof(InstDesc) / 16); t += blockDim.x)
        dst[t] = __ldcv(src + t);
    }
    __syncthreads();
    {
      const float4 *src = reinterpret_cast<const float4 *>(S->tab);
      float4 *dst = reinterpret_cast<float4 *>(sm.tab);
      const int n4 = sm.D.P.k * sm.D.P.Lp * kPairVec;
      for (int t = threadIdx.x; t < n4; t += blockDim.x) dst[t] = __ldcv(src + t);
      if (threadIdx.x < kInvPivots) sm.sid[threadIdx.x] = float(sm.D.P.invd[threadIdx.x]);
    }
    Stats *st = dstats + slot;
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      st->y0 = 0.0;
      st->z0 = 0.0;
      st->resid_bits = 0ull;
      st->iters_max = 0;
      st->nonconv = 0;
      st->timeout = 0;
      __threadfence();
    }
    __syncthreads();
    cl.sync();
    switch (sm.D.P.driver) {
      case BSDE_DRIVER_LIN_SIN: batch_instance<BSDE_DRIVER_LIN_SIN, true>(sm, pool, st, cl); break;
      case BSDE_DRIVER_BS: batch_instance<BSDE_DRIVER_BS, true>(sm, pool, st, cl); break;
      case BSDE_DRIVER_LB: batch_instance<BSDE_DRIVER_LB, true>(sm, pool, st, cl); break;
      case BSDE_DRIVER_EX1: batch_instance<BSDE_DRIVER_EX1, true>(sm, pool, st, cl); break;
      default: batch_instance<BSDE_DRIVER_EX2, true>(sm, pool, st, cl); break;
    }
    // batch_instance ends with the readout by rank 0 after the last barrier;
    // wait for the Picard statistics of every CTA, then publish
    cl.sync();
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      // the statistics were gathered by atomics in L2: read them there
      S->result.y0 = __ldcg(&st->y0);
      S->result.z0 = __ldcg(&st->z0);
      S->result.resid_bits = __ldcg(&st->resid_bits);
      S->result.iters_max = __ldcg(&st->iters_max);
      S->result.nonconv = __ldcg(&st->nonconv);
      S->result.timeout = __ldcg(&st->timeout);
      __threadfence_system();
      st_release_sys(&S->done, 1u);
    }
  }
}

}  // namespace bsde
