// Batched persistent stepping of many independent 2D grids (uneven sizes,
// eps, initial states) in one launch.
//
// Work items are the warp strips of the 2D streaming stencil: (instance,
// strip, row chunk).  One step-block s advances an item by the depth the
// instance's plan gives for s (k steps, or the remainder).  A ticket is a
// pair (s, item) numbered s * n_items + item; warps of a persistent grid
// draw tickets from one atomic counter, so tickets are claimed in
// increasing s.  Before working on (s, item) a warp waits until the 3 x 3
// neighbourhood of the item (the items whose outputs its halo reads, and
// whose reads of the buffer it is about to overwrite must be finished) has
// completed step-block s-1; every waited-on ticket has a smaller number and
// is held by a resident warp that only waits on smaller numbers, so the
// waits always end while the grid is fully resident (the host sizes it from
// the occupancy).  Each wait is bounded; on expiry the warp records
// AC_ERR_TIMEOUT and stops.
//
// Memory ordering: the item's stores are made visible with a fence and a
// release store of its progress counter; the consumer acquires the counters
// and then fences the async proxy before its TMA loads read that data.
#pragma once

#include "batch_types.h"
#include "stream2d.cuh"

namespace ac {

static_assert(kBatchBoxRows == kS2Rows, "batch tensor maps use the 2D kernel's box");

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait until *p >= target.
__device__ __forceinline__ bool wait_at_least(const int *p, int target, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (ld_acquire(p) >= target) return true;
    __nanosleep(128);
  }
  return false;
}

template <typename T, int D, int VPL>
__device__ __forceinline__ bool batch_item(const S2Ring<T> &ring, uint32_t &u, const CUtensorMap *map,
                                           T *dst, const S2Item &si, const BInst &in, int *status) {
  using C = typename Traits<T>::C;
  if (in.fastx)
    return s2_item<T, D, true, VPL>(ring.smem, ring.bars, u, map, dst, si, (C)in.alpha, (C)in.beta, status);
  return s2_item<T, D, false, VPL>(ring.smem, ring.bars, u, map, dst, si, (C)in.alpha, (C)in.beta, status);
}

// VPL: 16-byte vectors per lane of every strip (the storage type's default,
// or 2 for the 8-cell FP32 strips, depths up to kBatchKMaxWide).
template <typename T, int VPL>
__global__ void __launch_bounds__(kS2Warps * 32, 1)
    batch2d_k(const BInst *__restrict__ insts, const BItem *__restrict__ items, int n_items,
              const CUtensorMap *__restrict__ maps, int *progress,
              unsigned long long *ticket_counter, long long total_tickets, int *status,
              uint32_t wait_limit) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const S2Ring<T> ring = s2_ring<T, 1, VPL>(smem, warp);  // ring size depends on T and VPL only
  if (lane == 0) {
    for (int s = 0; s < kS2Stages; ++s) mbar_init(&ring.bars[s], 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t u = 0;
  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket_counter, 1ull);
    tk = __shfl_sync(0xffffffffu, tk, 0);
    if ((long long)tk >= total_tickets) break;
    const int s = (int)(tk / (unsigned long long)n_items);
    const int ii = (int)(tk % (unsigned long long)n_items);
    const BItem &it = items[ii];
    const int inst = it.inst;
    const BInst in = insts[inst];
    if (s >= in.S) continue;  // this instance has finished its steps
    if (s > 0) {
      bool ok = true;
      const int dep = lane < 9 ? it.deps[lane] : -1;
      if (dep >= 0) ok = wait_at_least(progress + dep, s, wait_limit);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) report_timeout(status);
        return;  // nothing of this item was issued
      }
      if (lane == 0) {
        // observe every neighbour's release from the issuing lane, then let
        // the async proxy (TMA) see the data those releases cover
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const int dq = it.deps[q];
          if (dq >= 0) (void)ld_acquire(progress + dq);
        }
        fence_proxy_async_global();
      }
      __syncwarp();
    }
    const int d = s < in.tail_start ? in.k : in.tail[s - in.tail_start];
    const CUtensorMap *map = maps + 2 * inst + (s & 1);
    T *dst = reinterpret_cast<T *>(in.buf[(s + 1) & 1]);
    S2Item si;
    si.xs = it.xs;
    si.y0 = it.y0;
    si.y1 = it.y1;
    si.hx = in.hx;
    si.nx = in.nx;
    si.ny = in.ny;
    si.pitch = in.pitch;
    constexpr bool WIDE = VPL != S2Cfg<T>::VPL;
    bool ok = false;
    switch (d) {
      case 1: ok = batch_item<T, 1, VPL>(ring, u, map, dst, si, in, status); break;
      case 2: ok = batch_item<T, 2, VPL>(ring, u, map, dst, si, in, status); break;
      case 3: ok = batch_item<T, 3, VPL>(ring, u, map, dst, si, in, status); break;
      case 4: ok = batch_item<T, 4, VPL>(ring, u, map, dst, si, in, status); break;
      case 5:
        if constexpr (WIDE) { ok = batch_item<T, 5, VPL>(ring, u, map, dst, si, in, status); break; }
        if (lane == 0) atomicExch(status, AC_ERR_INVALID);
        return;
      case 6:
        if constexpr (WIDE) { ok = batch_item<T, 6, VPL>(ring, u, map, dst, si, in, status); break; }
        if (lane == 0) atomicExch(status, AC_ERR_INVALID);
        return;
      default: if (lane == 0) atomicExch(status, AC_ERR_INVALID); return;
    }
    if (!ok) return;
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(progress + ii, s + 1);
  }
}

template <typename T, int VPL>
struct BatchGeom {
  static constexpr int SW = S2Geom<T, 1, VPL>::SW;
  static constexpr int V = Traits<T>::V;
  static constexpr int SMEM = S2Geom<T, 1, VPL>::SMEM;
};

template <typename T, int VPL = S2Cfg<T>::VPL>
cudaError_t batch2d_launch_t(const BInst *insts, const BItem *items, int n_items,
                             const CUtensorMap *maps, int *progress,
                             unsigned long long *ticket, long long total, int *status,
                             uint32_t wait_limit, int num_sms, cudaStream_t s, int *grid_out) {
  static KernelSetup ks;
  int occ = 1;
  cudaError_t e = kernel_setup(ks, (const void *)batch2d_k<T, VPL>, kS2Warps * 32,
                               BatchGeom<T, VPL>::SMEM, &occ);
  if (e != cudaSuccess) return e;
  // every CTA of the grid must be resident at once (the waits rely on it)
  const int blocks = std::max(1, num_sms) * occ;
  if (grid_out) *grid_out = blocks;
  batch2d_k<T, VPL><<<blocks, kS2Warps * 32, BatchGeom<T, VPL>::SMEM, s>>>(
      insts, items, n_items, maps, progress, ticket, total, status, wait_limit);
  return cudaGetLastError();
}

}  // namespace ac
