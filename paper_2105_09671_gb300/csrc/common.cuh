// Internal definitions shared by the CUDA kernels and the C-ABI layer.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ac.h"

namespace ac {

// --------------------------------------------------------------- types ----
// Storage type T -> compute type C and vector width V (elements per 16 B).
template <typename T> struct Traits;
template <> struct Traits<double> { using C = double; static constexpr int V = 2; };
template <> struct Traits<float> { using C = float; static constexpr int V = 4; };
template <> struct Traits<__half> { using C = float; static constexpr int V = 8; };

__device__ __forceinline__ double to_c(double x) { return x; }
__device__ __forceinline__ float to_c(float x) { return x; }
__device__ __forceinline__ float to_c(__half x) { return __half2float(x); }

template <typename T> __device__ __forceinline__ T from_c(typename Traits<T>::C x);
template <> __device__ __forceinline__ double from_c<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_c<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_c<__half>(float x) { return __float2half_rn(x); }

// FP64 value -> storage type with a single round-to-nearest-even.
template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ __half from_f64<__half>(double x) { return __double2half(x); }  // nearest-even

// V storage elements <-> one 16-byte word.
template <typename T>
__device__ __forceinline__ void unpack16(const uint4 &w, typename Traits<T>::C *out) {
  constexpr int V = Traits<T>::V;
  const T *e = reinterpret_cast<const T *>(&w);
#pragma unroll
  for (int i = 0; i < V; ++i) out[i] = to_c(e[i]);
}
template <typename T>
__device__ __forceinline__ uint4 pack16(const typename Traits<T>::C *in) {
  constexpr int V = Traits<T>::V;
  uint4 w;
  T *e = reinterpret_cast<T *>(&w);
#pragma unroll
  for (int i = 0; i < V; ++i) e[i] = from_c<T>(in[i]);
  return w;
}
// FP16 storage: convert in pairs (one conversion instruction per two
// values each way; rounding to nearest even as the scalar form).
template <>
__device__ __forceinline__ void unpack16<__half>(const uint4 &w, float *out) {
  const __half2 *p = reinterpret_cast<const __half2 *>(&w);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(p[i]);
    out[2 * i] = f.x;
    out[2 * i + 1] = f.y;
  }
}
template <>
__device__ __forceinline__ uint4 pack16<__half>(const float *in) {
  uint4 w;
  __half2 *p = reinterpret_cast<__half2 *>(&w);
#pragma unroll
  for (int i = 0; i < 4; ++i) p[i] = __floats2half2_rn(in[2 * i], in[2 * i + 1]);
  return w;
}

// ------------------------------------------------------------ the update --
// One explicit Euler step of Eq. (pytorchACeq) for one cell:
//   phi' = phi + beta * (nsum - 2 d phi) + alpha * (phi - phi^3),
// alpha = dt/eps^2, beta = dt/h^2, nsum = (W + E) + (S + N) [+ (B + F)] with
// clamped (replicated) neighbours at the domain faces.  phi = +-1 and 0 are
// reproduced exactly (phi - phi^3 and the Laplacian both vanish exactly).
template <typename C>
__device__ __forceinline__ C ac_update(C p, C nsum, C minus_2d, C alpha, C beta) {
  C lap = fma(minus_2d, p, nsum);
  C react = fma(-p * p, p, p);
  return fma(alpha, react, fma(beta, lap, p));
}

// ----------------------------------------------------------- parameters ---
struct GridParams {
  int64_t nx, ny, nz;
  int64_t pitch;  // elements between rows; plane stride = pitch * ny
  double alpha, beta;
  int *status;    // device error word (AC_ERR_TIMEOUT on an expired wait)
};

// ------------------------------------------------- PTX: mbarrier / TMA ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Programmatic dependent launch (a kernel launched with the programmatic
// stream serialization attribute): launch_dependents lets the next such
// kernel of the stream be scheduled once every CTA of this grid has issued it
// (or exited); wait blocks until the previous kernel of the stream has
// completed and its memory operations are visible.  Without the attribute
// both are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// One arrival (release semantics at CTA scope) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase: returns false after ~2^22 polls (each
// try_wait itself blocks for a hardware-defined interval), never hangs.
constexpr uint32_t kWaitPolls = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
// Tiled TMA loads into this CTA's shared memory; completion is signalled on
// `bar` as transaction bytes.  x must be a multiple of 16 bytes / element.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void report_timeout(int *status) {
  if (status) atomicExch(status, AC_ERR_TIMEOUT);
}

}  // namespace ac
