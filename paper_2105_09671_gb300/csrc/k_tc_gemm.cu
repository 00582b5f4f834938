// A minimal tensor-core GEMM, D[M x 32] = A[M x K] * B[32 x K]^T with BF16
// operands and FP32 accumulation (tcgen05, one 128-row tile per CTA).  It is
// the building block of the learned stepper's convolutions, exposed so that
// the operand layouts and descriptors can be checked on their own.
#include "kernels.h"
#include "tc.cuh"

namespace ac {

__global__ void __launch_bounds__(128) tc_gemm_n32_k(const __nv_bfloat16 *__restrict__ A,
                                                     const __nv_bfloat16 *__restrict__ B,
                                                     float *__restrict__ D, int K, int *status) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int KC = K / 8;
  unsigned char *sA = sm;                    // 128 x K, canonical K-major
  unsigned char *sB = sm + 128 * K * 2;      // 32 x K, canonical K-major
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + 32 * K * 2);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * 128;

  for (int i = tid; i < 128 * KC; i += 128) {
    const int r = i / KC, c = i - r * KC;
    const uint4 v = *reinterpret_cast<const uint4 *>(A + (m0 + r) * K + c * 8);
    *reinterpret_cast<uint4 *>(sA + tc_kmajor_off(r, c * 8, KC)) = v;
  }
  for (int i = tid; i < 32 * KC; i += 128) {
    const int r = i / KC, c = i - r * KC;
    const uint4 v = *reinterpret_cast<const uint4 *>(B + (int64_t)r * K + c * 8);
    *reinterpret_cast<uint4 *>(sB + tc_kmajor_off(r, c * 8, KC)) = v;
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(slot, 32);
    tmem_relinquish();
  }
  fence_proxy_async_smem();  // generic-proxy smem writes -> tensor-core reads
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (tid == 0) {
    constexpr uint32_t idesc = tc_idesc_bf16_f32(128, 32);
    const uint32_t sbo = (uint32_t)KC * 128;  // between 8-row groups
    for (int kk = 0; kk < K / 16; ++kk) {
      const uint64_t da = tc_smem_desc(sA + kk * 256, 128, sbo);
      const uint64_t db = tc_smem_desc(sB + kk * 256, 128, sbo);
      tc_mma_bf16(tmem, da, db, idesc, kk > 0);
    }
    tc_commit(bar);
  }
  bool ok = mbar_wait_bounded(bar, 0);
  if (!ok) {
    report_timeout(status);
    mbar_wait_bounded(bar, 0);  // let the MMAs drain before freeing tensor memory
  }
  tc_fence_after();
  float v[32];
  tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
  float *drow = D + (m0 + warp * 32 + lane) * 32;
#pragma unroll
  for (int j = 0; j < 32; j += 4)
    *reinterpret_cast<float4 *>(drow + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

cudaError_t launch_tc_gemm_n32(const void *a, const void *b, float *d, int64_t m, int k, int *status,
                               cudaStream_t s) {
  const int smem = 160 * k * 2 + 16;
  static KernelSetup ks;
  int occ = 0;
  cudaError_t e = kernel_setup(ks, (const void *)tc_gemm_n32_k, 128, 160 * 512 * 2 + 16, &occ);
  if (e != cudaSuccess) return e;
  tc_gemm_n32_k<<<(unsigned)(m / 128), 128, smem, s>>>((const __nv_bfloat16 *)a,
                                                        (const __nv_bfloat16 *)b, d, k, status);
  return cudaGetLastError();
}

}  // namespace ac
