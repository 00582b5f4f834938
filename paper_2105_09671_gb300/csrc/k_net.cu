// Kernels of the learned 16-step jump network (layout and definition in
// net.cuh).  Activations are BF16 with FP32 accumulation.
//
// Storage: every activation a_l that feeds a convolution is kept *padded*:
// [batch][nz+2][ny+2][nx+2][32] (2D: [batch][1][ny+2][nx+2][32]) with the
// ghost ring holding the replicated boundary cell (the zero-Neumann ghost),
// written by the layer that produces a_l.  Gradients wrt pre-activations are
// kept padded with a zero ghost ring.  So every tap of every convolution
// reads an in-bounds, unclamped shifted row.
//
//   net_first_fwd     1 -> 32 channels, CUDA cores (K = 9 / 27 is too short)
//   net_conv_rows     out[p][n] = sum_t sum_c in[p+t][c] Wx[n][t][c] on the
//                     tensor cores (k_net_conv.cu: TMA row ring, tcgen05,
//                     accumulators in TMEM); forward (bias, GELU, ghost
//                     writes) and the data gradient (flipped taps,
//                     transposed weights, raw FP32 out)
//   net_dgrad_finish  adds the gradient of ghost cells to the boundary cell
//                     they copy (adjoint of replicate padding), x gelu'
//   net_wgrad_tc      dW[t][ci][co] = sum_p a[p+t][ci] g[p][co] on the
//                     tensor cores, reduced over pixels; an all-ones row
//                     gives the bias gradient
//   net_last_fwd/bwd, net_first_wgrad   the 1-channel ends, CUDA cores
//   net_adam, net_pack                  optimiser and BF16 weight layouts
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.h"
#include "net.cuh"
#include "tc.cuh"

namespace ac {

template <int NDIM>
__device__ __forceinline__ void decode_cell(const NetShape &sh, int64_t i, int &b, int &z, int &y,
                                            int &x) {
  x = (int)(i % sh.nx);
  i /= sh.nx;
  y = (int)(i % sh.ny);
  i /= sh.ny;
  z = (int)(i % sh.nz);
  b = (int)(i / sh.nz);
}

// ------------------------------------------------------------ first layer --
template <int NDIM, bool TRAIN>
__global__ void __launch_bounds__(256) net_first_fwd_k(const float *__restrict__ phi,
                                                       const float *__restrict__ params,
                                                       int64_t w_off, int64_t b_off, NetShape sh,
                                                       bf16 *__restrict__ z1, bf16 *__restrict__ a1pad) {
  constexpr int T = net_taps(NDIM);
  __shared__ __align__(16) float w[T * kNetC];
  __shared__ float bb[kNetC];
  for (int i = threadIdx.x; i < T * kNetC; i += blockDim.x) w[i] = params[w_off + i];
  if (threadIdx.x < kNetC) bb[threadIdx.x] = params[b_off + threadIdx.x];
  __syncthreads();
  const int64_t n = sh.cells();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int b, z, y, x;
    decode_cell<NDIM>(sh, i, b, z, y, x);
    float acc[kNetC];
#pragma unroll
    for (int c = 0; c < kNetC; ++c) acc[c] = bb[c];
    for (int t = 0; t < T; ++t) {
      int oz, oy, ox;
      net_tap(NDIM, t, oz, oy, ox);
      const int xx = min(max(x + ox, 0), sh.nx - 1), yy = min(max(y + oy, 0), sh.ny - 1);
      const int zz = NDIM == 3 ? min(max(z + oz, 0), sh.nz - 1) : 0;
      const float v = phi[sh.u(b, zz, yy, xx)];
#pragma unroll
      for (int c = 0; c < kNetC; c += 4) {  // 16-byte weight reads (broadcast)
        const float4 wv = *reinterpret_cast<const float4 *>(w + t * kNetC + c);
        acc[c] = fmaf(v, wv.x, acc[c]);
        acc[c + 1] = fmaf(v, wv.y, acc[c + 1]);
        acc[c + 2] = fmaf(v, wv.z, acc[c + 2]);
        acc[c + 3] = fmaf(v, wv.w, acc[c + 3]);
      }
    }
    if (TRAIN) {
      uint4 *dz = reinterpret_cast<uint4 *>(z1 + i * kNetC);
#pragma unroll
      for (int c = 0; c < 4; ++c) dz[c] = pack8_bf16(acc + 8 * c);
    }
#pragma unroll
    for (int c = 0; c < kNetC; ++c) acc[c] = net_gelu_fast(acc[c]);
    store_replicated<NDIM>(a1pad, sh, b, z, y, x, acc);
  }
}


// -------------------------------------------------- tensor-core wgrad ------
// dW[t][ci][co] += sum_p a[p + t][ci] * g[p][co] and db[co] += sum_p g[p][co]
// as a GEMM with M = T*32 (+1 all-ones row for the bias), N = 32, K = pixels,
// 64 pixels per step, split over CTAs and added to the global gradient.
template <int NDIM>
struct WgradGeom {
  static constexpr int T = net_taps(NDIM);
  static constexpr int MROWS = T * kNetC + 1;
  static constexpr int MT = (MROWS + 127) / 128;       // 128-row tiles
  static constexpr int MPAD = MT * 128;
  static constexpr int KC = 8;                          // 64 pixels = 8 chunks
  static constexpr int A_BYTES = MPAD * 64 * 2;
  static constexpr int B_BYTES = 32 * 64 * 2;
  static constexpr int TMEM_COLS = MT * 32 <= 32 ? 32 : MT * 32 <= 64 ? 64 : MT * 32 <= 128 ? 128 : 256;
  static constexpr int SMEM = A_BYTES + B_BYTES + 16;
};

template <int NDIM>
__global__ void __launch_bounds__(128) net_wgrad_tc_k(const bf16 *__restrict__ apad,
                                                      const bf16 *__restrict__ gpad, NetShape sh,
                                                      float *__restrict__ gw, float *__restrict__ gb,
                                                      int *status) {
  using Gm = WgradGeom<NDIM>;
  constexpr int T = Gm::T;
  constexpr uint32_t idesc = tc_idesc_bf16_f32(128, 32);
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char *sA = sm;
  unsigned char *sB = sm + Gm::A_BYTES;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + Gm::B_BYTES);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < Gm::A_BYTES / 16; i += 128) reinterpret_cast<uint4 *>(sA)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(slot, Gm::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  uint32_t phase = 0;
  const int64_t n = sh.cells();
  const int64_t chunks = (n + 63) / 64;
  bool first = true;
  for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
    // A: rows (t, ci) = a[p_k + t][ci]; row T*32 = 1 (valid pixel) for the bias
    for (int i = tid; i < T * 64 * 4; i += 128) {
      const int c8 = i & 3, k = (i >> 2) & 63, t = i >> 8;
      const int64_t pi = ch * 64 + k;
      float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (pi < n) {
        int b, z, y, x, oz, oy, ox;
        decode_cell<NDIM>(sh, pi, b, z, y, x);
        net_tap(NDIM, t, oz, oy, ox);
        unpack8_bf16(*reinterpret_cast<const uint4 *>(apad + sh.ps(b, z, y, x, oz, oy, ox) * kNetC + c8 * 8), v);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e)
        *reinterpret_cast<bf16 *>(sA + tc_kmajor_off(t * kNetC + c8 * 8 + e, k, Gm::KC)) = __float2bfloat16_rn(v[e]);
    }
    for (int k = tid; k < 64; k += 128)
      *reinterpret_cast<bf16 *>(sA + tc_kmajor_off(T * kNetC, k, Gm::KC)) =
          __float2bfloat16_rn(ch * 64 + k < n ? 1.0f : 0.0f);
    // B: rows co = g[p_k][co]
    for (int i = tid; i < 64 * 4; i += 128) {
      const int c8 = i & 3, k = i >> 2;
      const int64_t pi = ch * 64 + k;
      float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (pi < n) {
        int b, z, y, x;
        decode_cell<NDIM>(sh, pi, b, z, y, x);
        unpack8_bf16(*reinterpret_cast<const uint4 *>(gpad + sh.ps(b, z, y, x, 0, 0, 0) * kNetC + c8 * 8), v);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e)
        *reinterpret_cast<bf16 *>(sB + tc_kmajor_off(c8 * 8 + e, k, Gm::KC)) = __float2bfloat16_rn(v[e]);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      for (int mt = 0; mt < Gm::MT; ++mt)
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t da = tc_smem_desc(sA + mt * (16 * Gm::KC * 128) + kk * 256, 128, Gm::KC * 128);
          const uint64_t db = tc_smem_desc(sB + kk * 256, 128, Gm::KC * 128);
          tc_mma_bf16(tmem + mt * 32, da, db, idesc, !first || kk > 0);
        }
      tc_commit(bar);
    }
    if (!mbar_wait_bounded(bar, phase)) {
      report_timeout(status);
      mbar_wait_bounded(bar, phase);
    }
    phase ^= 1u;
    first = false;
    tc_fence_before();
    __syncthreads();
  }
  if (!first) {
    tc_fence_after();
    for (int mt = 0; mt < Gm::MT; ++mt) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + mt * 32, v);
      const int m = mt * 128 + warp * 32 + (tid & 31);
      if (m < T * kNetC) {
#pragma unroll
        for (int c = 0; c < 32; ++c) atomicAdd(gw + (int64_t)m * kNetC + c, v[c]);
      } else if (m == T * kNetC) {
#pragma unroll
        for (int c = 0; c < 32; ++c) atomicAdd(gb + c, v[c]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, Gm::TMEM_COLS);
}

// Cells i with clamp(i + t) == p along one axis of extent n: [lo, hi].
__device__ __forceinline__ void clamp_preimage(int p, int t, int n, int &lo, int &hi) {
  const int a = (p == 0) ? -1000000 : p;       // lower bound on i + t
  const int b2 = (p == n - 1) ? 1000000 : p;   // upper bound on i + t
  lo = max(a - t, 0);
  hi = min(b2 - t, n - 1);
}

// ------------------------------------------------------------- last layer --
// z6 = conv(a5, W6) + b6 (32 -> 1 channel) and phi_hat = phi + s z6; in
// training also the scaled residual's gradient g6 and the loss sum.  A block
// covers 32 x 8 cells of one z: the 10 x 34 padded pixels (x 3 planes in 3D)
// it reads are staged once in shared memory with coalesced 16-byte loads
// (pixel stride 80 bytes: conflict-free 16-byte reads by consecutive lanes),
// then each thread forms one cell.
constexpr int kLastTX = 32, kLastTY = 8, kLastPix = 5;  // uint4 per staged pixel (4 + pad)

template <int NDIM>
__host__ __device__ constexpr int last_smem_bytes() {
  return (NDIM == 3 ? 3 : 1) * (kLastTY + 2) * (kLastTX + 2) * kLastPix * 16 +
         net_taps(NDIM) * kNetC * 4;
}

template <int NDIM, bool TRAIN>
__global__ void __launch_bounds__(256) net_last_fwd_k(const bf16 *__restrict__ a5pad,
                                                      const float *__restrict__ params, int64_t w_off,
                                                      int64_t b_off, NetShape sh,
                                                      const float *__restrict__ phi, float scale,
                                                      float *__restrict__ phihat,
                                                      const float *__restrict__ target,
                                                      float *__restrict__ g6, double *loss_acc) {
  constexpr int T = net_taps(NDIM);
  constexpr int NZR = NDIM == 3 ? 3 : 1;
  constexpr int RW = kLastTX + 2, RH = kLastTY + 2;
  extern __shared__ __align__(16) unsigned char lsm[];
  uint4 *tile = reinterpret_cast<uint4 *>(lsm);                         // [NZR][RH][RW][kLastPix]
  float *w = reinterpret_cast<float *>(lsm + NZR * RH * RW * kLastPix * 16);  // [T][32]
  __shared__ double red[8];
  for (int i = threadIdx.x; i < T * kNetC; i += blockDim.x) w[i] = params[w_off + i];
  const float b6 = params[b_off];
  const float inv_n = 1.0f / (float)sh.cells();
  const int tiles_x = (sh.nx + kLastTX - 1) / kLastTX, tiles_y = (sh.ny + kLastTY - 1) / kLastTY;
  const int64_t items = (int64_t)sh.batch * sh.nz * tiles_y * tiles_x;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  double lsum = 0.0;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int tx = (int)(item % tiles_x);
    int64_t r = item / tiles_x;
    const int ty = (int)(r % tiles_y);
    r /= tiles_y;
    const int z = (int)(r % sh.nz), b = (int)(r / sh.nz);
    const int x0 = tx * kLastTX, y0 = ty * kLastTY;
    __syncthreads();  // the previous item's tile (and w) is complete / released
    // padded pixels (xp, yp) = (x0 + i, y0 + j), i < RW, j < RH, of planes z .. z+2
    for (int i = threadIdx.x; i < NZR * RH * RW * 4; i += blockDim.x) {
      const int c = i & 3;
      const int q = i >> 2;
      const int px = q % RW, row = (q / RW) % RH, dz = q / (RW * RH);
      const int xp = x0 + px, yp = y0 + row;
      if (xp < sh.px() && yp < sh.py())
        tile[q * kLastPix + c] = *reinterpret_cast<const uint4 *>(
            a5pad + (sh.p(b, NDIM == 3 ? z + dz : 0, yp, xp) * kNetC + c * 8));
    }
    __syncthreads();
    const int x = x0 + lane, y = y0 + wy;
    if (x < sh.nx && y < sh.ny) {
      float acc = b6;
      for (int t = 0; t < T; ++t) {
        int oz, oy, ox;
        net_tap(NDIM, t, oz, oy, ox);
        const int dz = NDIM == 3 ? oz + 1 : 0;
        const uint4 *src = tile + ((dz * RH + wy + oy + 1) * RW + lane + ox + 1) * kLastPix;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v[8];
          unpack8_bf16(src[c], v);
#pragma unroll
          for (int e = 0; e < 8; e += 4) {  // 16-byte weight reads (broadcast)
            const float4 wv = *reinterpret_cast<const float4 *>(w + t * kNetC + c * 8 + e);
            acc = fmaf(v[e], wv.x, acc);
            acc = fmaf(v[e + 1], wv.y, acc);
            acc = fmaf(v[e + 2], wv.z, acc);
            acc = fmaf(v[e + 3], wv.w, acc);
          }
        }
      }
      const int64_t i = sh.u(b, z, y, x);
      const float ph = phi[i] + scale * acc;
      phihat[i] = ph;
      if (TRAIN) {
        const float rr = (ph - target[i]) / scale;
        g6[i] = 2.0f * rr * inv_n;
        lsum += (double)rr * (double)rr;
      }
    }
  }
  if (TRAIN) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) red[wy] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s2 = 0.0;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s2 += red[w2];
      atomicAdd(loss_acc, s2);
    }
  }
}

// Warp per cell, lane = channel: gradient of the last layer (weights, bias)
// and the gradient wrt z5 (replicate-padding adjoint, x gelu'(z5)).
template <int NDIM>
__global__ void __launch_bounds__(256) net_last_bwd_k(const float *__restrict__ g6,
                                                      const float *__restrict__ params, int64_t w_off,
                                                      NetShape sh, const bf16 *__restrict__ z5,
                                                      const bf16 *__restrict__ a5pad,
                                                      bf16 *__restrict__ gz5pad,
                                                      float *__restrict__ grads, int64_t gw_off,
                                                      int64_t gb_off) {
  constexpr int T = net_taps(NDIM);
  __shared__ float w[T * kNetC];
  for (int i = threadIdx.x; i < T * kNetC; i += blockDim.x) w[i] = params[w_off + i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  float dw[T];
#pragma unroll
  for (int t = 0; t < T; ++t) dw[t] = 0.f;
  float db = 0.f;
  const int64_t n = sh.cells();
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    int b, z, y, x;
    decode_cell<NDIM>(sh, i, b, z, y, x);
    const float gp = g6[i];
    db += gp;
    float ga = 0.f;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      int oz, oy, ox;
      net_tap(NDIM, t, oz, oy, ox);
      dw[t] = fmaf(__bfloat162float(a5pad[sh.ps(b, z, y, x, oz, oy, ox) * kNetC + lane]), gp, dw[t]);
      int xl, xh, yl, yh, zl = 0, zh = 0;
      clamp_preimage(x, ox, sh.nx, xl, xh);
      clamp_preimage(y, oy, sh.ny, yl, yh);
      if (NDIM == 3) clamp_preimage(z, oz, sh.nz, zl, zh);
      float s = 0.f;
      for (int zz = zl; zz <= zh; ++zz)
        for (int yy = yl; yy <= yh; ++yy)
          for (int xx = xl; xx <= xh; ++xx) s += g6[sh.u(b, zz, yy, xx)];
      ga = fmaf(w[t * kNetC + lane], s, ga);
    }
    const float zv = __bfloat162float(z5[i * kNetC + lane]);
    gz5pad[sh.ps(b, z, y, x, 0, 0, 0) * kNetC + lane] = __float2bfloat16_rn(ga * net_gelu_grad(zv));
  }
#pragma unroll
  for (int t = 0; t < T; ++t) atomicAdd(grads + gw_off + t * kNetC + lane, dw[t]);
  if (lane == 0) atomicAdd(grads + gb_off, db);
}

// Warp per cell: g_{l-1} = (raw + ghost-cell gradients folded in) x gelu'(z_{l-1}).
// raw[p] = sum_t W[t]^T g[p - t] comes from the tensor-core pass; a boundary
// cell also receives the gradient of each ghost cell that replicates it.
template <int NDIM>
__global__ void __launch_bounds__(256) net_dgrad_finish_k(const float *__restrict__ raw,
                                                          const bf16 *__restrict__ gpad,
                                                          const float *__restrict__ params,
                                                          int64_t w_off, NetShape sh,
                                                          const bf16 *__restrict__ zprev,
                                                          bf16 *__restrict__ gprevpad) {
  constexpr int T = net_taps(NDIM);
  extern __shared__ float wsm[];  // W[t][ci][co]
  for (int i = threadIdx.x; i < T * kNetC * kNetC; i += blockDim.x) wsm[i] = params[w_off + i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t n = sh.cells();
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    int b, z, y, x;
    decode_cell<NDIM>(sh, i, b, z, y, x);
    float g = raw[i * kNetC + lane];
    const bool bx = (x == 0 || x == sh.nx - 1), by = (y == 0 || y == sh.ny - 1);
    const bool bz = NDIM == 3 && (z == 0 || z == sh.nz - 1);
    if (bx || by || bz) {
      // ghost cells q (outside the grid) with clamp(q) == p
      for (int gz = (NDIM == 3 ? -1 : 0); gz <= (NDIM == 3 ? 1 : 0); ++gz)
        for (int gy = -1; gy <= 1; ++gy)
          for (int gx = -1; gx <= 1; ++gx) {
            const int qx = x + gx, qy = y + gy, qz = z + gz;
            const bool out = qx < 0 || qx >= sh.nx || qy < 0 || qy >= sh.ny ||
                             (NDIM == 3 && (qz < 0 || qz >= sh.nz));
            if (!out) continue;
            if (min(max(qx, 0), sh.nx - 1) != x || min(max(qy, 0), sh.ny - 1) != y) continue;
            if (NDIM == 3 && min(max(qz, 0), sh.nz - 1) != z) continue;
            if (qx < -1 || qx > sh.nx || qy < -1 || qy > sh.ny) continue;
            if (NDIM == 3 && (qz < -1 || qz > sh.nz)) continue;
            // gradient of the ghost cell q: sum_t W[t][ci = lane][co] g[q - t][co]
            float acc = 0.f;
            for (int t = 0; t < T; ++t) {
              int oz, oy, ox;
              net_tap(NDIM, t, oz, oy, ox);
              const int sx = qx - ox, sy = qy - oy, sz = qz - oz;
              if (sx < 0 || sx >= sh.nx || sy < 0 || sy >= sh.ny) continue;
              if (NDIM == 3 && (sz < 0 || sz >= sh.nz)) continue;
              const float gv = __bfloat162float(gpad[sh.ps(b, NDIM == 3 ? sz : 0, sy, sx, 0, 0, 0) * kNetC + lane]);
              // lane holds g[.][co = lane]; W[t][ci = lane][co] needs all co
              for (int co = 0; co < kNetC; ++co)
                acc = fmaf(wsm[(t * kNetC + lane) * kNetC + co], __shfl_sync(0xffffffffu, gv, co), acc);
            }
            g += acc;
          }
    }
    const float zv = __bfloat162float(zprev[i * kNetC + lane]);
    gprevpad[sh.ps(b, z, y, x, 0, 0, 0) * kNetC + lane] = __float2bfloat16_rn(g * net_gelu_grad(zv));
  }
}

// Warp per cell, lane = output channel: first-layer weight and bias gradients.
template <int NDIM>
__global__ void __launch_bounds__(256) net_first_wgrad_k(const float *__restrict__ phi,
                                                         const bf16 *__restrict__ g1pad, NetShape sh,
                                                         float *__restrict__ grads, int64_t gw_off,
                                                         int64_t gb_off) {
  constexpr int T = net_taps(NDIM);
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  float dw[T];
#pragma unroll
  for (int t = 0; t < T; ++t) dw[t] = 0.f;
  float db = 0.f;
  const int64_t n = sh.cells();
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    int b, z, y, x;
    decode_cell<NDIM>(sh, i, b, z, y, x);
    const float g = __bfloat162float(g1pad[sh.ps(b, z, y, x, 0, 0, 0) * kNetC + lane]);
    db += g;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      int oz, oy, ox;
      net_tap(NDIM, t, oz, oy, ox);
      const int xx = min(max(x + ox, 0), sh.nx - 1), yy = min(max(y + oy, 0), sh.ny - 1);
      const int zz = NDIM == 3 ? min(max(z + oz, 0), sh.nz - 1) : 0;
      dw[t] = fmaf(phi[sh.u(b, zz, yy, xx)], g, dw[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < T; ++t) atomicAdd(grads + gw_off + t * kNetC + lane, dw[t]);
  atomicAdd(grads + gb_off + lane, db);
}

// ---------------------------------------------------------- optimiser -----
__global__ void net_adam_k(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// BF16 B operands of the four 32 -> 32 layers: forward Wf[l][co][t][ci] =
// W[t][ci][co] and data gradient Wd[l][ci][t][co] = W[T-1-t][ci][co] (taps
// mirrored: the transposed convolution reads p - t).
__global__ void net_pack_k(const float *__restrict__ params, int T, int64_t w0, int64_t w1,
                           int64_t w2, int64_t w3, bf16 *__restrict__ wf, bf16 *__restrict__ wd) {
  const int64_t per = (int64_t)kNetC * T * kNetC;
  const int64_t total = 4 * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / per);
    int64_t r = i % per;
    const int c = (int)(r % kNetC);
    r /= kNetC;
    const int t = (int)(r % T);
    const int nrow = (int)(r / T);
    const int64_t woff = l == 0 ? w0 : l == 1 ? w1 : l == 2 ? w2 : w3;
    // forward: row n = co, column (t, ci = c)
    wf[i] = __float2bfloat16_rn(params[woff + ((int64_t)t * kNetC + c) * kNetC + nrow]);
    // data gradient: row n = ci, column (t, co = c) from tap T-1-t
    wd[i] = __float2bfloat16_rn(params[woff + ((int64_t)(T - 1 - t) * kNetC + nrow) * kNetC + c]);
  }
}

// ------------------------------------------------------------ launchers ----
static int grid_for(int64_t n, int per_block, int num_sms) {
  return (int)std::min<int64_t>((n + per_block - 1) / per_block, (int64_t)num_sms * 16);
}

// Dynamic shared-memory limits of the kernels that need more than the
// default, once per device (thread-safe; the occupancy query is unused).
template <int NDIM>
static cudaError_t setup_attrs() {
  static KernelSetup k_last_t, k_last_f, k_wgrad, k_dfin;
  int occ = 0;
  cudaError_t e;
  e = kernel_setup(k_last_t, (const void *)net_last_fwd_k<NDIM, true>, 32, last_smem_bytes<NDIM>(), &occ);
  if (e != cudaSuccess) return e;
  e = kernel_setup(k_last_f, (const void *)net_last_fwd_k<NDIM, false>, 32, last_smem_bytes<NDIM>(), &occ);
  if (e != cudaSuccess) return e;
  e = kernel_setup(k_wgrad, (const void *)net_wgrad_tc_k<NDIM>, 32, WgradGeom<NDIM>::SMEM, &occ);
  if (e != cudaSuccess) return e;
  return kernel_setup(k_dfin, (const void *)net_dgrad_finish_k<NDIM>, 32,
                      net_taps(NDIM) * kNetC * kNetC * 4, &occ);
}

template <int NDIM>
static cudaError_t net_forward_t(const NetBuffers &nb, const NetShape &sh, const float *phi,
                                 float scale, float *phihat, const float *target, bool train,
                                 int num_sms, cudaStream_t s) {
  cudaError_t e = setup_attrs<NDIM>();
  if (e != cudaSuccess) return e;
  const NetLayout &L = nb.layout;
  const int64_t n = sh.cells();
  if (train)
    net_first_fwd_k<NDIM, true><<<grid_for(n, 256, num_sms), 256, 0, s>>>(phi, nb.params, L.w[0], L.b[0], sh, nb.z[0], nb.a[0]);
  else
    net_first_fwd_k<NDIM, false><<<grid_for(n, 256, num_sms), 256, 0, s>>>(phi, nb.params, L.w[0], L.b[0], sh, nullptr, nb.a[0]);
  const int64_t per = (int64_t)kNetC * net_taps(NDIM) * kNetC;
  for (int l = 1; l <= 4; ++l) {
    bf16 *in = nb.a[(l - 1) % (train ? 5 : 2)];
    bf16 *out = nb.a[l % (train ? 5 : 2)];
    e = net_conv_rows(0, in, nb.wf + (l - 1) * per, nb.params + L.b[l], sh,
                      train ? nb.z[l] : nullptr, out, nullptr, nb.status, num_sms, s);
    if (e != cudaSuccess) return e;
  }
  const bf16 *a5 = nb.a[4 % (train ? 5 : 2)];
  const int64_t last_items = (int64_t)sh.batch * sh.nz * ((sh.ny + kLastTY - 1) / kLastTY) *
                             ((sh.nx + kLastTX - 1) / kLastTX);
  const int last_grid = (int)std::min<int64_t>(last_items, (int64_t)num_sms * 8);
  if (train)
    net_last_fwd_k<NDIM, true><<<last_grid, 256, last_smem_bytes<NDIM>(), s>>>(a5, nb.params, L.w[5], L.b[5], sh, phi, scale, phihat, target, nb.g6, nb.loss);
  else
    net_last_fwd_k<NDIM, false><<<last_grid, 256, last_smem_bytes<NDIM>(), s>>>(a5, nb.params, L.w[5], L.b[5], sh, phi, scale, phihat, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

template <int NDIM>
static cudaError_t net_backward_t(const NetBuffers &nb, const NetShape &sh, const float *phi,
                                  int num_sms, cudaStream_t s) {
  const NetLayout &L = nb.layout;
  const int64_t n = sh.cells();
  const int warps_grid = grid_for(n, 8, num_sms);
  net_last_bwd_k<NDIM><<<warps_grid, 256, 0, s>>>(nb.g6, nb.params, L.w[5], sh, nb.z[4], nb.a[4],
                                                 nb.gz[4], nb.grads, L.w[5], L.b[5]);
  const int wgrad_grid = (int)std::min<int64_t>((n + 63) / 64, (int64_t)num_sms);
  const int64_t per = (int64_t)kNetC * net_taps(NDIM) * kNetC;
  for (int l = 4; l >= 1; --l) {
    net_wgrad_tc_k<NDIM><<<wgrad_grid, 128, WgradGeom<NDIM>::SMEM, s>>>(
        nb.a[l - 1], nb.gz[l], sh, nb.grads + L.w[l], nb.grads + L.b[l], nb.status);
    cudaError_t e = net_conv_rows(1, nb.gz[l], nb.wd + (l - 1) * per, nullptr, sh, nullptr, nullptr,
                                  nb.raw, nb.status, num_sms, s);
    if (e != cudaSuccess) return e;
    net_dgrad_finish_k<NDIM><<<warps_grid, 256, net_taps(NDIM) * kNetC * kNetC * 4, s>>>(
        nb.raw, nb.gz[l], nb.params, L.w[l], sh, nb.z[l - 1], nb.gz[l - 1]);
  }
  net_first_wgrad_k<NDIM><<<warps_grid, 256, 0, s>>>(phi, nb.gz[0], sh, nb.grads, L.w[0], L.b[0]);
  return cudaGetLastError();
}

cudaError_t net_forward(const NetBuffers &nb, const NetShape &sh, const float *phi, float scale,
                        float *phihat, const float *target, bool train, int num_sms, cudaStream_t s) {
  return sh.ndim == 3 ? net_forward_t<3>(nb, sh, phi, scale, phihat, target, train, num_sms, s)
                      : net_forward_t<2>(nb, sh, phi, scale, phihat, target, train, num_sms, s);
}

cudaError_t net_backward(const NetBuffers &nb, const NetShape &sh, const float *phi, int num_sms,
                         cudaStream_t s) {
  return sh.ndim == 3 ? net_backward_t<3>(nb, sh, phi, num_sms, s) : net_backward_t<2>(nb, sh, phi, num_sms, s);
}

cudaError_t net_pack(const NetBuffers &nb, cudaStream_t s) {
  const NetLayout &L = nb.layout;
  net_pack_k<<<256, 256, 0, s>>>(nb.params, L.T, L.w[1], L.w[2], L.w[3], L.w[4], nb.wf, nb.wd);
  return cudaGetLastError();
}

cudaError_t net_adam(const NetBuffers &nb, float lr, float b1, float b2, float eps, int step,
                     cudaStream_t s) {
  const float c1 = 1.0f / (1.0f - powf(b1, (float)step));
  const float c2 = 1.0f / (1.0f - powf(b2, (float)step));
  net_adam_k<<<256, 256, 0, s>>>(nb.params, nb.grads, nb.m, nb.v, nb.layout.total, lr, b1, b2, eps, c1, c2);
  return net_pack(nb, s);
}

}  // namespace ac
