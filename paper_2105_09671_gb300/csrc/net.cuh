// Learned 16-step jump network: shapes, parameter layout and index helpers
// shared by its kernels (k_net.cu) and its C-ABI layer (ac_net.cu).
//
// Network (2D; 3D replaces 3x3 by 3x3x3, T = 3^d taps):
//   z1 = conv(phi, W1) + b1, a1 = gelu(z1)               1 -> 32 channels
//   zl = conv(a_{l-1}, Wl) + bl, al = gelu(zl)            32 -> 32, l = 2..5
//   z6 = conv(a5, W6) + b6                                32 -> 1
//   phi_hat = phi + s * z6
// conv uses replicate padding (the zero-Neumann ghost of Section 2); gelu is
// the tanh form.  Parameters (FP32, flat): for each layer W[t][ci][co] then
// b[co]; tap t enumerates offsets (-1, 0, 1)^d with the last axis (x)
// fastest.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace ac {

constexpr int kNetC = 32;       // hidden channels
constexpr int kNetLayers = 6;

__host__ __device__ constexpr int net_taps(int ndim) { return ndim == 3 ? 27 : 9; }

struct NetShape {
  int ndim;
  int batch;
  int nx, ny, nz;  // nz = 1 in 2D
  // padded extents: +2 on every spatial axis of the grid's dimension
  __host__ __device__ int px() const { return nx + 2; }
  __host__ __device__ int py() const { return ny + 2; }
  __host__ __device__ int pz() const { return ndim == 3 ? nz + 2 : 1; }
  __host__ __device__ int64_t cells() const { return (int64_t)batch * nz * ny * nx; }
  __host__ __device__ int64_t padded_cells() const { return (int64_t)batch * pz() * py() * px(); }
  // linear index of cell (b, z, y, x) and of padded cell (b, zp, yp, xp)
  __host__ __device__ int64_t u(int b, int z, int y, int x) const {
    return (((int64_t)b * nz + z) * ny + y) * nx + x;
  }
  __host__ __device__ int64_t p(int b, int zp, int yp, int xp) const {
    return (((int64_t)b * pz() + zp) * py() + yp) * px() + xp;
  }
  // padded index of the cell (b, z, y, x) shifted by (oz, oy, ox)
  __host__ __device__ int64_t ps(int b, int z, int y, int x, int oz, int oy, int ox) const {
    return p(b, ndim == 3 ? z + 1 + oz : 0, y + 1 + oy, x + 1 + ox);
  }
};

// Tap t -> offsets, x fastest: 2D t = (oy+1)*3 + (ox+1); 3D adds (oz+1)*9.
__host__ __device__ inline void net_tap(int ndim, int t, int &oz, int &oy, int &ox) {
  ox = t % 3 - 1;
  oy = (t / 3) % 3 - 1;
  oz = ndim == 3 ? t / 9 - 1 : 0;
}

// Parameter offsets (in floats) inside the flat vector.
struct NetLayout {
  int ndim, T;
  int64_t w[kNetLayers], b[kNetLayers], total;
  __host__ __device__ static int cin(int l) { return l == 0 ? 1 : kNetC; }
  __host__ __device__ static int cout(int l) { return l == kNetLayers - 1 ? 1 : kNetC; }
};

inline NetLayout net_layout(int ndim) {
  NetLayout L;
  L.ndim = ndim;
  L.T = net_taps(ndim);
  int64_t off = 0;
  for (int l = 0; l < kNetLayers; ++l) {
    L.w[l] = off;
    off += (int64_t)L.T * NetLayout::cin(l) * NetLayout::cout(l);
    L.b[l] = off;
    off += NetLayout::cout(l);
  }
  L.total = off;
  return L;
}

typedef __nv_bfloat16 bf16;

// Device buffers of one network (parameters, optimiser state, packed BF16
// weights) and of one batch shape (activations, pre-activations, gradients).
struct NetBuffers {
  NetLayout layout;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wf = nullptr, *wd = nullptr;  // B operands of layers 1..4 (forward, data gradient)
  bf16 *a[5] = {};                    // padded activations (inference uses a[0], a[1])
  bf16 *z[5] = {};                    // pre-activations (training)
  bf16 *gz[5] = {};                   // padded gradients wrt z (zero ghost ring)
  float *raw = nullptr;               // [cells][32] FP32 scratch of the data gradient
  float *g6 = nullptr;                // [cells] gradient wrt the last pre-activation
  double *loss = nullptr;             // sum of squared scaled errors
  int *status = nullptr;
};

cudaError_t net_forward(const NetBuffers &nb, const NetShape &sh, const float *phi, float scale,
                        float *phihat, const float *target, bool train, int num_sms, cudaStream_t s);
cudaError_t net_backward(const NetBuffers &nb, const NetShape &sh, const float *phi, int num_sms,
                         cudaStream_t s);
cudaError_t net_pack(const NetBuffers &nb, cudaStream_t s);
// One 32 -> 32 tensor-core convolution over padded activations `in` (mode 0:
// forward epilogue into zout / outpad; mode 1: raw FP32 into outraw).
cudaError_t net_conv_rows(int mode, const bf16 *in, const bf16 *Wx, const float *bias,
                          const NetShape &sh, bf16 *zout, bf16 *outpad, float *outraw, int *status,
                          int num_sms, cudaStream_t s);
cudaError_t net_adam(const NetBuffers &nb, float lr, float b1, float b2, float eps, int step,
                     cudaStream_t s);

// BF16 packing of 8 FP32 values into one 16-byte word and back.
__device__ __forceinline__ uint4 pack8_bf16(const float *v) {
  uint4 u;
  __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
  return u;
}
__device__ __forceinline__ void unpack8_bf16(const uint4 &u, float *v) {
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(h[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

// Store one cell's 32 activations at its padded position and at the ghost
// copies it stands for (replicate padding: a boundary cell is also its
// outside neighbour).
template <int NDIM>
__device__ __forceinline__ void store_replicated(bf16 *outpad, const NetShape &sh, int b, int z,
                                                 int y, int x, const float *a) {
  uint4 w[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) w[c] = pack8_bf16(a + 8 * c);
  int xs[3], ys[3], zs[3];
  int nxs = 0, nys = 0, nzs = 0;
  xs[nxs++] = x + 1;
  if (x == 0) xs[nxs++] = 0;
  if (x == sh.nx - 1) xs[nxs++] = sh.nx + 1;
  ys[nys++] = y + 1;
  if (y == 0) ys[nys++] = 0;
  if (y == sh.ny - 1) ys[nys++] = sh.ny + 1;
  if (NDIM == 3) {
    zs[nzs++] = z + 1;
    if (z == 0) zs[nzs++] = 0;
    if (z == sh.nz - 1) zs[nzs++] = sh.nz + 1;
  } else {
    zs[nzs++] = 0;
  }
  for (int iz = 0; iz < nzs; ++iz)
    for (int iy = 0; iy < nys; ++iy)
      for (int ix = 0; ix < nxs; ++ix) {
        uint4 *dst = reinterpret_cast<uint4 *>(outpad + sh.p(b, zs[iz], ys[iy], xs[ix]) * kNetC);
#pragma unroll
        for (int c = 0; c < 4; ++c) dst[c] = w[c];
      }
}

// The forward passes' GELU (tanh form) with the hardware tanh
// approximation (tanh.approx.f32, relative error about 2^-11, below the BF16
// rounding of the stored activation).
__device__ __forceinline__ float net_gelu_fast(float x) {
  const float k = 0.7978845608028654f;
  const float u = k * fmaf(0.044715f * x, x * x, x);
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return 0.5f * x * (1.0f + t);
}
// Its derivative for the backward passes (accurate tanh, FP32).
__device__ __forceinline__ float net_gelu_grad(float x) {
  const float k = 0.7978845608028654f;
  const float u = k * fmaf(0.044715f * x, x * x, x);
  const float t = tanhf(u);
  return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * k * fmaf(3.0f * 0.044715f, x * x, 1.0f);
}

}  // namespace ac
