// FP64 reductions over the field: the discrete Ginzburg-Landau energy terms,
// the phase volume and a non-finite sentinel, in one pass.
//
//   bulk = sum_cells F(phi),  F(phi) = (phi^2 - 1)^2 / 4       (Section 1)
//   grad = sum_{interior faces (a, b)} (phi_a - phi_b)^2
//   vol  = sum_cells (1 + phi) / 2
//
// The host turns these into E_h = h^d (bulk / eps^2 + grad / (2 h^2)) and
// V = h^d vol.  Sums over 1e8 cells need FP64 accumulation.  FP64 fields
// form every term in FP64.  FP32 / FP16 fields hold values that are exact in
// FP32, and GB300 runs FP32 at many times its FP64 rate, so there the terms
// are formed in float-float arithmetic (an unevaluated FP32 pair hi + lo):
// TwoSum (Knuth; Moller 1965) and the FMA form of TwoProduct (Dekker 1971;
// Ogita, Rump, Oishi 2005) give p^2 and phi_a - phi_b exactly, the squares
// keep ~46 bits, and each lane adds its terms in float-float over groups of
// kFFGroup cells before the group's sum is added in FP64 (relative error of
// the sums ~1e-15, against the FP64 oracle's ~1e-16).  The result is
// deterministic: a fixed grid of blocks each reduces a fixed set of rows in
// a fixed order, and a single block adds the per-block partials in index
// order.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "kernels.h"

namespace ac {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Error-free transformations in FP32 (every operation rounded as written).
struct FF {
  float h, l;
};
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// (h + l)^2 for |l| <= ulp(h): h^2 exactly plus 2 h l
__device__ __forceinline__ FF square_ff(float h, float l) {
  FF r = two_prod(h, h);
  r.l = __fmaf_rn(__fmul_rn(2.0f, h), l, r.l);
  return r;
}
// acc += t (t a float-float term)
__device__ __forceinline__ void add_ff(FF &acc, FF t) {
  const FF s = two_sum(acc.h, t.h);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, t.l));
}
constexpr int kFFGroup = 16;

template <typename T>
__global__ void __launch_bounds__(256) observe_partial(const T *__restrict__ phi, GridParams g,
                                                       double *__restrict__ partials) {
  constexpr int kWarps = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double bulk = 0.0, grad = 0.0, vol = 0.0, bad = 0.0;
  const int64_t rows = g.ny * g.nz;
  const int64_t plane = g.pitch * g.ny;
  // each warp takes whole rows, rows strided over all warps of the grid
  for (int64_t r = (int64_t)blockIdx.x * kWarps + warp; r < rows;
       r += (int64_t)gridDim.x * kWarps) {
    const int64_t j = r % g.ny, k = r / g.ny;
    const T *row = phi + k * plane + j * g.pitch;
    const bool has_up = j + 1 < g.ny, has_front = k + 1 < g.nz;
    if constexpr (std::is_same_v<T, double>) {
      for (int64_t i = lane; i < g.nx; i += 32) {
        const double p = row[i];
        if (!isfinite(p)) bad += 1.0;
        const double q = p * p - 1.0;
        bulk += 0.25 * q * q;
        vol += 0.5 * (1.0 + p);
        if (i + 1 < g.nx) { double d = row[i + 1] - p; grad += d * d; }
        if (has_up) { double d = row[i + g.pitch] - p; grad += d * d; }
        if (has_front) { double d = row[i + plane] - p; grad += d * d; }
      }
    } else {
      for (int64_t i0 = lane; i0 < g.nx; i0 += 32 * kFFGroup) {
        FF b{0.f, 0.f}, gr{0.f, 0.f}, sp{0.f, 0.f};
        int cnt = 0;
#pragma unroll 4
        for (int u = 0; u < kFFGroup; ++u) {
          const int64_t i = i0 + 32 * u;
          if (i >= g.nx) break;
          const float p = to_c(row[i]);
          if (!isfinite(p)) bad += 1.0;
          ++cnt;
          // (p^2 - 1)^2: p^2 = p2.h + p2.l exactly, q = p^2 - 1 to ~48 bits
          const FF p2 = two_prod(p, p);
          FF q = two_sum(p2.h, -1.0f);
          q.l = __fadd_rn(q.l, p2.l);
          add_ff(b, square_ff(q.h, q.l));
          add_ff(sp, FF{p, 0.f});
          // (phi_a - p)^2 over the faces to the +x, +y, +z neighbours
          if (i + 1 < g.nx) {
            const FF d = two_sum(to_c(row[i + 1]), -p);
            add_ff(gr, square_ff(d.h, d.l));
          }
          if (has_up) {
            const FF d = two_sum(to_c(row[i + g.pitch]), -p);
            add_ff(gr, square_ff(d.h, d.l));
          }
          if (has_front) {
            const FF d = two_sum(to_c(row[i + plane]), -p);
            add_ff(gr, square_ff(d.h, d.l));
          }
        }
        bulk += 0.25 * ((double)b.h + (double)b.l);
        grad += (double)gr.h + (double)gr.l;
        vol += 0.5 * (double)cnt + 0.5 * ((double)sp.h + (double)sp.l);
      }
    }
  }
  __shared__ double red[4][kWarps];
  bulk = warp_sum(bulk); grad = warp_sum(grad); vol = warp_sum(vol); bad = warp_sum(bad);
  if (lane == 0) { red[0][warp] = bulk; red[1][warp] = grad; red[2][warp] = vol; red[3][warp] = bad; }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += red[threadIdx.x][w];
    partials[(int64_t)blockIdx.x * 4 + threadIdx.x] = s;
  }
}

// One block of 128 threads: thread t adds partials t, t+128, ... in order,
// then a fixed tree over the 128 thread sums.
__global__ void __launch_bounds__(128) observe_final(const double *__restrict__ partials, int nb,
                                                     double *__restrict__ out) {
  __shared__ double s[4][128];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += 128)
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] += partials[(int64_t)b * 4 + q];
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = s[threadIdx.x][0];
}

template <typename T>
static cudaError_t observe_t(const GridParams &g, const void *phi, double *partials, double *out,
                             cudaStream_t s) {
  observe_partial<T><<<kReduceBlocks, 256, 0, s>>>((const T *)phi, g, partials);
  observe_final<<<1, 128, 0, s>>>(partials, kReduceBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_observe(int dtype, const GridParams &g, const void *phi, double *partials,
                           double *out, cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return observe_t<double>(g, phi, partials, out, s);
    case AC_F32: return observe_t<float>(g, phi, partials, out, s);
    case AC_F16S: return observe_t<__half>(g, phi, partials, out, s);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------- allocation-free variant --
// ac_observe_noalloc (see include/ac.h) runs the same per-block partial-sum
// kernel, but over a grid of one block per kNoAllocRowsPerBlock rows, with
// its partial sums in the fixed array below instead of a buffer from
// ac_create.  The array is a module global: every GPU that loads the library
// holds its 512 KiB until the process exits, and all calls on a device share
// it.  Each call writes every partial slot it later reads, so nothing in it
// has to start at zero; two calls that overlap on the GPU (e.g. on different
// streams) would overwrite each other's partials.

constexpr int kNoAllocMaxBlocks = 16384;
constexpr int kNoAllocRowsPerBlock = 64;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 4];

// Sums the partials in a fixed order (as observe_final) and forms the
// observables on the device: out[0] = E_h, out[1] = V, out[2] = non-finite count.
__global__ void __launch_bounds__(128) observe_final_noalloc(const double *__restrict__ partials,
                                                             int nb, double hd, double inv_eps2,
                                                             double half_inv_h2,
                                                             double *__restrict__ out) {
  __shared__ double s[4][128];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += 128)
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] += partials[(int64_t)b * 4 + q];
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = hd * (s[0][0] * inv_eps2 + s[1][0] * half_inv_h2);
    out[1] = hd * s[2][0];
    out[2] = s[3][0];
  }
}

// Device address of g_noalloc_partials, looked up once per device (with that
// device current) on the first call that uses it.
static double *noalloc_scratch(int device, cudaError_t *err) {
  static std::mutex mu;
  static double *addr[64] = {nullptr};
  std::lock_guard<std::mutex> lk(mu);
  if (device < 0 || device >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!addr[device]) {
    void *p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (*err != cudaSuccess) return nullptr;
    addr[device] = static_cast<double *>(p);
  }
  *err = cudaSuccess;
  return addr[device];
}

int64_t observe_noalloc_max_rows() { return (int64_t)kNoAllocMaxBlocks * kNoAllocRowsPerBlock; }

cudaError_t launch_observe_noalloc(int dtype, const GridParams &g, const void *phi, double hd,
                                   double eps, double h, double *out_dev, cudaStream_t s) {
  const int64_t rows = g.ny * g.nz;
  if (rows > observe_noalloc_max_rows()) return cudaErrorInvalidValue;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return e;
  double *scratch = noalloc_scratch(device, &e);
  if (!scratch) return e;
  const int nb = (int)std::max<int64_t>(1, (rows + kNoAllocRowsPerBlock - 1) / kNoAllocRowsPerBlock);
  switch (dtype) {
    case AC_F64: observe_partial<double><<<nb, 256, 0, s>>>((const double *)phi, g, scratch); break;
    case AC_F32: observe_partial<float><<<nb, 256, 0, s>>>((const float *)phi, g, scratch); break;
    case AC_F16S: observe_partial<__half><<<nb, 256, 0, s>>>((const __half *)phi, g, scratch); break;
    default: return cudaErrorInvalidValue;
  }
  observe_final_noalloc<<<1, 128, 0, s>>>(scratch, nb, hd, 1.0 / (eps * eps), 0.5 / (h * h), out_dev);
  return cudaGetLastError();
}

}  // namespace ac

namespace ac {

// Guard quantities of a learned jump phi -> phi_hat over n Euler steps:
//   out[0] = max |phi_hat|,
//   out[1] = max |phi_hat - phi - n dt RHS(phi)|,
// with dt RHS(phi) = beta (nsum - 2d phi) + alpha (phi - phi^3) the increment
// of one explicit Euler step of Eq. (pytorchACeq) (clamped neighbours).
// FP32 inputs with pitch == nx; maxima are formed on the absolute values'
// bit patterns (non-negative floats order as unsigned integers).
__global__ void __launch_bounds__(256) guard_kernel(const float *__restrict__ phi,
                                                    const float *__restrict__ phat, GridParams g,
                                                    int ndim, float nsteps,
                                                    unsigned int *__restrict__ out) {
  float mabs = 0.f, mres = 0.f;
  const int64_t n = g.nx * g.ny * g.nz;
  const float a = (float)g.alpha, b = (float)g.beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % g.nx, r = i / g.nx, y = r % g.ny, z = r / g.ny;
    const float p = phi[i];
    float s = phi[i - x + (x > 0 ? x - 1 : 0)] + phi[i - x + (x + 1 < g.nx ? x + 1 : x)];
    s += phi[i + ((y > 0 ? y - 1 : 0) - y) * g.nx] + phi[i + ((y + 1 < g.ny ? y + 1 : y) - y) * g.nx];
    if (ndim == 3)
      s += phi[i + ((z > 0 ? z - 1 : 0) - z) * g.nx * g.ny] +
           phi[i + ((z + 1 < g.nz ? z + 1 : z) - z) * g.nx * g.ny];
    const float inc = b * (s - 2.0f * ndim * p) + a * (p - p * p * p);
    const float q = phat[i];
    mabs = fmaxf(mabs, fabsf(q));
    mres = fmaxf(mres, fabsf(q - p - nsteps * inc));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mabs = fmaxf(mabs, __shfl_xor_sync(0xffffffffu, mabs, o));
    mres = fmaxf(mres, __shfl_xor_sync(0xffffffffu, mres, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __float_as_uint(mabs));
    atomicMax(out + 1, __float_as_uint(mres));
  }
}

cudaError_t launch_guard(const float *phi, const float *phat, const GridParams &g, int ndim,
                         int nsteps, unsigned int *out_dev, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out_dev, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  guard_kernel<<<1216, 256, 0, s>>>(phi, phat, g, ndim, (float)nsteps, out_dev);
  return cudaGetLastError();
}

}  // namespace ac
