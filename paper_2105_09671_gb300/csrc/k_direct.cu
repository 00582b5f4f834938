// Direct stencil kernels: one explicit Euler step (Eq. pytorchACeq) per
// launch, every neighbour read from global memory with its index clamped to
// the domain, which realises the zero-Neumann ghost copy of Section 2
// (the ghost equals its adjacent interior cell).  This is the plain variant
// the streaming kernels are checked and timed against.
#include "kernels.h"

namespace ac {

template <typename T>
__device__ __forceinline__ void step2d_cell(const T *__restrict__ src, T *__restrict__ dst,
                                            const GridParams &g, int64_t i, int64_t j) {
  using C = typename Traits<T>::C;
  const int64_t im = i > 0 ? i - 1 : 0, ip = i + 1 < g.nx ? i + 1 : i;
  const int64_t jm = j > 0 ? j - 1 : 0, jp = j + 1 < g.ny ? j + 1 : j;
  const T *row = src + j * g.pitch;
  C p = to_c(row[i]);
  C w = to_c(row[im]), e = to_c(row[ip]);
  C s = to_c(src[jm * g.pitch + i]), n = to_c(src[jp * g.pitch + i]);
  C nsum = (w + e) + (s + n);
  dst[j * g.pitch + i] = from_c<T>(ac_update<C>(p, nsum, C(-4), C(g.alpha), C(g.beta)));
}

template <typename T>
__device__ __forceinline__ void step3d_cell(const T *__restrict__ src, T *__restrict__ dst,
                                            const GridParams &g, int64_t i, int64_t j, int64_t k) {
  using C = typename Traits<T>::C;
  const int64_t im = i > 0 ? i - 1 : 0, ip = i + 1 < g.nx ? i + 1 : i;
  const int64_t jm = j > 0 ? j - 1 : 0, jp = j + 1 < g.ny ? j + 1 : j;
  const int64_t km = k > 0 ? k - 1 : 0, kp = k + 1 < g.nz ? k + 1 : k;
  const int64_t plane = g.pitch * g.ny;
  const T *row = src + k * plane + j * g.pitch;
  C p = to_c(row[i]);
  C w = to_c(row[im]), e = to_c(row[ip]);
  C s = to_c(src[k * plane + jm * g.pitch + i]), n = to_c(src[k * plane + jp * g.pitch + i]);
  C b = to_c(src[km * plane + j * g.pitch + i]), f = to_c(src[kp * plane + j * g.pitch + i]);
  C nsum = ((w + e) + (s + n)) + (b + f);
  dst[k * plane + j * g.pitch + i] = from_c<T>(ac_update<C>(p, nsum, C(-6), C(g.alpha), C(g.beta)));
}

// one thread per x; y and z as for_cell_yz (see cell_grid)
template <typename T, bool TALL>
__global__ void __launch_bounds__(256) step2d_direct(const T *__restrict__ src,
                                                     T *__restrict__ dst, GridParams g) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  for_cell_yz<TALL>(g, [&](int64_t j, int64_t) { step2d_cell(src, dst, g, i, j); });
}

template <typename T, bool TALL>
__global__ void __launch_bounds__(256) step3d_direct(const T *__restrict__ src,
                                                     T *__restrict__ dst, GridParams g) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  for_cell_yz<TALL>(g, [&](int64_t j, int64_t k) { step3d_cell(src, dst, g, i, j, k); });
}

template <typename T>
static cudaError_t direct_t(int ndim, const GridParams &g, const void *src, void *dst,
                            cudaStream_t s) {
  const dim3 block(kCellBlockX, kCellBlockY), grid = cell_grid(g);
  const bool tall = cell_grid_tall(g);
  if (ndim == 2) {
    if (tall) step2d_direct<T, true><<<grid, block, 0, s>>>((const T *)src, (T *)dst, g);
    else step2d_direct<T, false><<<grid, block, 0, s>>>((const T *)src, (T *)dst, g);
  } else {
    if (tall) step3d_direct<T, true><<<grid, block, 0, s>>>((const T *)src, (T *)dst, g);
    else step3d_direct<T, false><<<grid, block, 0, s>>>((const T *)src, (T *)dst, g);
  }
  return cudaGetLastError();
}

cudaError_t launch_direct(int ndim, int dtype, const GridParams &g, const void *src, void *dst,
                          cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return direct_t<double>(ndim, g, src, dst, s);
    case AC_F32: return direct_t<float>(ndim, g, src, dst, s);
    case AC_F16S: return direct_t<__half>(ndim, g, src, dst, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ac
