// Device-side initial conditions of Section 3.1, so that large grids are
// never generated on the host.
//   sphere/circle: phi = tanh((r0 - |x - c|) / (sqrt(2) eps)) at the cell
//                  centres x_i = lower + (i + 1/2) h (Section 2), in FP64,
//                  rounded once (nearest-even) to the storage type.
//   random:        phi = amplitude * (2 u - 1), u = (z >> 11) * 2^-53, with z
//                  the SplitMix64 output number (c + 1) for seed s and cell
//                  linear index c (Steele, Lea, Flood, OOPSLA 2014).
#include "kernels.h"

namespace ac {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void init_sphere_k(T *__restrict__ phi, GridParams g, double h, double lx, double ly,
                              double lz, double cx, double cy, double cz, double r0,
                              double width) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  const int64_t k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  // each operation rounded separately (no contraction), as written
  const double x = __dadd_rn(lx, __dmul_rn(__dadd_rn((double)i, 0.5), h));
  const double y = __dadd_rn(ly, __dmul_rn(__dadd_rn((double)j, 0.5), h));
  const double dx = __dsub_rn(x, cx), dy = __dsub_rn(y, cy);
  double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (g.nz > 1) {
    const double z = __dadd_rn(lz, __dmul_rn(__dadd_rn((double)k, 0.5), h));
    const double dz = __dsub_rn(z, cz);
    r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
  }
  const double v = tanh(__ddiv_rn(__dsub_rn(r0, __dsqrt_rn(r2)), width));
  phi[(k * g.ny + j) * g.pitch + i] = from_f64<T>(v);
}

template <typename T>
__global__ void init_random_k(T *__restrict__ phi, GridParams g, uint64_t seed, double amp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  const int64_t k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const uint64_t c = (uint64_t)((k * g.ny + j) * g.nx + i);
  const uint64_t z = splitmix64_at(seed, c);
  const double u = (double)(z >> 11) * 0x1.0p-53;
  const double r = __dsub_rn(__dmul_rn(2.0, u), 1.0);
  const double v = __dmul_rn(amp, r);
  phi[(k * g.ny + j) * g.pitch + i] = from_f64<T>(v);
}

template <typename T>
static cudaError_t sphere_t(const GridParams &g, void *phi, double h, const double *lo,
                            const double *c, double r0, double eps, cudaStream_t s) {
  dim3 block(64, 4);
  dim3 grid((unsigned)((g.nx + 63) / 64), (unsigned)((g.ny + 3) / 4), (unsigned)g.nz);
  const double width = sqrt(2.0) * eps;
  init_sphere_k<T><<<grid, block, 0, s>>>((T *)phi, g, h, lo[0], lo[1], lo[2], c[0], c[1], c[2],
                                          r0, width);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t random_t(const GridParams &g, void *phi, uint64_t seed, double amp,
                            cudaStream_t s) {
  dim3 block(64, 4);
  dim3 grid((unsigned)((g.nx + 63) / 64), (unsigned)((g.ny + 3) / 4), (unsigned)g.nz);
  init_random_k<T><<<grid, block, 0, s>>>((T *)phi, g, seed, amp);
  return cudaGetLastError();
}

cudaError_t launch_init_sphere(int dtype, const GridParams &g, void *phi, double h,
                               const double lower[3], const double center[3], double r0,
                               double eps, cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return sphere_t<double>(g, phi, h, lower, center, r0, eps, s);
    case AC_F32: return sphere_t<float>(g, phi, h, lower, center, r0, eps, s);
    case AC_F16S: return sphere_t<__half>(g, phi, h, lower, center, r0, eps, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_init_random(int dtype, const GridParams &g, void *phi, uint64_t seed,
                               double amplitude, cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return random_t<double>(g, phi, seed, amplitude, s);
    case AC_F32: return random_t<float>(g, phi, seed, amplitude, s);
    case AC_F16S: return random_t<__half>(g, phi, seed, amplitude, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ac
