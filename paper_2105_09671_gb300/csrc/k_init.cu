// Device-side initial conditions of Section 3.1, so that large grids are
// never generated on the host.
//   sphere/circle: phi = tanh((r0 - |x - c|) / (sqrt(2) eps)) at the cell
//                  centres x_i = lower + (i + 1/2) h (Section 2), in FP64,
//                  rounded once (nearest-even) to the storage type.
//   dumbbell, star, torus: the further shapes of Section 3.1 (shape_value);
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

// tanh(num / w), w > 0, with the saturated range short-cut: for
// |num / w| >= 20 (less one rounding), 1 - tanh|a| = 2 / (e^{2|a|} + 1)
// < 2 e^{-39.9} < 2^-54 (half an ulp below 1), so the correctly rounded value
// is exactly +-1.  Most cells of a tanh profile lie there and skip the FP64
// division and tanh.
__device__ __forceinline__ double tanh_ratio(double num, double w, double sat = 20.0) {
  return fabs(num) >= __dmul_rn(sat, w) ? copysign(1.0, num) : tanh(__ddiv_rn(num, w));
}

// Where a profile value is stored as it is (the sphere), the short-cut can
// start where tanh rounds to +-1 in the storage type: 1 - tanh a < 2 e^{-2a}
// is below half the spacing under 1 (2^-25 for FP32, 2^-12 for FP16) from
// a = 9.5 (2 e^{-19} = 1.1e-8) and a = 6 (2 e^{-12} = 1.2e-5) on, so the
// FP64 value there rounds to exactly +-1 too and the stored field is the
// same.  (Shapes that add several tanh terms keep the FP64 threshold.)
template <typename T> struct SatArg { static constexpr double value = 20.0; };
template <> struct SatArg<float> { static constexpr double value = 9.5; };
template <> struct SatArg<__half> { static constexpr double value = 6.0; };

template <typename T>
__device__ __forceinline__ void sphere_cell(T *__restrict__ phi, const GridParams &g, int64_t i,
                                            int64_t j, int64_t k, double h, double lx, double ly,
                                            double lz, double cx, double cy, double cz, double r0,
                                            double width) {
  constexpr double kSat = SatArg<T>::value;
  // Far from the interface the stored profile is exactly +-1 (|arg| >= kSat,
  // see SatArg).  An FP32 estimate of the distance decides that for most
  // cells, in FP32 throughout: its error is below 1e-6 (1 + r + |r0| +
  // |lower| + |c|) (a few FP32 roundings of values of that size), so beyond
  // twenty times that margin the FP64 argument is past kSat on the same side.
  {
    const float xf = (float)lx + ((float)i + 0.5f) * (float)h - (float)cx;
    const float yf = (float)ly + ((float)j + 0.5f) * (float)h - (float)cy;
    float r2f = xf * xf + yf * yf;
    if (g.nz > 1) {
      const float zf = (float)lz + ((float)k + 0.5f) * (float)h - (float)cz;
      r2f += zf * zf;
    }
    const float rf = sqrtf(r2f);
    const float gapf = (float)r0 - rf;
    const float margin = 2e-5f * (1.0f + rf + fabsf((float)r0) + fabsf((float)lx) + fabsf((float)ly) +
                                  fabsf((float)lz) + fabsf((float)cx) + fabsf((float)cy) + fabsf((float)cz));
    if (fabsf(gapf) >= (float)(kSat * width) + margin) {
      phi[(k * g.ny + j) * g.pitch + i] = from_f64<T>(gapf > 0.0f ? 1.0 : -1.0);
      return;
    }
  }
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
  const double v = tanh_ratio(__dsub_rn(r0, __dsqrt_rn(r2)), width, kSat);
  phi[(k * g.ny + j) * g.pitch + i] = from_f64<T>(v);
}

// one thread per x; y and z as for_cell_yz (see cell_grid)
template <typename T, bool TALL>
__global__ void init_sphere_k(T *__restrict__ phi, GridParams g, double h, double lx, double ly,
                              double lz, double cx, double cy, double cz, double r0,
                              double width) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  for_cell_yz<TALL>(g, [&](int64_t j, int64_t k) {
    sphere_cell(phi, g, i, j, k, h, lx, ly, lz, cx, cy, cz, r0, width);
  });
}

template <typename T, bool TALL>
__global__ void init_random_k(T *__restrict__ phi, GridParams g, uint64_t seed, double amp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  for_cell_yz<TALL>(g, [&](int64_t j, int64_t k) {
    const uint64_t c = (uint64_t)((k * g.ny + j) * g.nx + i);
    const uint64_t z = splitmix64_at(seed, c);
    const double u = (double)(z >> 11) * 0x1.0p-53;
    const double r = __dsub_rn(__dmul_rn(2.0, u), 1.0);
    const double v = __dmul_rn(amp, r);
    phi[(k * g.ny + j) * g.pitch + i] = from_f64<T>(v);
  });
}

// Polar angle of the star (Section 3.1): atan(v/u) for u > 0, pi + atan(v/u)
// otherwise; u == 0 takes the limits +-pi/2 of atan (0 at the centre).
__device__ __forceinline__ double star_theta(double u, double v) {
  double base;
  if (u == 0.0)
    base = v > 0.0 ? 1.5707963267948966 : (v < 0.0 ? -1.5707963267948966 : 0.0);
  else
    base = atan(__ddiv_rn(v, u));
  return u > 0.0 ? base : __dadd_rn(3.141592653589793, base);
}

// The further shapes of Section 3.1 at one point (FP64, every operation
// rounded separately as written):
//   dumbbell: 1 inside the bar 0.4 < x < 1.6, 0.4 < y (, z) < 0.6, else
//             1 + tanh((p0 - |p - (0.3, .5[, .5])|)/w) + tanh((p0 - |p - (1.7, .5[, .5])|)/w)
//   star:     2D tanh((0.25 + 0.1 cos 6t - |p - (.5, .5)|)/w), t the angle about (.5, .5);
//             3D tanh((0.7 + 0.2 cos 6t - |p|)/w), t the angle of (x, z) about 0
//   torus:    2D -1 + tanh((p0 - r)/w) - tanh((p1 - r)/w), r = |p - (.5, .5)|;
//             3D tanh((p1 - sqrt(z^2 + (sqrt(x^2 + y^2) - p0)^2))/w)
// with w = sqrt(2) eps.
__device__ double shape_value(int kind, int ndim, double x, double y, double z, double p0,
                              double p1, double w) {
  if (kind == AC_SHAPE_DUMBBELL) {
    double tr = __dmul_rn(__dsub_rn(y, 0.5), __dsub_rn(y, 0.5));
    bool bar = x > 0.4 && x < 1.6 && y > 0.4 && y < 0.6;
    if (ndim == 3) {
      tr = __dadd_rn(tr, __dmul_rn(__dsub_rn(z, 0.5), __dsub_rn(z, 0.5)));
      bar = bar && z > 0.4 && z < 0.6;
    }
    if (bar) return 1.0;
    const double dl = __dsub_rn(x, 0.3), dr = __dsub_rn(x, 1.7);
    const double left = tanh_ratio(__dsub_rn(p0, __dsqrt_rn(__dadd_rn(__dmul_rn(dl, dl), tr))), w);
    const double right = tanh_ratio(__dsub_rn(p0, __dsqrt_rn(__dadd_rn(__dmul_rn(dr, dr), tr))), w);
    return __dadd_rn(__dadd_rn(1.0, left), right);
  }
  if (kind == AC_SHAPE_STAR) {
    if (ndim == 2) {
      const double u = __dsub_rn(x, 0.5), v = __dsub_rn(y, 0.5);
      const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)));
      const double rs = __dadd_rn(0.25, __dmul_rn(0.1, cos(__dmul_rn(6.0, star_theta(u, v)))));
      return tanh_ratio(__dsub_rn(rs, r), w);
    }
    const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    const double rs = __dadd_rn(0.7, __dmul_rn(0.2, cos(__dmul_rn(6.0, star_theta(x, z)))));
    return tanh_ratio(__dsub_rn(rs, r), w);
  }
  // torus
  if (ndim == 2) {
    const double u = __dsub_rn(x, 0.5), v = __dsub_rn(y, 0.5);
    const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)));
    return __dsub_rn(__dadd_rn(-1.0, tanh_ratio(__dsub_rn(p0, r), w)),
                     tanh_ratio(__dsub_rn(p1, r), w));
  }
  const double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
  const double q = __dsub_rn(rho, p0);
  const double d = __dsub_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(z, z), __dmul_rn(q, q))), p1);
  return tanh_ratio(-d, w);
}

template <typename T, bool TALL>
__global__ void init_shape_k(T *__restrict__ phi, GridParams g, int kind, int ndim, double h,
                             double lx, double ly, double lz, double p0, double p1, double width) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  const double x = __dadd_rn(lx, __dmul_rn(__dadd_rn((double)i, 0.5), h));
  for_cell_yz<TALL>(g, [&](int64_t j, int64_t k) {
    const double y = __dadd_rn(ly, __dmul_rn(__dadd_rn((double)j, 0.5), h));
    const double z = __dadd_rn(lz, __dmul_rn(__dadd_rn((double)k, 0.5), h));
    phi[(k * g.ny + j) * g.pitch + i] = from_f64<T>(shape_value(kind, ndim, x, y, z, p0, p1, width));
  });
}

template <typename T>
static cudaError_t shape_t(const GridParams &g, void *phi, int kind, int ndim, double h,
                           const double *lo, double p0, double p1, double eps, cudaStream_t s) {
  const dim3 block(kCellBlockX, kCellBlockY), grid = cell_grid(g);
  const double w = sqrt(2.0) * eps;
  if (cell_grid_tall(g))
    init_shape_k<T, true><<<grid, block, 0, s>>>((T *)phi, g, kind, ndim, h, lo[0], lo[1], lo[2], p0, p1, w);
  else
    init_shape_k<T, false><<<grid, block, 0, s>>>((T *)phi, g, kind, ndim, h, lo[0], lo[1], lo[2], p0, p1, w);
  return cudaGetLastError();
}

cudaError_t launch_init_shape(int dtype, const GridParams &g, void *phi, int kind, int ndim,
                              double h, const double lower[3], double p0, double p1, double eps,
                              cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return shape_t<double>(g, phi, kind, ndim, h, lower, p0, p1, eps, s);
    case AC_F32: return shape_t<float>(g, phi, kind, ndim, h, lower, p0, p1, eps, s);
    case AC_F16S: return shape_t<__half>(g, phi, kind, ndim, h, lower, p0, p1, eps, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t sphere_t(const GridParams &g, void *phi, double h, const double *lo,
                            const double *c, double r0, double eps, cudaStream_t s) {
  const dim3 block(kCellBlockX, kCellBlockY), grid = cell_grid(g);
  const double width = sqrt(2.0) * eps;
  if (cell_grid_tall(g))
    init_sphere_k<T, true><<<grid, block, 0, s>>>((T *)phi, g, h, lo[0], lo[1], lo[2], c[0], c[1], c[2],
                                                  r0, width);
  else
    init_sphere_k<T, false><<<grid, block, 0, s>>>((T *)phi, g, h, lo[0], lo[1], lo[2], c[0], c[1], c[2],
                                                   r0, width);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t random_t(const GridParams &g, void *phi, uint64_t seed, double amp,
                            cudaStream_t s) {
  const dim3 block(kCellBlockX, kCellBlockY), grid = cell_grid(g);
  if (cell_grid_tall(g)) init_random_k<T, true><<<grid, block, 0, s>>>((T *)phi, g, seed, amp);
  else init_random_k<T, false><<<grid, block, 0, s>>>((T *)phi, g, seed, amp);
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
