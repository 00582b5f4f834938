// Checks of a learned jump against the plain stepper itself.
//
// Spot check: the n-step result of the explicit scheme (Eq. pytorchACeq) at
// a cell depends only on the cells within n cells of it (one neighbour per
// step), so the plain stepper's result can be computed exactly on a small
// box of the grid: copy the box, advance it n steps with the zero-Neumann
// clamp at every box edge, and keep the cells at distance >= n from every
// box edge that is not a face of the domain (at a domain face the clamp is
// the true ghost of Section 2).  Boxes of side P + 2n (clipped to the grid)
// at pseudo-random places, one CTA each; the arithmetic is the plain
// stepper's own (ac_update on the same neighbour sum order in FP32), so the
// reference values equal the plain stepper's output bit for bit.  The
// comparison with the jump phi_hat is reduced per box and then over the
// boxes in index order.
//
// Difference norms: max |a - b|, sum (a - b)^2 and sum b^2 over a whole
// field (FP64 accumulation, fixed order), used when calibrating the guard.
#include "kernels.h"

namespace ac {

namespace {

__device__ __forceinline__ uint64_t spot_mix(uint64_t z) {
  // SplitMix64 finaliser (Steele, Lea, Flood 2014) as a hash
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Block-wide reduction of (max, sum, sum, count) in a fixed order; the
// result is valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_reduce4(float &mx, double &a, double &b, double &c) {
  __shared__ float smx[NT / 32];
  __shared__ double sa[NT / 32], sb[NT / 32], sc[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) { smx[warp] = mx; sa[warp] = a; sb[warp] = b; sc[warp] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) {
      mx = fmaxf(mx, smx[w]);
      a += sa[w];
      b += sb[w];
      c += sc[w];
    }
  }
}

constexpr int kSpotThreads = 512;

// One CTA per box.  scratch holds two boxes per sample; partials[s] =
// {max |phat - ref|, sum (phat - ref)^2, sum ref^2, cells compared}.
__global__ void __launch_bounds__(kSpotThreads) spot_check_k(
    const float *__restrict__ phi, const float *__restrict__ phat, GridParams g, int ndim,
    int nsteps, int bx, int by, int bz, uint64_t seed, float *scratch, double *partials) {
  const int s = blockIdx.x;
  const int64_t cols = (int64_t)bx * by, box = cols * bz;
  float *bufa = scratch + (int64_t)s * 2 * box;
  float *bufb = bufa + box;
  // box origin, uniform over the positions that keep the box in the grid
  const uint64_t hs = spot_mix(seed ^ spot_mix((uint64_t)s + 1));
  const int ox = (int)(spot_mix(hs + 1) % (uint64_t)(g.nx - bx + 1));
  const int oy = (int)(spot_mix(hs + 2) % (uint64_t)(g.ny - by + 1));
  const int oz = ndim == 3 ? (int)(spot_mix(hs + 3) % (uint64_t)(g.nz - bz + 1)) : 0;
  const int64_t plane = g.pitch * g.ny;
  const float *src_g = phi + (int64_t)oz * plane + (int64_t)oy * g.pitch + ox;
  for (int64_t col = threadIdx.x; col < cols; col += kSpotThreads) {
    const int x = (int)(col % bx), y = (int)(col / bx);
    for (int z = 0; z < bz; ++z) bufa[z * cols + col] = src_g[z * plane + (int64_t)y * g.pitch + x];
  }
  __syncthreads();

  const float alpha = (float)g.alpha, beta = (float)g.beta;
  const float m2d = ndim == 3 ? -6.0f : -4.0f;
  float *src = bufa, *dst = bufb;
  for (int t = 0; t < nsteps; ++t) {
    for (int64_t col = threadIdx.x; col < cols; col += kSpotThreads) {
      const int x = (int)(col % bx), y = (int)(col / bx);
      const int dw = x > 0 ? -1 : 0, de = x + 1 < bx ? 1 : 0;
      const int64_t ds = y > 0 ? -(int64_t)bx : 0, dn = y + 1 < by ? (int64_t)bx : 0;
      for (int z = 0; z < bz; ++z) {
        const int64_t c = z * cols + col;
        const float p = src[c];
        float nsum = (src[c + dw] + src[c + de]) + (src[c + ds] + src[c + dn]);
        if (ndim == 3) {
          const int64_t db = z > 0 ? -cols : 0, df = z + 1 < bz ? cols : 0;
          nsum = nsum + (src[c + db] + src[c + df]);
        }
        dst[c] = ac_update<float>(p, nsum, m2d, alpha, beta);
      }
    }
    __syncthreads();
    float *tmp = src;
    src = dst;
    dst = tmp;
  }

  // cells at distance >= n from every box edge inside the domain are exact
  const int vx0 = ox > 0 ? nsteps : 0, vx1 = ox + bx < g.nx ? bx - nsteps : bx;
  const int vy0 = oy > 0 ? nsteps : 0, vy1 = oy + by < g.ny ? by - nsteps : by;
  const int vz0 = (ndim == 3 && oz > 0) ? nsteps : 0;
  const int vz1 = (ndim == 3 && oz + bz < g.nz) ? bz - nsteps : bz;
  const float *hat_g = phat + (int64_t)oz * plane + (int64_t)oy * g.pitch + ox;
  float mx = 0.f;
  double d2 = 0.0, r2 = 0.0, cnt = 0.0;
  for (int64_t col = threadIdx.x; col < cols; col += kSpotThreads) {
    const int x = (int)(col % bx), y = (int)(col / bx);
    if (x < vx0 || x >= vx1 || y < vy0 || y >= vy1) continue;
    for (int z = vz0; z < vz1; ++z) {
      const float ref = src[z * cols + col];
      const float d = hat_g[z * plane + (int64_t)y * g.pitch + x] - ref;
      mx = fmaxf(mx, fabsf(d));
      if (d != d) mx = __int_as_float(0x7f800000);  // a NaN jump fails the check
      d2 += (double)d * (double)d;
      r2 += (double)ref * (double)ref;
      cnt += 1.0;
    }
  }
  block_reduce4<kSpotThreads>(mx, d2, r2, cnt);
  if (threadIdx.x == 0) {
    partials[4 * s + 0] = (double)mx;
    partials[4 * s + 1] = d2;
    partials[4 * s + 2] = r2;
    partials[4 * s + 3] = cnt;
  }
}

// Partials -> out[4] = {max, sum, sum, count}, one thread, index order.
__global__ void spot_final_k(const double *__restrict__ partials, int n, double *__restrict__ out) {
  if (threadIdx.x != 0) return;
  double m = 0.0, a = 0.0, b = 0.0, c = 0.0;
  for (int i = 0; i < n; ++i) {
    m = fmax(m, partials[4 * i]);
    if (partials[4 * i] != partials[4 * i]) m = partials[4 * i];
    a += partials[4 * i + 1];
    b += partials[4 * i + 2];
    c += partials[4 * i + 3];
  }
  out[0] = m;
  out[1] = a;
  out[2] = b;
  out[3] = c;
}

constexpr int kNormBlocks = 1216;
constexpr int kNormThreads = 256;

__global__ void __launch_bounds__(kNormThreads) diff_norms_k(const float *__restrict__ a,
                                                             const float *__restrict__ b, int64_t n,
                                                             double *__restrict__ partials) {
  float mx = 0.f;
  double d2 = 0.0, r2 = 0.0, cnt = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kNormThreads + threadIdx.x; i < n;
       i += (int64_t)kNormBlocks * kNormThreads) {
    const float d = a[i] - b[i];
    mx = fmaxf(mx, fabsf(d));
    if (d != d) mx = __int_as_float(0x7f800000);
    d2 += (double)d * (double)d;
    r2 += (double)b[i] * (double)b[i];
    cnt += 1.0;
  }
  block_reduce4<kNormThreads>(mx, d2, r2, cnt);
  if (threadIdx.x == 0) {
    partials[4 * blockIdx.x + 0] = (double)mx;
    partials[4 * blockIdx.x + 1] = d2;
    partials[4 * blockIdx.x + 2] = r2;
    partials[4 * blockIdx.x + 3] = cnt;
  }
}

}  // namespace

void spot_box(const GridParams &g, int ndim, int nsteps, int size, int box[3]) {
  const int64_t side = (int64_t)size + 2 * (int64_t)nsteps;
  box[0] = (int)std::min<int64_t>(side, g.nx);
  box[1] = (int)std::min<int64_t>(side, g.ny);
  box[2] = ndim == 3 ? (int)std::min<int64_t>(side, g.nz) : 1;
}

size_t spot_scratch_floats(const GridParams &g, int ndim, int nsteps, int samples, int size) {
  int b[3];
  spot_box(g, ndim, nsteps, size, b);
  return (size_t)samples * 2 * (size_t)b[0] * b[1] * b[2];
}

cudaError_t launch_spot_check(const float *phi, const float *phat, const GridParams &g, int ndim,
                              int nsteps, int samples, int size, uint64_t seed, float *scratch,
                              double *partials, double *out, cudaStream_t s) {
  if (samples < 1 || size < 1 || nsteps < 1) return cudaErrorInvalidValue;
  int b[3];
  spot_box(g, ndim, nsteps, size, b);
  spot_check_k<<<samples, kSpotThreads, 0, s>>>(phi, phat, g, ndim, nsteps, b[0], b[1], b[2], seed,
                                                 scratch, partials);
  spot_final_k<<<1, 32, 0, s>>>(partials, samples, out);
  return cudaGetLastError();
}

int diff_norms_blocks() { return kNormBlocks; }

cudaError_t launch_diff_norms(const float *a, const float *b, int64_t n, double *partials,
                              double *out, cudaStream_t s) {
  diff_norms_k<<<kNormBlocks, kNormThreads, 0, s>>>(a, b, n, partials);
  spot_final_k<<<1, 32, 0, s>>>(partials, kNormBlocks, out);
  return cudaGetLastError();
}

}  // namespace ac
