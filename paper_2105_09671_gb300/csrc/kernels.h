// Host-side launchers of the CUDA kernels (called by the C-ABI layer).
#pragma once

#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace ac {

// Geometry of the 2D streaming kernel for a storage type and depth k.
struct Stream2DGeom {
  int box_x, box_y;   // TMA box (elements, rows)
  int halo_x;         // halo columns on each side (multiple of the vector width)
  int out_w;          // output columns per warp strip
};
// Geometry of the 3D streaming kernel.
struct Stream3DGeom {
  int box_x, box_y;   // TMA box per plane (elements, rows)
  int halo_x;         // halo columns per side
  int out_x, out_y;   // output tile
  int threads;
  int smem_bytes;
};

// 2D strip widths ("tiles"): 0 = the storage type's default (FP32: 4 cells
// per lane), 1 = 8 FP32 cells per lane (FP32 only).
bool stream2d_supported(int dtype, int k, int tile);
Stream2DGeom stream2d_geom(int dtype, int k, int tile);
bool stream3d_supported(int dtype, int k, int tile);
Stream3DGeom stream3d_geom(int dtype, int k, int tile);

// One step per launch, clamped global-memory neighbours (2D and 3D).
// Launch shape of the cell-wise kernels (direct stencil, initial
// conditions): 64 x 4 threads per block over (x, y) and one block layer per
// z, with y and z capped at CUDA's 65535 blocks per grid dimension; the
// kernels cover the rest of y and z by grid-stride loops.
constexpr unsigned kCellBlockX = 64, kCellBlockY = 4;
// Whether cell_grid leaves y or z to the kernels' grid-stride loops.
inline bool cell_grid_tall(const GridParams &g) {
  return (g.ny + kCellBlockY - 1) / kCellBlockY > 65535 || g.nz > 65535;
}
// Calls f(j, k) for this thread's (y, z) cells: once (the grid covers the
// domain, no loop), or by grid-stride loops for TALL grids.
template <bool TALL, typename F>
__device__ __forceinline__ void for_cell_yz(const GridParams &g, F &&f) {
  const int64_t j0 = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  if constexpr (!TALL) {
    if (j0 < g.ny) f(j0, (int64_t)blockIdx.z);
  } else {
    for (int64_t k = blockIdx.z; k < g.nz; k += gridDim.z)
      for (int64_t j = j0; j < g.ny; j += (int64_t)gridDim.y * blockDim.y) f(j, k);
  }
}
inline dim3 cell_grid(const GridParams &g) {
  return dim3((unsigned)((g.nx + kCellBlockX - 1) / kCellBlockX),
              (unsigned)std::min<int64_t>((g.ny + kCellBlockY - 1) / kCellBlockY, 65535),
              (unsigned)std::min<int64_t>(g.nz, 65535));
}

cudaError_t launch_direct(int ndim, int dtype, const GridParams &g, const void *src, void *dst,
                          cudaStream_t s);
// k steps per launch.  src_map describes the source field with the box of
// stream{2,3}d_geom(dtype, k).
cudaError_t launch_stream2d(int dtype, int k, int tile, const GridParams &g, const CUtensorMap *src_map,
                            void *dst, int num_sms, cudaStream_t s);
cudaError_t launch_stream3d(int dtype, int k, int tile, const GridParams &g,
                            const CUtensorMap *src_map, void *dst, int num_sms, cudaStream_t s);

// FP64 reductions: out[0] = sum F(phi), out[1] = sum over interior faces of
// (phi_a - phi_b)^2, out[2] = sum (1 + phi)/2, out[3] = non-finite count.
// partials must hold kReduceBlocks * 4 doubles.
constexpr int kReduceBlocks = 1216;
cudaError_t launch_observe(int dtype, const GridParams &g, const void *phi, double *partials,
                           double *out, cudaStream_t s);

// Allocation-free variant of launch_observe: partial sums in a module-global
// array (one block per 64 rows, at most observe_noalloc_max_rows() rows);
// writes E_h, V and the non-finite count to out_dev[0..2] on the device.
int64_t observe_noalloc_max_rows();
cudaError_t launch_observe_noalloc(int dtype, const GridParams &g, const void *phi, double hd,
                                   double eps, double h, double *out_dev, cudaStream_t s);

// Guard of a learned jump (FP32, pitch == nx): out_dev[0] = bits of
// max |phi_hat|, out_dev[1] = bits of max |phi_hat - phi - n dt RHS(phi)|.
cudaError_t launch_guard(const float *phi, const float *phat, const GridParams &g, int ndim,
                         int nsteps, unsigned int *out_dev, cudaStream_t s);

// Spot check of a learned jump (FP32 fields, pitch == nx): the plain
// stepper's nsteps-step result from phi, computed exactly on `samples` boxes
// of side size + 2 nsteps (clipped to the grid) placed by `seed`, compared
// with phat on the exact cells.  scratch: spot_scratch_floats() floats;
// partials: 4 * samples doubles; out[4] = {max |phat - ref|, sum (phat -
// ref)^2, sum ref^2, cells compared} (device memory).
void spot_box(const GridParams &g, int ndim, int nsteps, int size, int box[3]);
size_t spot_scratch_floats(const GridParams &g, int ndim, int nsteps, int samples, int size);
cudaError_t launch_spot_check(const float *phi, const float *phat, const GridParams &g, int ndim,
                              int nsteps, int samples, int size, uint64_t seed, float *scratch,
                              double *partials, double *out, cudaStream_t s);
// out[4] = {max |a - b|, sum (a - b)^2, sum b^2, n} over n contiguous floats;
// partials: 4 * diff_norms_blocks() doubles.
int diff_norms_blocks();
cudaError_t launch_diff_norms(const float *a, const float *b, int64_t n, double *partials,
                              double *out, cudaStream_t s);

cudaError_t launch_init_sphere(int dtype, const GridParams &g, void *phi, double h,
                               const double lower[3], const double center[3], double r0,
                               double eps, cudaStream_t s);
cudaError_t launch_init_shape(int dtype, const GridParams &g, void *phi, int kind, int ndim,
                              double h, const double lower[3], double p0, double p1, double eps,
                              cudaStream_t s);
cudaError_t launch_init_random(int dtype, const GridParams &g, void *phi, uint64_t seed,
                               double amplitude, cudaStream_t s);

// D[m x 32] = A[m x k] * B[32 x k]^T on the tensor cores (BF16 in, FP32 out);
// m a multiple of 128, k a multiple of 16 in [16, 512].
cudaError_t launch_tc_gemm_n32(const void *a, const void *b, float *d, int64_t m, int k, int *status,
                               cudaStream_t s);

// ---- helpers shared by the C-ABI translation units (defined in ac_api.cu)
int set_error(int code, const char *msg);

// One-time, per-device set-up of a kernel that takes `smem` bytes of
// dynamic shared memory: raises its dynamic shared-memory limit and returns
// in *occ the CTAs of `threads` threads that fit on one SM (at least 1).
// Each kernel keeps one KernelSetup (a static of its launcher); the first
// launch on a device does the set-up under a process-wide mutex and
// publishes the result with release semantics, later launches read it
// without locking.  Devices beyond the cache are set up on every launch.
// Safe to call from several host threads at once.
constexpr int kSetupDevices = 64;
struct KernelSetup {
  std::atomic<int> occ[kSetupDevices];  // 0 = not set up on that device yet
};
// carveout >= 0 also sets the preferred shared-memory carveout (percent).
cudaError_t kernel_setup(KernelSetup &ks, const void *func, int threads, int smem, int *occ,
                         int carveout = -1);

}  // namespace ac

#include <vector>
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
int ac_validate_desc(const ac_grid_desc *d);
int ac_default_depth(const ac_grid_desc *d);  // temporal-block depth of the default schedule
bool ac_plan_depths(int64_t n, int k, std::vector<int> &depths);
EncodeTiledFn ac_encode_fn();
CUtensorMapDataType ac_tmap_type(int dtype);
size_t ac_elem_size(int dtype);
