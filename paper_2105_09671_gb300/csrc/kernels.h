// Host-side launchers of the CUDA kernels (called by the C-ABI layer).
#pragma once

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

bool stream2d_supported(int dtype, int k);
Stream2DGeom stream2d_geom(int dtype, int k);
bool stream3d_supported(int dtype, int k, int tile);
Stream3DGeom stream3d_geom(int dtype, int k, int tile);

// One step per launch, clamped global-memory neighbours (2D and 3D).
cudaError_t launch_direct(int ndim, int dtype, const GridParams &g, const void *src, void *dst,
                          cudaStream_t s);
// k steps per launch.  src_map describes the source field with the box of
// stream{2,3}d_geom(dtype, k).
cudaError_t launch_stream2d(int dtype, int k, const GridParams &g, const CUtensorMap *src_map,
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

}  // namespace ac

#include <vector>
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
int ac_validate_desc(const ac_grid_desc *d);
bool ac_plan_depths(int64_t n, int k, std::vector<int> &depths);
EncodeTiledFn ac_encode_fn();
CUtensorMapDataType ac_tmap_type(int dtype);
size_t ac_elem_size(int dtype);
