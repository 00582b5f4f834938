// 3D streaming stencil for float storage, one tile shape per object
// (the build compiles this file once for each AC_S3_TILE in 0..kS3Tiles-1).
#include "stream3d.cuh"

#ifndef AC_S3_TILE
#error "compile with -DAC_S3_TILE=<tile>"
#endif

namespace ac {

template <typename T, int TILE>
cudaError_t stream3d_launch_tile(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                                 int num_sms, cudaStream_t s) {
  return s3_dispatch_tile<T, TILE>(k, g, map, dst, num_sms, s);
}

template cudaError_t stream3d_launch_tile<float, AC_S3_TILE>(int, const GridParams &,
                                                          const CUtensorMap *, void *, int,
                                                          cudaStream_t);

}  // namespace ac
