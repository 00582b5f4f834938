// Storage-type dispatch of the 3D streaming stencil (kernel in stream3d.cuh).
#include "stream3d.cuh"

namespace ac {

bool stream3d_supported(int dtype, int k, int tile) {
  if (k < 1 || tile < 0 || tile >= kS3Tiles) return false;
  switch (dtype) {
    case AC_F64: return k <= S3Cfg<double, 0>::KMAX;
    case AC_F32: return k <= S3Cfg<float, 0>::KMAX;
    case AC_F16S: return k <= S3Cfg<__half, 0>::KMAX;
  }
  return false;
}

template <typename T>
static Stream3DGeom geom_tiles(int k, int tile) {
  switch (tile) {
    case 0: return s3_geom_tile<T, 0>(k);
    case 1: return s3_geom_tile<T, 1>(k);
    case 2: return s3_geom_tile<T, 2>(k);
  }
  return Stream3DGeom{0, 0, 0, 0, 0, 0, 0};
}

Stream3DGeom stream3d_geom(int dtype, int k, int tile) {
  switch (dtype) {
    case AC_F64: return geom_tiles<double>(k, tile);
    case AC_F32: return geom_tiles<float>(k, tile);
    case AC_F16S: return geom_tiles<__half>(k, tile);
  }
  return Stream3DGeom{0, 0, 0, 0, 0, 0, 0};
}

template <typename T>
static cudaError_t launch_tiles(int k, int tile, const GridParams &g, const CUtensorMap *map,
                                void *dst, int num_sms, cudaStream_t s) {
  static_assert(kS3Tiles == 3, "one case per tile");
  switch (tile) {
    case 0: return stream3d_launch_tile<T, 0>(k, g, map, dst, num_sms, s);
    case 1: return stream3d_launch_tile<T, 1>(k, g, map, dst, num_sms, s);
    case 2: return stream3d_launch_tile<T, 2>(k, g, map, dst, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_stream3d(int dtype, int k, int tile, const GridParams &g,
                            const CUtensorMap *src_map, void *dst, int num_sms, cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return launch_tiles<double>(k, tile, g, src_map, dst, num_sms, s);
    case AC_F32: return launch_tiles<float>(k, tile, g, src_map, dst, num_sms, s);
    case AC_F16S: return launch_tiles<__half>(k, tile, g, src_map, dst, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ac
