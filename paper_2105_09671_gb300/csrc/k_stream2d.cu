// Storage-type and strip-width dispatch of the 2D streaming stencil (kernel
// in stream2d.cuh).
#include "stream2d.cuh"

namespace ac {

bool stream2d_supported(int dtype, int k, int tile) {
  if (k < 1 || tile < 0 || tile >= kS2Tiles) return false;
  switch (dtype) {
    case AC_F64: return k <= s2_kmax<double>(tile);
    case AC_F32: return k <= s2_kmax<float>(tile);
    case AC_F16S: return k <= s2_kmax<__half>(tile);
  }
  return false;
}

Stream2DGeom stream2d_geom(int dtype, int k, int tile) {
  if (!stream2d_supported(dtype, k, tile)) return Stream2DGeom{0, 0, 0, 0};
  switch (dtype) {
    case AC_F64: return s2_geom<double, S2Cfg<double>::VPL>(k);
    case AC_F32: return tile == 1 ? s2_geom<float, 2>(k) : s2_geom<float, S2Cfg<float>::VPL>(k);
    case AC_F16S: return s2_geom<__half, S2Cfg<__half>::VPL>(k);
  }
  return Stream2DGeom{0, 0, 0, 0};
}

cudaError_t launch_stream2d(int dtype, int k, int tile, const GridParams &g, const CUtensorMap *src_map,
                            void *dst, int num_sms, cudaStream_t s) {
  if (!stream2d_supported(dtype, k, tile)) return cudaErrorInvalidValue;
  switch (dtype) {
    case AC_F64: return stream2d_launch_f64(k, g, src_map, dst, num_sms, s);
    case AC_F32:
      return tile == 1 ? stream2d_launch_f32_wide(k, g, src_map, dst, num_sms, s)
                       : stream2d_launch_f32(k, g, src_map, dst, num_sms, s);
    case AC_F16S: return stream2d_launch_f16(k, g, src_map, dst, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ac
