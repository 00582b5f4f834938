// Storage-type dispatch of the 2D streaming stencil (kernel in stream2d.cuh).
#include "stream2d.cuh"

namespace ac {

bool stream2d_supported(int dtype, int k) {
  if (k < 1) return false;
  switch (dtype) {
    case AC_F64: return k <= S2Cfg<double>::KMAX;
    case AC_F32: return k <= S2Cfg<float>::KMAX;
    case AC_F16S: return k <= S2Cfg<__half>::KMAX;
  }
  return false;
}

Stream2DGeom stream2d_geom(int dtype, int k) {
  switch (dtype) {
    case AC_F64: return s2_geom<double>(k);
    case AC_F32: return s2_geom<float>(k);
    case AC_F16S: return s2_geom<__half>(k);
  }
  return Stream2DGeom{0, 0, 0, 0};
}

cudaError_t launch_stream2d(int dtype, int k, const GridParams &g, const CUtensorMap *src_map,
                            void *dst, int num_sms, cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return stream2d_launch_f64(k, g, src_map, dst, num_sms, s);
    case AC_F32: return stream2d_launch_f32(k, g, src_map, dst, num_sms, s);
    case AC_F16S: return stream2d_launch_f16(k, g, src_map, dst, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ac
