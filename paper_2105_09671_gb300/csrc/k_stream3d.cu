// Storage-type dispatch of the 3D streaming stencil (kernel in stream3d.cuh).
#include "stream3d.cuh"

namespace ac {

bool stream3d_supported(int dtype, int k) {
  if (k < 1) return false;
  switch (dtype) {
    case AC_F64: return k <= S3Cfg<double>::KMAX;
    case AC_F32: return k <= S3Cfg<float>::KMAX;
    case AC_F16S: return k <= S3Cfg<__half>::KMAX;
  }
  return false;
}

Stream3DGeom stream3d_geom(int dtype, int k) {
  switch (dtype) {
    case AC_F64: return s3_geom<double>(k);
    case AC_F32: return s3_geom<float>(k);
    case AC_F16S: return s3_geom<__half>(k);
  }
  return Stream3DGeom{0, 0, 0, 0, 0, 0, 0};
}

cudaError_t launch_stream3d(int dtype, int k, const GridParams &g, const CUtensorMap *src_map,
                            void *dst, int num_sms, cudaStream_t s) {
  switch (dtype) {
    case AC_F64: return stream3d_launch_f64(k, g, src_map, dst, num_sms, s);
    case AC_F32: return stream3d_launch_f32(k, g, src_map, dst, num_sms, s);
    case AC_F16S: return stream3d_launch_f16(k, g, src_map, dst, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ac
