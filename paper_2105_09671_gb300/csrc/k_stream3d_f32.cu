// 3D streaming stencil instantiated for float storage (see stream3d.cuh).
#include "stream3d.cuh"

namespace ac {

cudaError_t stream3d_launch_f32(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                              int num_sms, cudaStream_t s) {
  return s3_dispatch<float>(k, g, map, dst, num_sms, s);
}

}  // namespace ac
