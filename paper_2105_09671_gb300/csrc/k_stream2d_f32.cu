// 2D streaming stencil instantiated for float storage (see stream2d.cuh).
#include "stream2d.cuh"

namespace ac {

cudaError_t stream2d_launch_f32(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                              int num_sms, cudaStream_t s) {
  return s2_dispatch<float, S2Cfg<float>::VPL>(k, g, map, dst, num_sms, s);
}

}  // namespace ac
