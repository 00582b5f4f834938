// 2D streaming stencil instantiated for __half storage (see stream2d.cuh).
#include "stream2d.cuh"

namespace ac {

cudaError_t stream2d_launch_f16(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                              int num_sms, cudaStream_t s) {
  return s2_dispatch<__half, S2Cfg<__half>::VPL>(k, g, map, dst, num_sms, s);
}

}  // namespace ac
