// 2D streaming stencil for float storage with strips of two 16-byte
// vectors per lane (tile 1; see stream2d.cuh).
#include "stream2d.cuh"

namespace ac {

cudaError_t stream2d_launch_f32_wide(int k, const GridParams &g, const CUtensorMap *map, void *dst,
                                     int num_sms, cudaStream_t s) {
  return s2_dispatch<float, 2>(k, g, map, dst, num_sms, s);
}

}  // namespace ac
