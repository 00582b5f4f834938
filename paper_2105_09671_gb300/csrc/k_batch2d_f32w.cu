// Batched persistent 2D stepping for float storage with strips of two
// 16-byte vectors per lane (tile 1; see batch2d.cuh).
#include "batch2d.cuh"

namespace ac {

cudaError_t batch2d_launch_f32_wide(const BInst *insts, const BItem *items, int n_items,
                                    const CUtensorMap *maps, int *progress, unsigned long long *ticket,
                                    long long total, int *status, uint32_t wait_limit, int num_sms,
                                    cudaStream_t s, int *grid_out) {
  return batch2d_launch_t<float, 2>(insts, items, n_items, maps, progress, ticket, total, status,
                                    wait_limit, num_sms, s, grid_out);
}

}  // namespace ac
