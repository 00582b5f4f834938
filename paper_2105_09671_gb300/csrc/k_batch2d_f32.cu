// Batched persistent 2D stepping instantiated for float storage (see batch2d.cuh).
#include "batch2d.cuh"

namespace ac {

cudaError_t batch2d_launch_f32(const BInst *insts, const BItem *items, int n_items,
                             const CUtensorMap *maps, int *progress, unsigned long long *ticket,
                             long long total, int *status, uint32_t wait_limit, int num_sms,
                             cudaStream_t s, int *grid_out) {
  return batch2d_launch_t<float>(insts, items, n_items, maps, progress, ticket, total, status,
                                 wait_limit, num_sms, s, grid_out);
}

}  // namespace ac
