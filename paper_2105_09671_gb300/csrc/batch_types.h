// Work-item and instance tables of the batched persistent 2D stepper,
// shared by its kernel (batch2d.cuh) and its C-ABI layer (ac_batch.cu).
#pragma once

#include "kernels.h"

namespace ac {

struct BInst {
  void *buf[2];          // phi, workspace (step-block s reads buf[s & 1])
  int nx, ny;
  int64_t pitch;
  double alpha, beta;
  int S;                 // step-blocks of the current plan
  int k;                 // depth of step-blocks before tail_start
  int tail_start;        // first step-block whose depth comes from tail[]
  int tail[4];
  int fastx;             // nx is a multiple of the vector width
  int hx;                // halo columns per strip side
};

struct BItem {
  int inst, xs, y0, y1;
  int deps[9];           // items of the 3 x 3 neighbourhood (self included), -1 = none
};

constexpr int kBatchKMax = 4;
constexpr int kBatchBoxRows = 2;  // rows per TMA box (equals the 2D kernel's)

cudaError_t batch2d_launch(int dtype, const BInst *insts, const BItem *items, int n_items,
                           const CUtensorMap *maps, int *progress, unsigned long long *ticket,
                           long long total, int *status, uint32_t wait_limit, int num_sms,
                           cudaStream_t s, int *grid_out);
cudaError_t batch2d_launch_f64(const BInst *, const BItem *, int, const CUtensorMap *, int *, unsigned long long *, long long, int *, uint32_t, int, cudaStream_t, int *);
cudaError_t batch2d_launch_f32(const BInst *, const BItem *, int, const CUtensorMap *, int *, unsigned long long *, long long, int *, uint32_t, int, cudaStream_t, int *);
cudaError_t batch2d_launch_f16(const BInst *, const BItem *, int, const CUtensorMap *, int *, unsigned long long *, long long, int *, uint32_t, int, cudaStream_t, int *);

// Strip geometry the batch uses for a storage type and plan depth k.
inline void batch_strip_geom(int dtype, int k, int *sw, int *hx, int *ow, int *vec) {
  const int V = dtype == AC_F64 ? 2 : dtype == AC_F32 ? 4 : 8;
  const int E = dtype == AC_F64 ? 4 : V;  // cells per lane (S2Cfg::VPL * V)
  *vec = V;
  *sw = 32 * E;
  *hx = V * ((k + V - 1) / V);
  *ow = *sw - 2 * *hx;
}

}  // namespace ac
