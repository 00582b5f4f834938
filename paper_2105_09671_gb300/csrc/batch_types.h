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

constexpr int kBatchKMax = 4;      // depths of the default strips (tile 0)
constexpr int kBatchKMaxWide = 6;  // depths of the 8-cell FP32 strips (tile 1)
constexpr int kBatchBoxRows = 2;   // rows per TMA box (equals the 2D kernel's)

// tile 0: the storage type's default strips; tile 1: FP32 strips of two
// 16-byte vectors per lane (as tile 1 of the single-grid 2D stepper)
inline int batch_kmax(int dtype, int tile) {
  return tile == 0 ? kBatchKMax : (tile == 1 && dtype == AC_F32 ? kBatchKMaxWide : 0);
}

cudaError_t batch2d_launch(int dtype, int tile, const BInst *insts, const BItem *items, int n_items,
                           const CUtensorMap *maps, int *progress, unsigned long long *ticket,
                           long long total, int *status, uint32_t wait_limit, int num_sms,
                           cudaStream_t s, int *grid_out);
cudaError_t batch2d_launch_f64(const BInst *, const BItem *, int, const CUtensorMap *, int *, unsigned long long *, long long, int *, uint32_t, int, cudaStream_t, int *);
cudaError_t batch2d_launch_f32(const BInst *, const BItem *, int, const CUtensorMap *, int *, unsigned long long *, long long, int *, uint32_t, int, cudaStream_t, int *);
cudaError_t batch2d_launch_f32_wide(const BInst *, const BItem *, int, const CUtensorMap *, int *, unsigned long long *, long long, int *, uint32_t, int, cudaStream_t, int *);
cudaError_t batch2d_launch_f16(const BInst *, const BItem *, int, const CUtensorMap *, int *, unsigned long long *, long long, int *, uint32_t, int, cudaStream_t, int *);

// Strip geometry the batch uses for a storage type, plan depth k and tile.
inline void batch_strip_geom(int dtype, int k, int tile, int *sw, int *hx, int *ow, int *vec) {
  const int V = dtype == AC_F64 ? 2 : dtype == AC_F32 ? 4 : 8;
  int E = dtype == AC_F64 ? 4 : V;  // cells per lane (S2Cfg::VPL * V)
  if (tile == 1) E = 2 * V;
  *vec = V;
  *sw = 32 * E;
  *hx = V * ((k + V - 1) / V);
  *ow = *sw - 2 * *hx;
}

}  // namespace ac
