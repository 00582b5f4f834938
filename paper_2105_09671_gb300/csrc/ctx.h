// Internal layout of a stepping context (shared by the C-ABI translation
// units).
#pragma once

#include "kernels.h"

struct MapPair {
  bool valid = false;
  CUtensorMap phi, ws;
};

struct ac_ctx {
  ac_grid_desc d;
  void *phi = nullptr, *ws = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 1;
  ac::GridParams gp;
  int *d_status = nullptr;
  double *d_partials = nullptr, *d_out = nullptr, *h_out = nullptr;
  int variant = AC_VARIANT_AUTO, k = 0;  // user request
  int tile = AC_TILE_AUTO;               // user request (3D streaming tile)
  int tuned_variant = 0, tuned_k = 0;    // autotuner result (0 = none)
  int tuned_tile = 0;
  MapPair maps[AC_NUM_TILES_3D][AC_MAX_K + 1];
  // graph replay
  bool use_graph = false;
  int64_t graph_n = -1;
  int graph_variant = -1, graph_k = -1, graph_tile = -1;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_launches = 0;  // kernels in the captured graph
  // kernels this context has put on its stream (graph replays count their nodes)
  int64_t launches = 0;
};

