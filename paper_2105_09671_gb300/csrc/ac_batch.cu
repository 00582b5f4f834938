// C ABI of the batched persistent stepper (many independent 2D grids in one
// launch): validation, work-item tables, per-instance plans, graph replay.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "batch_types.h"

using namespace ac;

static int bfail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_error(code, buf);
}

#define BC_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(AC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
  } while (0)

static size_t bfield_bytes(const ac_grid_desc &d) {
  return (size_t)d.pitch_x * (size_t)d.ny * (size_t)d.nz * ac_elem_size(d.dtype);
}
static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

constexpr uint32_t kDefaultWaitPolls = 1u << 22;

struct ac_batch {
  int count = 0, dtype = 0;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 1;
  std::vector<ac_grid_desc> d;
  std::vector<void *> phi, ws;
  int k = 0;            // plan depth (0 = default)
  int tile = 0;         // strip width (0: default strips, 1: 8-cell FP32 strips)
  int chunk_rows = 64;  // rows per work item
  bool items_valid = false;
  int items_k = -1, items_tile = -1;
  // host / device tables
  std::vector<BInst> h_inst;
  std::vector<BItem> h_items;
  std::vector<int64_t> cur_n;
  std::vector<int> odd;  // instances whose plan ends in the workspace
  BInst *d_inst = nullptr;
  BItem *d_items = nullptr;
  CUtensorMap *d_maps = nullptr;       // [instance][phi, ws], box of tile-0 strips
  CUtensorMap *d_maps_wide = nullptr;  // the same for tile-1 strips (FP32 only)
  int *d_progress = nullptr;
  unsigned long long *d_ticket = nullptr;
  int *d_status = nullptr;
  double *d_partials = nullptr, *d_out = nullptr, *h_out = nullptr;
  long long total_tickets = 0;
  uint32_t wait_limit = kDefaultWaitPolls;
  int64_t launches = 0;
  // graph replay
  bool use_graph = false;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_launches = 0;
};

static int default_k(int dtype) { return dtype == AC_F64 ? 1 : 4; }

static void release_items(ac_batch *b) {
  cudaFree(b->d_items);
  cudaFree(b->d_progress);
  b->d_items = nullptr;
  b->d_progress = nullptr;
  b->items_valid = false;
}

static void release_graph(ac_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

// Work items for plan depth k: per instance, strips of the 2D streaming
// kernel (halo HX(k)) times row chunks, each with its 3 x 3 neighbourhood.
static int build_items(ac_batch *b, int k) {
  if (b->items_valid && b->items_k == k && b->items_tile == b->tile) return AC_OK;
  release_items(b);
  release_graph(b);
  int sw, hx, ow, vec;
  batch_strip_geom(b->dtype, k, b->tile, &sw, &hx, &ow, &vec);
  b->h_items.clear();
  for (int i = 0; i < b->count; ++i) {
    const ac_grid_desc &d = b->d[i];
    const int ns = (int)((d.nx + ow - 1) / ow);
    const int nc = (int)((d.ny + b->chunk_rows - 1) / b->chunk_rows);
    const int base = (int)b->h_items.size();
    for (int c = 0; c < nc; ++c)
      for (int s = 0; s < ns; ++s) {
        BItem it;
        it.inst = i;
        it.xs = s * ow - hx;
        it.y0 = c * b->chunk_rows;
        it.y1 = (int)std::min<int64_t>(d.ny, (int64_t)(c + 1) * b->chunk_rows);
        int q = 0;
        for (int dc = -1; dc <= 1; ++dc)
          for (int ds = -1; ds <= 1; ++ds) {
            const int cc = c + dc, ss = s + ds;
            it.deps[q++] = (cc >= 0 && cc < nc && ss >= 0 && ss < ns) ? base + cc * ns + ss : -1;
          }
        b->h_items.push_back(it);
      }
    b->h_inst[i].hx = hx;
    b->h_inst[i].fastx = (d.nx % vec) == 0;
  }
  const size_t bytes = sizeof(BItem) * b->h_items.size();
  BC_CUDA(cudaMalloc(&b->d_items, bytes));
  BC_CUDA(cudaMemcpy(b->d_items, b->h_items.data(), bytes, cudaMemcpyHostToDevice));
  BC_CUDA(cudaMalloc(&b->d_progress, sizeof(int) * b->h_items.size()));
  b->items_valid = true;
  b->items_k = k;
  b->items_tile = b->tile;
  return AC_OK;
}

extern "C" int ac_batch_workspace_bytes(const ac_grid_desc *descs, int32_t count, size_t *out) {
  if (!descs || count < 1 || !out) return bfail(AC_ERR_INVALID, "descs, count >= 1 and out required");
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    int rc = ac_validate_desc(&descs[i]);
    if (rc) return rc;
    total += round256(bfield_bytes(descs[i]));
  }
  *out = total;
  return AC_OK;
}

extern "C" int ac_batch_create(const ac_grid_desc *descs, void *const *phi_devs, int32_t count,
                               void *workspace_dev, void *cuda_stream, ac_batch **out) {
  if (!out) return bfail(AC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!descs || !phi_devs || count < 1 || !workspace_dev)
    return bfail(AC_ERR_INVALID, "descs, phi_devs, count >= 1 and workspace required");
  for (int i = 0; i < count; ++i) {
    int rc = ac_validate_desc(&descs[i]);
    if (rc) return rc;
    if (descs[i].ndim != 2)
      return bfail(AC_ERR_UNSUPPORTED, "instance %d: the batched stepper takes 2D grids", i);
    if (descs[i].dtype != descs[0].dtype)
      return bfail(AC_ERR_INVALID, "instance %d: all instances must share one dtype", i);
    if (descs[i].nx > (1 << 29) || descs[i].ny > (1 << 29))
      return bfail(AC_ERR_INVALID, "instance %d: grid too large", i);
    if (!phi_devs[i] || ((uintptr_t)phi_devs[i] & 15))
      return bfail(AC_ERR_INVALID, "instance %d: phi must be a 16-byte aligned device pointer", i);
  }
  if ((uintptr_t)workspace_dev & 255)
    return bfail(AC_ERR_INVALID, "workspace must be 256-byte aligned");
  ac_batch *b = new (std::nothrow) ac_batch();
  if (!b) return bfail(AC_ERR_NOMEM, "out of host memory");
  b->count = count;
  b->dtype = descs[0].dtype;
  b->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  b->d.assign(descs, descs + count);
  b->phi.assign(phi_devs, phi_devs + count);
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    b->ws.push_back(static_cast<char *>(workspace_dev) + off);
    off += round256(bfield_bytes(descs[i]));
  }
  b->h_inst.resize(count);
  for (int i = 0; i < count; ++i) {
    BInst &in = b->h_inst[i];
    memset(&in, 0, sizeof in);
    in.buf[0] = b->phi[i];
    in.buf[1] = b->ws[i];
    in.nx = (int)descs[i].nx;
    in.ny = (int)descs[i].ny;
    in.pitch = descs[i].pitch_x;
    in.alpha = descs[i].dt / (descs[i].eps * descs[i].eps);
    in.beta = descs[i].dt / (descs[i].h * descs[i].h);
  }
  // per-instance tensor maps of phi and workspace (box SW x rows, zero fill)
  // for each strip width the storage type offers; over-aligned type: a
  // plain 64-byte aligned host array
  const int n_tiles = batch_kmax(b->dtype, 1) > 0 ? 2 : 1;
  const size_t n_maps = 2 * (size_t)count;
  CUtensorMap *maps = static_cast<CUtensorMap *>(
      std::aligned_alloc(64, (sizeof(CUtensorMap) * n_maps * n_tiles + 63) / 64 * 64));
  if (!maps) { delete b; return bfail(AC_ERR_NOMEM, "out of host memory"); }
  EncodeTiledFn fn = ac_encode_fn();
  const size_t es = ac_elem_size(b->dtype);
  int rc = AC_OK;
  if (!fn) rc = bfail(AC_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  for (int t = 0; t < n_tiles && rc == AC_OK; ++t) {
    int sw, hx, ow, vec;
    batch_strip_geom(b->dtype, 1, t, &sw, &hx, &ow, &vec);
    for (int i = 0; i < count && rc == AC_OK; ++i)
      for (int w = 0; w < 2 && rc == AC_OK; ++w) {
        cuuint64_t dims[2] = {(cuuint64_t)descs[i].nx, (cuuint64_t)descs[i].ny};
        cuuint64_t strides[1] = {(cuuint64_t)(descs[i].pitch_x * es)};
        cuuint32_t box[2] = {(cuuint32_t)sw, (cuuint32_t)kBatchBoxRows}, estr[2] = {1, 1};
        CUresult r = fn(&maps[t * n_maps + 2 * i + w], ac_tmap_type(b->dtype), 2, w ? b->ws[i] : b->phi[i],
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) rc = bfail(AC_ERR_CUDA, "instance %d: tensor map encode failed (%d)", i, (int)r);
      }
  }
  cudaError_t e = cudaSuccess;
  if (rc == AC_OK) {
    e = cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * n_maps);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_maps, maps, sizeof(CUtensorMap) * n_maps, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_tiles > 1) e = cudaMalloc(&b->d_maps_wide, sizeof(CUtensorMap) * n_maps);
    if (e == cudaSuccess && n_tiles > 1)
      e = cudaMemcpy(b->d_maps_wide, maps + n_maps, sizeof(CUtensorMap) * n_maps, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, sizeof(BInst) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ticket, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_partials, sizeof(double) * 4 * kReduceBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_out, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_out, sizeof(double) * 4);
    if (e != cudaSuccess) rc = bfail(AC_ERR_NOMEM, "internal allocation failed: %s", cudaGetErrorString(e));
  }
  std::free(maps);
  if (rc != AC_OK) {
    cudaGetLastError();
    cudaFree(b->d_maps); cudaFree(b->d_maps_wide); cudaFree(b->d_inst); cudaFree(b->d_ticket); cudaFree(b->d_status);
    cudaFree(b->d_partials); cudaFree(b->d_out); cudaFreeHost(b->h_out);
    delete b;
    return rc;
  }
  *out = b;
  return AC_OK;
}

extern "C" int ac_batch_destroy(ac_batch *b) {
  if (!b) return AC_OK;
  cudaStreamSynchronize(b->stream);
  release_graph(b);
  release_items(b);
  cudaFree(b->d_maps); cudaFree(b->d_maps_wide); cudaFree(b->d_inst); cudaFree(b->d_ticket); cudaFree(b->d_status);
  cudaFree(b->d_partials); cudaFree(b->d_out); cudaFreeHost(b->h_out);
  delete b;
  return AC_OK;
}

extern "C" int ac_batch_set_schedule(ac_batch *b, int32_t k) {
  if (!b) return bfail(AC_ERR_INVALID, "batch is NULL");
  const int kmax = batch_kmax(b->dtype, b->tile);
  if (k < 0 || k > kmax)
    return bfail(AC_ERR_INVALID, "k must be in 0..%d (0 = default) for tile %d", kmax, b->tile);
  if (k != b->k) release_graph(b);
  b->k = k;
  b->cur_n.clear();
  return AC_OK;
}

extern "C" int ac_batch_set_tile(ac_batch *b, int32_t tile) {
  if (!b) return bfail(AC_ERR_INVALID, "batch is NULL");
  if (tile < 0 || tile > 1) return bfail(AC_ERR_INVALID, "tile must be 0 or 1");
  if (batch_kmax(b->dtype, tile) == 0)
    return bfail(AC_ERR_UNSUPPORTED, "tile %d is offered for FP32 storage only", tile);
  if (b->k > batch_kmax(b->dtype, tile))
    return bfail(AC_ERR_UNSUPPORTED, "depth %d is not offered with tile %d", b->k, tile);
  if (tile != b->tile) release_graph(b);
  b->tile = tile;
  b->cur_n.clear();
  return AC_OK;
}

extern "C" int ac_batch_get_tile(ac_batch *b, int32_t *tile) {
  if (!b || !tile) return bfail(AC_ERR_INVALID, "NULL argument");
  *tile = b->tile;
  return AC_OK;
}

extern "C" int ac_batch_get_schedule(ac_batch *b, int32_t *k) {
  if (!b || !k) return bfail(AC_ERR_INVALID, "NULL argument");
  *k = b->k ? b->k : default_k(b->dtype);
  return AC_OK;
}

// Per-instance plan for n steps at depth k (the same launch-depth rule as
// ac_step: an even number of step-blocks whenever possible).
static int make_plans(ac_batch *b, const int64_t *n, int k) {
  b->odd.clear();
  int smax = 0;
  for (int i = 0; i < b->count; ++i) {
    if (n[i] < 0) return bfail(AC_ERR_INVALID, "instance %d: n must be >= 0", i);
    if (n[i] > (int64_t)1 << 30) return bfail(AC_ERR_INVALID, "instance %d: n too large", i);
    std::vector<int> dep;
    bool even = true;
    if (n[i] > 0) even = ac_plan_depths(n[i], k, dep);
    BInst &in = b->h_inst[i];
    in.S = (int)dep.size();
    in.k = k;
    in.tail_start = std::max(0, in.S - 4);
    for (int q = 0; q < 4; ++q) in.tail[q] = 1;
    for (int s = in.tail_start; s < in.S; ++s) in.tail[s - in.tail_start] = dep[s];
    for (int s = 0; s < in.tail_start; ++s)
      if (dep[s] != k) return bfail(AC_ERR_INVALID, "internal: unexpected plan shape");
    if (!even) b->odd.push_back(i);
    smax = std::max(smax, in.S);
  }
  b->total_tickets = (long long)smax * (long long)b->h_items.size();
  BC_CUDA(cudaStreamSynchronize(b->stream));
  BC_CUDA(cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(BInst) * b->count, cudaMemcpyHostToDevice));
  return AC_OK;
}

static int enqueue(ac_batch *b) {
  BC_CUDA(cudaMemsetAsync(b->d_progress, 0, sizeof(int) * b->h_items.size(), b->stream));
  BC_CUDA(cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned long long), b->stream));
  int grid = 0;
  if (b->total_tickets > 0) {
    cudaError_t e = batch2d_launch(b->dtype, b->tile, b->d_inst, b->d_items, (int)b->h_items.size(),
                                   b->tile ? b->d_maps_wide : b->d_maps, b->d_progress, b->d_ticket,
                                   b->total_tickets,
                                   b->d_status, b->wait_limit, b->num_sms, b->stream, &grid);
    if (e != cudaSuccess) return bfail(AC_ERR_CUDA, "batched launch failed: %s", cudaGetErrorString(e));
    ++b->launches;
  }
  const size_t es = ac_elem_size(b->dtype);
  for (int i : b->odd) {
    const ac_grid_desc &d = b->d[i];
    BC_CUDA(cudaMemcpy2DAsync(b->phi[i], d.pitch_x * es, b->ws[i], d.pitch_x * es, d.nx * es,
                              (size_t)d.ny, cudaMemcpyDeviceToDevice, b->stream));
  }
  return AC_OK;
}

extern "C" int ac_batch_step(ac_batch *b, const int64_t *n_per_instance) {
  if (!b || !n_per_instance) return bfail(AC_ERR_INVALID, "NULL argument");
  const int k = b->k ? b->k : default_k(b->dtype);
  int rc = build_items(b, k);
  if (rc) return rc;
  const bool same = b->cur_n.size() == (size_t)b->count &&
                    std::equal(b->cur_n.begin(), b->cur_n.end(), n_per_instance);
  if (!same) {
    release_graph(b);
    rc = make_plans(b, n_per_instance, k);
    if (rc) return rc;
    b->cur_n.assign(n_per_instance, n_per_instance + b->count);
  }
  if (!b->use_graph || b->stream == nullptr) return enqueue(b);
  if (!b->graph) {
    BC_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
    const int64_t before = b->launches;
    rc = enqueue(b);
    b->graph_launches = b->launches - before;
    b->launches = before;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return bfail(AC_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return bfail(AC_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e)); }
  }
  BC_CUDA(cudaGraphLaunch(b->graph, b->stream));
  b->launches += b->graph_launches;
  return AC_OK;
}

extern "C" int ac_batch_set_graph(ac_batch *b, int32_t enable) {
  if (!b) return bfail(AC_ERR_INVALID, "batch is NULL");
  if (enable && b->stream == nullptr)
    return bfail(AC_ERR_UNSUPPORTED, "graph replay needs a non-default stream");
  b->use_graph = enable != 0;
  if (!b->use_graph) release_graph(b);
  return AC_OK;
}

extern "C" int ac_batch_observe(ac_batch *b, int32_t i, double out[3]) {
  if (!b || !out) return bfail(AC_ERR_INVALID, "NULL argument");
  if (i < 0 || i >= b->count) return bfail(AC_ERR_INVALID, "instance %d out of range", i);
  const ac_grid_desc &d = b->d[i];
  GridParams g;
  g.nx = d.nx; g.ny = d.ny; g.nz = d.nz; g.pitch = d.pitch_x;
  g.alpha = b->h_inst[i].alpha; g.beta = b->h_inst[i].beta; g.status = nullptr;
  cudaError_t e = launch_observe(b->dtype, g, b->phi[i], b->d_partials, b->d_out, b->stream);
  if (e != cudaSuccess) return bfail(AC_ERR_CUDA, "reduction launch failed: %s", cudaGetErrorString(e));
  b->launches += 2;
  BC_CUDA(cudaMemcpyAsync(b->h_out, b->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  BC_CUDA(cudaStreamSynchronize(b->stream));
  const double hd = d.h * d.h;
  out[0] = hd * (b->h_out[0] / (d.eps * d.eps) + 0.5 * b->h_out[1] / (d.h * d.h));
  out[1] = hd * b->h_out[2];
  out[2] = b->h_out[3];
  if (b->h_out[3] > 0) return bfail(AC_ERR_NONFINITE, "instance %d holds non-finite values", i);
  return AC_OK;
}

extern "C" int ac_batch_status(ac_batch *b) {
  if (!b) return bfail(AC_ERR_INVALID, "batch is NULL");
  int h = 0;
  BC_CUDA(cudaStreamSynchronize(b->stream));
  BC_CUDA(cudaMemcpy(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    BC_CUDA(cudaMemset(b->d_status, 0, sizeof(int)));
    return bfail(h == AC_ERR_TIMEOUT ? AC_ERR_TIMEOUT : AC_ERR_CUDA,
                 "the batched kernel reported status %d (a bounded wait expired)", h);
  }
  return AC_OK;
}

extern "C" int ac_batch_set_wait_limit(ac_batch *b, uint32_t polls) {
  if (!b) return bfail(AC_ERR_INVALID, "batch is NULL");
  b->wait_limit = polls ? polls : kDefaultWaitPolls;
  release_graph(b);
  return AC_OK;
}

extern "C" int ac_batch_launch_count(ac_batch *b, int64_t *out) {
  if (!b || !out) return bfail(AC_ERR_INVALID, "NULL argument");
  *out = b->launches;
  return AC_OK;
}

extern "C" int ac_batch_autotune(ac_batch *b, int64_t steps_per_trial) {
  if (!b) return bfail(AC_ERR_INVALID, "batch is NULL");
  if (steps_per_trial < 1) return bfail(AC_ERR_INVALID, "steps_per_trial must be >= 1");
  // back up every field, time each depth on the real instances, restore
  size_t total = 0;
  for (int i = 0; i < b->count; ++i) total += round256(bfield_bytes(b->d[i]));
  char *backup = nullptr;
  BC_CUDA(cudaMalloc(&backup, total));
  std::vector<size_t> offs;
  size_t off = 0;
  for (int i = 0; i < b->count; ++i) {
    offs.push_back(off);
    BC_CUDA(cudaMemcpyAsync(backup + off, b->phi[i], bfield_bytes(b->d[i]), cudaMemcpyDeviceToDevice, b->stream));
    off += round256(bfield_bytes(b->d[i]));
  }
  const bool graph_was = b->use_graph;
  b->use_graph = false;
  const int k_was = b->k, tile_was = b->tile;
  std::vector<int64_t> n(b->count, steps_per_trial);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best_k = default_k(b->dtype), best_tile = 0, rc = AC_OK;
  float best = 1e30f;
  std::vector<std::pair<int, int>> cand;  // (tile, k)
  for (int t = 0; t < 2; ++t)
    for (int k = 1; k <= batch_kmax(b->dtype, t); ++k) cand.push_back({t, k});
  for (size_t ci = 0; ci < cand.size() && rc == AC_OK; ++ci) {
    const int k = cand[ci].second;
    b->tile = cand[ci].first;
    b->k = k;
    b->cur_n.clear();
    rc = ac_batch_step(b, n.data());  // warm-up (builds items, plans)
    if (rc) break;
    cudaEventRecord(e0, b->stream);
    rc = ac_batch_step(b, n.data());
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_k = k; best_tile = b->tile; }
    for (int i = 0; i < b->count; ++i)
      cudaMemcpyAsync(b->phi[i], backup + offs[i], bfield_bytes(b->d[i]), cudaMemcpyDeviceToDevice, b->stream);
  }
  cudaStreamSynchronize(b->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(backup);
  b->use_graph = graph_was;
  b->k = rc == AC_OK ? best_k : k_was;
  b->tile = rc == AC_OK ? best_tile : tile_was;
  b->cur_n.clear();
  release_graph(b);
  return rc;
}

namespace ac {
cudaError_t batch2d_launch(int dtype, int tile, const BInst *insts, const BItem *items, int n_items,
                           const CUtensorMap *maps, int *progress, unsigned long long *ticket,
                           long long total, int *status, uint32_t wait_limit, int num_sms,
                           cudaStream_t s, int *grid_out) {
  if (batch_kmax(dtype, tile) == 0) return cudaErrorInvalidValue;
  switch (dtype) {
    case AC_F64: return batch2d_launch_f64(insts, items, n_items, maps, progress, ticket, total, status, wait_limit, num_sms, s, grid_out);
    case AC_F32:
      if (tile == 1)
        return batch2d_launch_f32_wide(insts, items, n_items, maps, progress, ticket, total, status, wait_limit, num_sms, s, grid_out);
      return batch2d_launch_f32(insts, items, n_items, maps, progress, ticket, total, status, wait_limit, num_sms, s, grid_out);
    case AC_F16S: return batch2d_launch_f16(insts, items, n_items, maps, progress, ticket, total, status, wait_limit, num_sms, s, grid_out);
  }
  return cudaErrorInvalidValue;
}
}  // namespace ac
