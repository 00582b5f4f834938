// C ABI of the Allen-Cahn stepper: validation, contexts, launch planning,
// reductions, initial conditions, autotuning and CUDA-graph replay.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ctx.h"

using namespace ac;

// ---------------------------------------------------------------- errors --
static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

namespace ac {
int set_error(int code, const char *msg) {
  g_err = msg;
  return code;
}

cudaError_t kernel_setup(KernelSetup &ks, const void *func, int threads, int smem, int *occ,
                         int carveout) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < kSetupDevices;
  if (cached) {
    const int v = ks.occ[dev].load(std::memory_order_acquire);
    if (v > 0) {
      *occ = v;
      return cudaSuccess;
    }
  }
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (cached) {
    const int v = ks.occ[dev].load(std::memory_order_relaxed);
    if (v > 0) {
      *occ = v;
      return cudaSuccess;
    }
  }
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (carveout >= 0) {
    e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    if (e != cudaSuccess) return e;
  }
  int n = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, smem);
  if (e != cudaSuccess) return e;
  n = n > 1 ? n : 1;
  if (cached) ks.occ[dev].store(n, std::memory_order_release);
  *occ = n;
  return cudaSuccess;
}
}  // namespace ac

#define AC_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(AC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
  } while (0)

// ----------------------------------------------------------- tensor maps --

EncodeTiledFn ac_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

size_t ac_elem_size(int dtype) { return dtype == AC_F64 ? 8 : dtype == AC_F32 ? 4 : 2; }

CUtensorMapDataType ac_tmap_type(int dtype) {
  return dtype == AC_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
         : dtype == AC_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
}

int ac_validate_desc(const ac_grid_desc *d) {
  if (!d) return fail(AC_ERR_INVALID, "descriptor is NULL");
  if (d->ndim != 2 && d->ndim != 3) return fail(AC_ERR_INVALID, "ndim must be 2 or 3 (got %d)", d->ndim);
  if (d->dtype != AC_F64 && d->dtype != AC_F32 && d->dtype != AC_F16S)
    return fail(AC_ERR_INVALID, "unknown dtype %d", d->dtype);
  if (d->nx < 1 || d->ny < 1 || d->nz < 1)
    return fail(AC_ERR_INVALID, "grid sizes must be >= 1 (got %lld x %lld x %lld)",
                (long long)d->nx, (long long)d->ny, (long long)d->nz);
  if (d->ndim == 2 && d->nz != 1) return fail(AC_ERR_INVALID, "2D grids need nz == 1");
  const int64_t lim = (int64_t)1 << 30;
  if (d->nx >= lim || d->ny >= lim || d->nz >= lim || d->pitch_x >= lim)
    return fail(AC_ERR_INVALID, "grid extent too large (each axis and pitch < 2^30)");
  if (d->pitch_x < d->nx) return fail(AC_ERR_INVALID, "pitch_x < nx");
  if ((d->pitch_x * (int64_t)ac_elem_size(d->dtype)) % 16 != 0)
    return fail(AC_ERR_INVALID, "pitch_x * element size must be a multiple of 16 bytes");
  // eps = +inf is the heat equation (alpha = 0); NaN and eps <= 0 are not
  if (!(std::isfinite(d->h) && d->h > 0) || !(d->eps > 0) ||
      !(std::isfinite(d->dt) && d->dt > 0))
    return fail(AC_ERR_INVALID, "h and dt must be finite and > 0, eps > 0 (or +inf)");
  const double lap_limit = d->h * d->h / (2.0 * d->ndim);
  if (d->dt > lap_limit * (1.0 + 1e-12))
    return fail(AC_ERR_INVALID, "dt = %g exceeds the explicit stability limit h^2/(2 ndim) = %g",
                d->dt, lap_limit);
  if (d->dt > d->eps * d->eps * (1.0 + 1e-12))
    return fail(AC_ERR_INVALID, "dt = %g exceeds eps^2 = %g (reaction step alpha > 1)", d->dt,
                d->eps * d->eps);
  return AC_OK;
}

static size_t field_bytes(const ac_grid_desc *d) {
  return (size_t)d->pitch_x * (size_t)d->ny * (size_t)d->nz * ac_elem_size(d->dtype);
}

extern "C" int ac_workspace_bytes(const ac_grid_desc *desc, size_t *out) {
  int rc = ac_validate_desc(desc);
  if (rc) return rc;
  if (!out) return fail(AC_ERR_INVALID, "out is NULL");
  *out = field_bytes(desc);
  return AC_OK;
}

static int encode_map(ac_ctx *c, void *base, int kind, int k, int tile, CUtensorMap *out) {
  EncodeTiledFn fn = ac_encode_fn();
  if (!fn) return fail(AC_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  const ac_grid_desc &d = c->d;
  const size_t es = ac_elem_size(d.dtype);
  cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  cuuint64_t strides[2] = {(cuuint64_t)(d.pitch_x * es), (cuuint64_t)(d.pitch_x * d.ny * es)};
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  cuuint32_t rank;
  if (kind == 2) {
    Stream2DGeom gm = stream2d_geom(d.dtype, k, tile);
    box[0] = gm.box_x; box[1] = gm.box_y; box[2] = 1;
    rank = 2;
  } else {
    Stream3DGeom gm = stream3d_geom(d.dtype, k, tile);
    box[0] = gm.box_x; box[1] = gm.box_y; box[2] = 1;
    rank = 3;
  }
  CUresult r = fn(out, ac_tmap_type(d.dtype), rank, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(AC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return AC_OK;
}

static int ensure_maps(ac_ctx *c, int k, int tile) {
  MapPair &m = c->maps[tile][k];
  if (m.valid) return AC_OK;
  const int kind = c->d.ndim;
  int rc = encode_map(c, c->phi, kind, k, tile, &m.phi);
  if (rc) return rc;
  rc = encode_map(c, c->ws, kind, k, tile, &m.ws);
  if (rc) return rc;
  m.valid = true;
  return AC_OK;
}

static void release_graph(ac_ctx *c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  c->graph_n = -1;
}

extern "C" int ac_create(const ac_grid_desc *desc, void *phi_dev, void *workspace_dev,
                         void *cuda_stream, ac_ctx **out) {
  int rc = ac_validate_desc(desc);
  if (rc) return rc;
  if (!out) return fail(AC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!phi_dev || !workspace_dev) return fail(AC_ERR_INVALID, "phi and workspace must be non-NULL");
  if (((uintptr_t)phi_dev | (uintptr_t)workspace_dev) & 15)
    return fail(AC_ERR_INVALID, "phi and workspace must be 16-byte aligned");
  const size_t bytes = field_bytes(desc);
  const uintptr_t a = (uintptr_t)phi_dev, b = (uintptr_t)workspace_dev;
  if (a < b + bytes && b < a + bytes) return fail(AC_ERR_INVALID, "phi and workspace overlap");
  cudaPointerAttributes pa{}, pb{};
  if (cudaPointerGetAttributes(&pa, phi_dev) != cudaSuccess ||
      cudaPointerGetAttributes(&pb, workspace_dev) != cudaSuccess ||
      (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) ||
      (pb.type != cudaMemoryTypeDevice && pb.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return fail(AC_ERR_INVALID, "phi and workspace must be CUDA device memory");
  }
  ac_ctx *c = new (std::nothrow) ac_ctx();
  if (!c) return fail(AC_ERR_NOMEM, "out of host memory");
  c->d = *desc;
  c->phi = phi_dev;
  c->ws = workspace_dev;
  c->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  c->gp.nx = desc->nx;
  c->gp.ny = desc->ny;
  c->gp.nz = desc->nz;
  c->gp.pitch = desc->pitch_x;
  c->gp.alpha = desc->dt / (desc->eps * desc->eps);
  c->gp.beta = desc->dt / (desc->h * desc->h);
  cudaError_t e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_partials, sizeof(double) * 4 * kReduceBlocks);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_out, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_out, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) {
    cudaFree(c->d_status); cudaFree(c->d_partials); cudaFree(c->d_out); cudaFreeHost(c->h_out);
    delete c;
    cudaGetLastError();
    return fail(AC_ERR_NOMEM, "internal allocation failed: %s", cudaGetErrorString(e));
  }
  c->gp.status = c->d_status;
  *out = c;
  return AC_OK;
}

extern "C" int ac_destroy(ac_ctx *c) {
  if (!c) return AC_OK;
  cudaStreamSynchronize(c->stream);
  release_graph(c);
  cudaFree(c->d_status);
  cudaFree(c->d_partials);
  cudaFree(c->d_out);
  cudaFreeHost(c->h_out);
  delete c;
  return AC_OK;
}

// ------------------------------------------------------------- schedules --
static bool schedule_ok(const ac_ctx *c, int variant, int k, int tile = 0) {
  if (variant == AC_VARIANT_DIRECT) return k == 1;
  if (variant == AC_VARIANT_STREAM)
    return c->d.ndim == 2 ? stream2d_supported(c->d.dtype, k, tile)
                          : stream3d_supported(c->d.dtype, k, tile);
  return false;
}

// 2D FP32 grids from kWideStripCells cells on take the 8-cell strips at
// k = 6 by default: measured on GB300, 4096^2 runs at 1636 Gcell-updates/s
// (1712 graph-replayed) against 1573 for 4-cell strips at k = 5, 8192^2 at
// 2006 against 1841 (k = 4).  Below that the 240-column strips leave too few
// warps busy: 2048^2 runs at 876 with them against 1021 (k = 5) and 1090
// (k = 8) with 4-cell strips, 1024^2 at 236 against 365 (k = 5), so grids
// from kMidCells take 4-cell strips at k = 5, smaller ones k = 4 (bound by
// launch latency; 512 grids of 64^2 .. 1024^2 stepped one by one: 3.2 s
// against 4.5 s with the wide strips).
constexpr double kWideStripCells = 4096.0 * 4096.0;
constexpr double kMidCells = 1024.0 * 1024.0;

static bool wide_default(const ac_grid_desc *d) {
  return d->ndim == 2 && d->dtype == AC_F32 && (double)d->nx * (double)d->ny >= kWideStripCells;
}

// 2D FP16-storage grids from this many cells take k = 6 (measured on GB300:
// 1827 / 2196 Gcell-updates/s at 4096^2 / 8192^2 against 1657 / 1906 at
// k = 4; at 2048^2 and below k = 4 or 5 is faster).
constexpr double kDeepHalfCells = 4096.0 * 4096.0;

int ac_default_depth(const ac_grid_desc *d) {
  // FP64 is bound by the GPU's FP64 rate, where the redundant halo work of
  // temporal blocking costs more than the memory traffic it saves: one step
  // per launch.  FP32 / FP16 storage stream with k > 1 (measured best on
  // GB300: 3D k = 2; 2D k = 4, or 6 with the 8-cell FP32 strips and for
  // large FP16-storage grids).
  if (d->dtype == AC_F64) return 1;
  if (d->ndim == 3) return 2;
  const double cells = (double)d->nx * (double)d->ny;
  if (d->dtype == AC_F16S && cells >= kDeepHalfCells) return 6;
  if (wide_default(d)) return 6;
  return d->dtype == AC_F32 && cells >= kMidCells ? 5 : 4;
}

static void default_schedule(const ac_ctx *c, int *variant, int *k) {
  *variant = c->d.dtype == AC_F64 ? AC_VARIANT_DIRECT : AC_VARIANT_STREAM;
  *k = ac_default_depth(&c->d);
  if (*variant == AC_VARIANT_STREAM && !schedule_ok(c, *variant, *k, 0) &&
      !schedule_ok(c, *variant, *k, 1))
    *k = 1;
}

static void effective_schedule(const ac_ctx *c, int *variant, int *k) {
  if (c->variant != AC_VARIANT_AUTO) { *variant = c->variant; *k = c->k; return; }
  if (c->tuned_variant) { *variant = c->tuned_variant; *k = c->tuned_k; return; }
  default_schedule(c, variant, k);
}

// Default 3D tile per storage type and depth, measured on GB300 (512^3
// FP32 / FP16, 256^3 FP64): two rows per thread at 128 x 32 (tile 0) for
// k <= 2 (FP16 storage at k <= 2: two CTAs per SM, tile 1, 1150 against
// 1114 Gcell-updates/s at k = 2); k = 3 needs the register room of four rows
// per thread with half the threads (tile 2).
static int default_tile(const ac_ctx *c, int k) {
  // 2D FP32 grids from 4096^2 cells on: strips of 8 cells per lane wherever
  // they are offered (k <= 6; see kWideStripCells)
  if (c->d.ndim == 2) return wide_default(&c->d) && k <= 6 ? 1 : 0;
  if (c->d.dtype == AC_F64) return k == 1 ? 0 : 2;
  if (c->d.dtype == AC_F16S) return k <= 2 ? 1 : 0;
  return k == 3 ? 2 : 0;
}

// The tile of a streaming launch: the user's, else the autotuner's (when it
// is available at this depth), else the default.
static int effective_tile(const ac_ctx *c, int variant, int k) {
  if (variant != AC_VARIANT_STREAM) return 0;
  if (c->tile != AC_TILE_AUTO && schedule_ok(c, variant, k, c->tile)) return c->tile;
  if (c->tuned_variant && schedule_ok(c, variant, k, c->tuned_tile)) return c->tuned_tile;
  const int t = default_tile(c, k);
  return schedule_ok(c, variant, k, t) ? t : 0;
}

extern "C" int ac_set_schedule(ac_ctx *c, int32_t variant, int32_t k) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  if (variant == AC_VARIANT_AUTO && k == 0) {
    c->variant = AC_VARIANT_AUTO;
    c->k = 0;
    return AC_OK;
  }
  if (k < 1 || k > AC_MAX_K) return fail(AC_ERR_INVALID, "k must be in 1..%d", AC_MAX_K);
  if (variant != AC_VARIANT_DIRECT && variant != AC_VARIANT_STREAM)
    return fail(AC_ERR_INVALID, "unknown variant %d", variant);
  if (!schedule_ok(c, variant, k))
    return fail(AC_ERR_UNSUPPORTED, "variant %d with k = %d is not available for ndim %d dtype %d",
                variant, k, c->d.ndim, c->d.dtype);
  c->variant = variant;
  c->k = k;
  return AC_OK;
}

extern "C" int ac_set_tile(ac_ctx *c, int32_t tile) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  if (tile == AC_TILE_AUTO) { c->tile = AC_TILE_AUTO; return AC_OK; }
  const int ntiles = c->d.ndim == 3 ? AC_NUM_TILES_3D : AC_NUM_TILES_2D;
  if (tile < 0 || tile >= ntiles) return fail(AC_ERR_INVALID, "tile must be in 0..%d", ntiles - 1);
  if (c->d.ndim == 2 && tile != 0 && !stream2d_supported(c->d.dtype, 1, tile))
    return fail(AC_ERR_UNSUPPORTED, "2D tile %d is offered for FP32 storage only", tile);
  c->tile = tile;
  return AC_OK;
}

extern "C" int ac_get_tile(ac_ctx *c, int32_t *tile) {
  if (!c || !tile) return fail(AC_ERR_INVALID, "NULL argument");
  int v, kk;
  effective_schedule(c, &v, &kk);
  *tile = effective_tile(c, v, kk);
  return AC_OK;
}

extern "C" int ac_get_schedule(ac_ctx *c, int32_t *variant, int32_t *k) {
  if (!c || !variant || !k) return fail(AC_ERR_INVALID, "NULL argument");
  int v, kk;
  effective_schedule(c, &v, &kk);
  *variant = v;
  *k = kk;
  return AC_OK;
}

// ------------------------------------------------------------- stepping ---
// Depths of the launches for n steps at depth k: as many k as fit, then the
// remainder; an odd launch count is made even by splitting a launch of
// depth >= 2, so that the result lands back in phi.  Returns false if the
// count stays odd (all depths 1): the caller then copies ws -> phi.
bool ac_plan_depths(int64_t n, int k, std::vector<int> &depths) {
  depths.clear();
  for (int64_t i = 0; i < n / k; ++i) depths.push_back(k);
  if (n % k) depths.push_back((int)(n % k));
  if (depths.size() % 2 == 0) return true;
  for (size_t i = depths.size(); i-- > 0;) {
    if (depths[i] >= 2) {
      const int a = depths[i] / 2, b = depths[i] - a;
      depths[i] = b;
      depths.insert(depths.begin() + i + 1, a);
      return true;
    }
  }
  return false;
}

static int issue_steps(ac_ctx *c, int64_t n, int variant, int k, int tile) {
  std::vector<int> depths;
  const bool even = variant == AC_VARIANT_DIRECT ? (n % 2 == 0) : ac_plan_depths(n, k, depths);
  if (variant == AC_VARIANT_DIRECT) depths.assign((size_t)n, 1);
  bool src_is_phi = true;
  for (int dep : depths) {
    void *src = src_is_phi ? c->phi : c->ws;
    void *dst = src_is_phi ? c->ws : c->phi;
    cudaError_t e;
    if (variant == AC_VARIANT_DIRECT) {
      e = launch_direct(c->d.ndim, c->d.dtype, c->gp, src, dst, c->stream);
    } else {
      // a remainder depth the tile does not offer runs on tile 0
      const int tl = schedule_ok(c, variant, dep, tile) ? tile : 0;
      int rc = ensure_maps(c, dep, tl);
      if (rc) return rc;
      const CUtensorMap *m = src_is_phi ? &c->maps[tl][dep].phi : &c->maps[tl][dep].ws;
      e = c->d.ndim == 2 ? launch_stream2d(c->d.dtype, dep, tl, c->gp, m, dst, c->num_sms, c->stream)
                         : launch_stream3d(c->d.dtype, dep, tl, c->gp, m, dst, c->num_sms, c->stream);
    }
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "stencil launch failed: %s", cudaGetErrorString(e));
    ++c->launches;
    src_is_phi = !src_is_phi;
  }
  if (!even) {
    const size_t es = ac_elem_size(c->d.dtype);
    AC_CUDA(cudaMemcpy2DAsync(c->phi, c->d.pitch_x * es, c->ws, c->d.pitch_x * es, c->d.nx * es,
                              (size_t)(c->d.ny * c->d.nz), cudaMemcpyDeviceToDevice, c->stream));
  }
  return AC_OK;
}

extern "C" int ac_step(ac_ctx *c, int64_t n) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  if (n < 0) return fail(AC_ERR_INVALID, "n must be >= 0");
  if (n == 0) return AC_OK;
  int variant, k;
  effective_schedule(c, &variant, &k);
  const int tile = effective_tile(c, variant, k);
  if (!c->use_graph || c->stream == nullptr) return issue_steps(c, n, variant, k, tile);
  // graph replay: capture the launch sequence for this (n, schedule) once
  if (c->graph_exec == nullptr || c->graph_n != n || c->graph_variant != variant ||
      c->graph_k != k || c->graph_tile != tile) {
    release_graph(c);
    AC_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    const int64_t before = c->launches;
    int rc = issue_steps(c, n, variant, k, tile);
    c->graph_launches = c->launches - before;
    c->launches = before;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { c->graph_exec = nullptr; return fail(AC_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e)); }
    c->graph_n = n;
    c->graph_variant = variant;
    c->graph_k = k;
    c->graph_tile = tile;
  }
  AC_CUDA(cudaGraphLaunch(c->graph_exec, c->stream));
  c->launches += c->graph_launches;
  return AC_OK;
}

// ----------------------------------------------------------- reductions ---
static int observe(ac_ctx *c, double out[4]) {
  cudaError_t e = launch_observe(c->d.dtype, c->gp, c->phi, c->d_partials, c->d_out, c->stream);
  if (e != cudaSuccess) return fail(AC_ERR_CUDA, "reduction launch failed: %s", cudaGetErrorString(e));
  c->launches += 2;
  AC_CUDA(cudaMemcpyAsync(c->h_out, c->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  AC_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(out, c->h_out, 4 * sizeof(double));
  return AC_OK;
}

static double cell_measure(const ac_ctx *c) {
  return c->d.ndim == 3 ? c->d.h * c->d.h * c->d.h : c->d.h * c->d.h;
}

extern "C" int ac_observe(ac_ctx *c, double res[3]) {
  if (!c || !res) return fail(AC_ERR_INVALID, "NULL argument");
  double s[4];
  int rc = observe(c, s);
  if (rc) return rc;
  const double hd = cell_measure(c);
  res[0] = hd * (s[0] / (c->d.eps * c->d.eps) + 0.5 * s[1] / (c->d.h * c->d.h));
  res[1] = hd * s[2];
  res[2] = s[3];
  if (s[3] > 0) return fail(AC_ERR_NONFINITE, "phi holds %.0f non-finite values", s[3]);
  return AC_OK;
}

extern "C" int ac_energy(ac_ctx *c, double *out) {
  if (!out) return fail(AC_ERR_INVALID, "out is NULL");
  double r[3];
  int rc = ac_observe(c, r);
  if (rc && rc != AC_ERR_NONFINITE) return rc;
  *out = r[0];
  return rc;
}

extern "C" int ac_phase_volume(ac_ctx *c, double *out) {
  if (!out) return fail(AC_ERR_INVALID, "out is NULL");
  double r[3];
  int rc = ac_observe(c, r);
  if (rc && rc != AC_ERR_NONFINITE) return rc;
  *out = r[1];
  return rc;
}

extern "C" int ac_status(ac_ctx *c) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  int h = 0;
  AC_CUDA(cudaStreamSynchronize(c->stream));
  AC_CUDA(cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    AC_CUDA(cudaMemset(c->d_status, 0, sizeof(int)));
    return fail(AC_ERR_TIMEOUT, "a bounded device wait expired (status %d)", h);
  }
  return AC_OK;
}

// ---------------------------------------------------- initial conditions --
extern "C" int ac_init_sphere(ac_ctx *c, double lx, double ly, double lz, double cx, double cy,
                              double cz, double r0) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  if (!std::isfinite(r0)) return fail(AC_ERR_INVALID, "r0 must be finite");
  const double lo[3] = {lx, ly, lz}, ce[3] = {cx, cy, cz};
  cudaError_t e = launch_init_sphere(c->d.dtype, c->gp, c->phi, c->d.h, lo, ce, r0, c->d.eps, c->stream);
  if (e != cudaSuccess) return fail(AC_ERR_CUDA, "init launch failed: %s", cudaGetErrorString(e));
  ++c->launches;
  return AC_OK;
}

extern "C" int ac_init_shape(ac_ctx *c, int32_t kind, double lx, double ly, double lz, double p0,
                             double p1) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  if (kind != AC_SHAPE_DUMBBELL && kind != AC_SHAPE_STAR && kind != AC_SHAPE_TORUS)
    return fail(AC_ERR_INVALID, "unknown shape %d", kind);
  if (!std::isfinite(lx) || !std::isfinite(ly) || !std::isfinite(lz) || !std::isfinite(p0) ||
      !std::isfinite(p1))
    return fail(AC_ERR_INVALID, "shape parameters must be finite");
  const double lo[3] = {lx, ly, lz};
  cudaError_t e = launch_init_shape(c->d.dtype, c->gp, c->phi, kind, c->d.ndim, c->d.h, lo, p0, p1,
                                    c->d.eps, c->stream);
  if (e != cudaSuccess) return fail(AC_ERR_CUDA, "init launch failed: %s", cudaGetErrorString(e));
  ++c->launches;
  return AC_OK;
}

extern "C" int ac_init_random(ac_ctx *c, uint64_t seed, double amplitude) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  if (!std::isfinite(amplitude)) return fail(AC_ERR_INVALID, "amplitude must be finite");
  cudaError_t e = launch_init_random(c->d.dtype, c->gp, c->phi, seed, amplitude, c->stream);
  if (e != cudaSuccess) return fail(AC_ERR_CUDA, "init launch failed: %s", cudaGetErrorString(e));
  ++c->launches;
  return AC_OK;
}

// -------------------------------------------------------------- autotune --
namespace {
// Tuning results are keyed by grid kind, storage type, size class (log2 of
// the cell count) and the device model (name and SM count, so that a cache
// file carries over between processes and between GPUs of the same model).
struct TuneKey {
  int ndim, dtype, cls;
  std::string device;
  int graph;  // timed as graph replay (1) or as launches (0)
  bool operator<(const TuneKey &o) const {
    return std::tie(ndim, dtype, cls, device, graph) < std::tie(o.ndim, o.dtype, o.cls, o.device, o.graph);
  }
};
std::mutex g_tune_mu;
struct TuneChoice {
  int variant, k, tile;
};
std::map<TuneKey, TuneChoice> g_tune_cache;
std::string g_tune_file;  // optional on-disk cache (empty: none)

std::string device_key(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
  std::string name(prop.name);
  for (char &ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  return name + "_sm" + std::to_string(prop.multiProcessorCount);
}

// File format, one entry per line:
//   ac-tune-v2 <ndim> <dtype> <size class> <device> <graph> <variant> <k> <tile>
// (lines of the earlier "ac-tune-v1" form, without <graph>, are choices
// timed as launches).  Unreadable lines are skipped; the last entry for a
// key wins.
bool file_lookup(const TuneKey &key, TuneChoice *out) {
  if (g_tune_file.empty()) return false;
  FILE *f = fopen(g_tune_file.c_str(), "r");
  if (!f) return false;
  char line[512], tag[32], dev[256];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    int nd, dt, cls, gr, v, k, t;
    if (sscanf(line, "%31s", tag) != 1) continue;
    if (strcmp(tag, "ac-tune-v2") == 0) {
      if (sscanf(line, "%31s %d %d %d %255s %d %d %d %d", tag, &nd, &dt, &cls, dev, &gr, &v, &k, &t) != 9)
        continue;
    } else if (strcmp(tag, "ac-tune-v1") == 0) {
      if (sscanf(line, "%31s %d %d %d %255s %d %d %d", tag, &nd, &dt, &cls, dev, &v, &k, &t) != 8) continue;
      gr = 0;
    } else {
      continue;
    }
    if (nd == key.ndim && dt == key.dtype && cls == key.cls && key.device == dev && gr == key.graph) {
      *out = TuneChoice{v, k, t};
      found = true;
    }
  }
  fclose(f);
  return found;
}

void file_append(const TuneKey &key, const TuneChoice &c) {
  if (g_tune_file.empty()) return;
  FILE *f = fopen(g_tune_file.c_str(), "a");
  if (!f) return;
  fprintf(f, "ac-tune-v2 %d %d %d %s %d %d %d %d\n", key.ndim, key.dtype, key.cls, key.device.c_str(),
          key.graph, c.variant, c.k, c.tile);
  fclose(f);
}
}  // namespace

static int size_class(const ac_grid_desc &d) {
  const double cells = (double)d.nx * (double)d.ny * (double)d.nz;
  return (int)std::floor(std::log2(std::max(1.0, cells)));
}

extern "C" int ac_autotune(ac_ctx *c, int64_t steps_per_trial) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  if (steps_per_trial < 1) return fail(AC_ERR_INVALID, "steps_per_trial must be >= 1");
  const TuneKey key{c->d.ndim, c->d.dtype, size_class(c->d), device_key(c->device),
                    (c->use_graph && c->stream != nullptr) ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    TuneChoice fc;
    if (it == g_tune_cache.end() && file_lookup(key, &fc) && schedule_ok(c, fc.variant, fc.k, fc.tile))
      it = g_tune_cache.emplace(key, fc).first;
    if (it != g_tune_cache.end()) {
      c->tuned_variant = it->second.variant;
      c->tuned_k = it->second.k;
      c->tuned_tile = it->second.tile;
      return AC_OK;
    }
  }
  // candidates: the direct kernel and every streaming depth and tile
  std::vector<TuneChoice> cand;
  cand.push_back({AC_VARIANT_DIRECT, 1, 0});
  for (int k = 1; k <= AC_MAX_K; ++k)
    for (int tile = 0; tile < (c->d.ndim == 3 ? AC_NUM_TILES_3D : AC_NUM_TILES_2D); ++tile)
      if (schedule_ok(c, AC_VARIANT_STREAM, k, tile)) cand.push_back({AC_VARIANT_STREAM, k, tile});
  const size_t bytes = field_bytes(&c->d);
  void *backup = nullptr;
  AC_CUDA(cudaMalloc(&backup, bytes));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = AC_OK;
  float best = 1e30f;
  TuneChoice best_c = cand.front();
  cudaMemcpyAsync(backup, c->phi, bytes, cudaMemcpyDeviceToDevice, c->stream);
  // A context that replays its steps through a CUDA graph has them timed the
  // same way (small grids are bound by launch overhead, which graphs remove).
  const bool graphed = c->use_graph && c->stream != nullptr;
  for (auto &cd : cand) {
    // steps rounded to a multiple of 2k so every candidate runs full passes
    const int64_t n = std::max<int64_t>(2 * cd.k, steps_per_trial / (2 * cd.k) * (2 * cd.k));
    rc = issue_steps(c, 2 * cd.k, cd.variant, cd.k, cd.tile);  // warm-up
    if (rc) break;
    cudaGraphExec_t gx = nullptr;
    if (graphed) {
      cudaGraph_t gr = nullptr;
      const int64_t before = c->launches;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        rc = fail(AC_ERR_CUDA, "stream capture failed");
        break;
      }
      rc = issue_steps(c, n, cd.variant, cd.k, cd.tile);
      const cudaError_t ec = cudaStreamEndCapture(c->stream, &gr);
      c->launches = before;
      if (rc == AC_OK && ec != cudaSuccess) rc = fail(AC_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(ec));
      if (rc == AC_OK && cudaGraphInstantiate(&gx, gr, 0) != cudaSuccess)
        rc = fail(AC_ERR_CUDA, "graph instantiate failed");
      if (gr) cudaGraphDestroy(gr);
      if (rc == AC_OK && cudaGraphLaunch(gx, c->stream) != cudaSuccess)  // warm-up replay
        rc = fail(AC_ERR_CUDA, "graph launch failed");
      if (rc) {
        if (gx) cudaGraphExecDestroy(gx);
        break;
      }
    }
    cudaEventRecord(e0, c->stream);
    if (graphed) {
      if (cudaGraphLaunch(gx, c->stream) != cudaSuccess) rc = fail(AC_ERR_CUDA, "graph launch failed");
    } else {
      rc = issue_steps(c, n, cd.variant, cd.k, cd.tile);
    }
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    if (gx) cudaGraphExecDestroy(gx);
    if (rc) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const float per_step = ms / (float)n;
    if (per_step < best) { best = per_step; best_c = cd; }
    cudaMemcpyAsync(c->phi, backup, bytes, cudaMemcpyDeviceToDevice, c->stream);
  }
  cudaStreamSynchronize(c->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(backup);
  if (rc) return rc;
  c->tuned_variant = best_c.variant;
  c->tuned_k = best_c.k;
  c->tuned_tile = best_c.tile;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best_c;
  file_append(key, best_c);
  return AC_OK;
}

extern "C" int ac_set_tune_cache(const char *path) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_file = path ? path : "";
  g_tune_cache.clear();
  return AC_OK;
}

extern "C" int ac_set_graph(ac_ctx *c, int32_t enable) {
  if (!c) return fail(AC_ERR_INVALID, "ctx is NULL");
  if (enable && c->stream == nullptr)
    return fail(AC_ERR_UNSUPPORTED, "graph replay needs a non-default stream");
  c->use_graph = enable != 0;
  if (!c->use_graph) release_graph(c);
  return AC_OK;
}

// Allocation-free observation: no context, no cudaMalloc/cudaFree, no pinned
// or pageable host buffers; the partial sums live in the library's fixed
// module-global array (see k_reduce.cu) and the results in the caller's
// device buffer.
extern "C" int ac_observe_noalloc(const ac_grid_desc *desc, const void *phi_dev, void *cuda_stream,
                                  double *out_dev) {
  int rc = ac_validate_desc(desc);
  if (rc) return rc;
  if (!phi_dev || !out_dev) return fail(AC_ERR_INVALID, "phi_dev and out_dev must be non-NULL");
  if (((uintptr_t)phi_dev & 15) || ((uintptr_t)out_dev & 7))
    return fail(AC_ERR_INVALID, "phi_dev must be 16-byte and out_dev 8-byte aligned");
  const int64_t rows = desc->ny * desc->nz;
  if (rows > observe_noalloc_max_rows())
    return fail(AC_ERR_INVALID,
                "ac_observe_noalloc: ny * nz = %lld rows exceeds the fixed scratch limit of %lld "
                "rows (use ac_observe through a context instead)",
                (long long)rows, (long long)observe_noalloc_max_rows());
  GridParams g;
  g.nx = desc->nx;
  g.ny = desc->ny;
  g.nz = desc->nz;
  g.pitch = desc->pitch_x;
  g.alpha = desc->dt / (desc->eps * desc->eps);
  g.beta = desc->dt / (desc->h * desc->h);
  g.status = nullptr;
  const double hd = desc->ndim == 3 ? desc->h * desc->h * desc->h : desc->h * desc->h;
  cudaError_t e = launch_observe_noalloc(desc->dtype, g, phi_dev, hd, desc->eps, desc->h, out_dev,
                                         (cudaStream_t)cuda_stream);
  if (e != cudaSuccess)
    return fail(AC_ERR_CUDA, "ac_observe_noalloc launch failed: %s", cudaGetErrorString(e));
  return AC_OK;
}

extern "C" int ac_tc_gemm_bf16_n32(const void *a_dev, const void *b_dev, float *d_dev, int64_t m,
                                   int32_t k, void *cuda_stream) {
  if (!a_dev || !b_dev || !d_dev) return fail(AC_ERR_INVALID, "NULL operand");
  if (m < 128 || m % 128 || k < 16 || k > 512 || k % 16)
    return fail(AC_ERR_INVALID, "need m a multiple of 128 and k a multiple of 16 in [16, 512]");
  if (((uintptr_t)a_dev | (uintptr_t)b_dev | (uintptr_t)d_dev) & 15)
    return fail(AC_ERR_INVALID, "operands must be 16-byte aligned");
  // one status word per device, allocated on the device's first call
  static std::mutex mu;
  static int *status_of[kSetupDevices] = {nullptr};
  int dev = 0;
  AC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kSetupDevices) return fail(AC_ERR_UNSUPPORTED, "device index %d too large", dev);
  int *status = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!status_of[dev] && cudaMalloc(&status_of[dev], sizeof(int)) != cudaSuccess) {
      status_of[dev] = nullptr;
      cudaGetLastError();
      return fail(AC_ERR_NOMEM, "status word allocation failed");
    }
    status = status_of[dev];
  }
  cudaError_t e = launch_tc_gemm_n32(a_dev, b_dev, d_dev, m, k, status, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return fail(AC_ERR_CUDA, "tensor-core GEMM launch failed: %s", cudaGetErrorString(e));
  return AC_OK;
}

extern "C" int ac_launch_count(ac_ctx *c, int64_t *out) {
  if (!c || !out) return fail(AC_ERR_INVALID, "NULL argument");
  *out = c->launches;
  return AC_OK;
}

extern "C" const char *ac_last_error(void) { return g_err.c_str(); }

extern "C" const char *ac_version(void) { return "1.0.0 sm_103a"; }
