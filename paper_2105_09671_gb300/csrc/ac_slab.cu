// Slab decomposition of one grid along its slowest axis: the plan (host
// arithmetic only) and in-process slabs that each run the ordinary stepper
// on an extended slab, with halo planes refreshed between blocks of steps.
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "ctx.h"

using namespace ac;

static int sfail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_error(code, buf);
}

extern "C" int ac_slab_plan(int64_t extent, int32_t parts, int32_t halo, ac_slab_part *out) {
  if (!out) return sfail(AC_ERR_INVALID, "out is NULL");
  if (extent < 1 || parts < 1 || parts > extent)
    return sfail(AC_ERR_INVALID, "need 1 <= parts (%d) <= extent (%lld)", parts, (long long)extent);
  if (halo < 1) return sfail(AC_ERR_INVALID, "halo must be >= 1");
  const int64_t base = extent / parts, extra = extent % parts;
  if (parts > 1 && base < halo)
    return sfail(AC_ERR_INVALID, "a part would own %lld planes, fewer than the halo of %d",
                 (long long)base, halo);
  int64_t lo = 0;
  for (int32_t p = 0; p < parts; ++p) {
    const int64_t own = base + (p < extra ? 1 : 0);
    out[p].own_lo = lo;
    out[p].own_hi = lo + own;
    out[p].ext_lo = p > 0 ? lo - halo : 0;
    out[p].ext_hi = p + 1 < parts ? lo + own + halo : extent;
    lo += own;
  }
  return AC_OK;
}

struct SlabPart {
  ac_slab_part plan{};
  void *phi = nullptr, *ws = nullptr;
  ac_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;  // the part's own stream (several parts)
  cudaEvent_t done = nullptr;     // end of the part's block of steps
  int64_t graph_kernels = 0;  // kernels of this part in the captured graph
  int64_t extra = 0;          // correction of the context's own launch count
};

struct ac_slab {
  ac_grid_desc desc{};
  int parts = 0, halo = 0;
  size_t plane_bytes = 0;  // bytes per plane of the slow axis (3D: pitch * ny, 2D: pitch)
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;  // start of a block of steps on the slab's stream
  std::vector<SlabPart> part;
  bool fresh = false;      // halos hold their neighbours' current owned planes
  int64_t copies = 0;
  // graph replay of ac_slab_step: the sequence for (n, fresh at the start)
  bool use_graph = false;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_n = -1;
  bool graph_fresh = false;
  int64_t graph_copies = 0;
};

static void slab_release_graph(ac_slab *s) {
  if (s->graph) cudaGraphExecDestroy(s->graph);
  s->graph = nullptr;
  s->graph_n = -1;
}

static char *at(void *base, int64_t planes, size_t plane_bytes) {
  return static_cast<char *>(base) + (size_t)planes * plane_bytes;
}

static void slab_free(ac_slab *s) {
  slab_release_graph(s);
  for (SlabPart &p : s->part) {
    if (p.ctx) ac_destroy(p.ctx);
    cudaFree(p.phi);
    cudaFree(p.ws);
    if (p.done) cudaEventDestroy(p.done);
    if (p.stream) cudaStreamDestroy(p.stream);
  }
  if (s->fork) cudaEventDestroy(s->fork);
  delete s;
}

extern "C" int ac_slab_create(const ac_grid_desc *desc, int32_t parts, int32_t halo, void *cuda_stream,
                              ac_slab **out) {
  if (!out) return sfail(AC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int rc = ac_validate_desc(desc);
  if (rc) return rc;
  const bool d3 = desc->ndim == 3;
  const int64_t extent = d3 ? desc->nz : desc->ny;
  if (halo == 0) halo = 2 * ac_default_depth(desc);  // two full passes per block
  std::vector<ac_slab_part> plan(parts > 0 ? parts : 1);
  rc = ac_slab_plan(extent, parts, halo, plan.data());
  if (rc) return rc;
  ac_slab *s = new (std::nothrow) ac_slab();
  if (!s) return sfail(AC_ERR_NOMEM, "out of host memory");
  s->desc = *desc;
  s->parts = parts;
  s->halo = halo;
  s->stream = (cudaStream_t)cuda_stream;
  const size_t es = ac_elem_size(desc->dtype);
  s->plane_bytes = (size_t)desc->pitch_x * es * (d3 ? (size_t)desc->ny : 1);
  s->part.resize(parts);
  // several parts step concurrently, each on its own stream, forked from and
  // joined to the slab's stream around every block of steps
  if (parts > 1 && cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    s->fork = nullptr;
    slab_free(s);
    return sfail(AC_ERR_CUDA, "event creation failed");
  }
  for (int p = 0; p < parts; ++p) {
    SlabPart &sp = s->part[p];
    sp.plan = plan[p];
    if (parts > 1 && (cudaStreamCreateWithFlags(&sp.stream, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&sp.done, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      slab_free(s);
      return sfail(AC_ERR_CUDA, "slab %d: stream or event creation failed", p);
    }
    ac_grid_desc ld = *desc;
    const int64_t n_ext = sp.plan.ext_hi - sp.plan.ext_lo;
    if (d3) ld.nz = n_ext; else ld.ny = n_ext;
    const size_t bytes = (size_t)n_ext * s->plane_bytes;
    if (cudaMalloc(&sp.phi, bytes) != cudaSuccess || cudaMalloc(&sp.ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      slab_free(s);
      return sfail(AC_ERR_NOMEM, "slab %d: %zu bytes per field do not fit", p, bytes);
    }
    rc = ac_create(&ld, sp.phi, sp.ws, parts > 1 ? (void *)sp.stream : cuda_stream, &sp.ctx);
    if (rc) {
      slab_free(s);
      return rc;
    }
  }
  *out = s;
  return AC_OK;
}

static int copy_planes(ac_slab *s, void *dst, const void *src, int64_t planes) {
  if (planes <= 0) return AC_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)planes * s->plane_bytes, cudaMemcpyDeviceToDevice,
                                  s->stream);
  if (e != cudaSuccess) return sfail(AC_ERR_CUDA, "halo copy failed: %s", cudaGetErrorString(e));
  ++s->copies;
  return AC_OK;
}

extern "C" int ac_slab_scatter(ac_slab *s, const void *phi_dev) {
  if (!s || !phi_dev) return sfail(AC_ERR_INVALID, "NULL argument");
  for (SlabPart &p : s->part) {
    int rc = copy_planes(s, p.phi, at(const_cast<void *>(phi_dev), p.plan.ext_lo, s->plane_bytes),
                         p.plan.ext_hi - p.plan.ext_lo);
    if (rc) return rc;
  }
  s->fresh = true;
  return AC_OK;
}

extern "C" int ac_slab_gather(ac_slab *s, void *phi_dev) {
  if (!s || !phi_dev) return sfail(AC_ERR_INVALID, "NULL argument");
  for (SlabPart &p : s->part) {
    int rc = copy_planes(s, at(phi_dev, p.plan.own_lo, s->plane_bytes),
                         at(p.phi, p.plan.own_lo - p.plan.ext_lo, s->plane_bytes),
                         p.plan.own_hi - p.plan.own_lo);
    if (rc) return rc;
  }
  return AC_OK;
}

// Refresh every halo from the neighbour that owns its planes.
static int exchange(ac_slab *s) {
  for (int p = 1; p < s->parts; ++p) {
    SlabPart &lo = s->part[p - 1], &hi = s->part[p];
    // lower halo of hi: planes [hi.ext_lo, hi.own_lo), owned by lo
    int rc = copy_planes(s, hi.phi, at(lo.phi, hi.plan.ext_lo - lo.plan.ext_lo, s->plane_bytes),
                         hi.plan.own_lo - hi.plan.ext_lo);
    if (rc) return rc;
    // upper halo of lo: planes [lo.own_hi, lo.ext_hi), owned by hi
    rc = copy_planes(s, at(lo.phi, lo.plan.own_hi - lo.plan.ext_lo, s->plane_bytes),
                     at(hi.phi, lo.plan.own_hi - hi.plan.ext_lo, s->plane_bytes),
                     lo.plan.ext_hi - lo.plan.own_hi);
    if (rc) return rc;
  }
  s->fresh = true;
  return AC_OK;
}

static int slab_issue(ac_slab *s, int64_t n) {
  while (n > 0) {
    const int64_t b = n < s->halo ? n : s->halo;
    if (!s->fresh) {
      int rc = exchange(s);
      if (rc) return rc;
    }
    if (s->parts == 1) {
      int rc = ac_step(s->part[0].ctx, b);
      if (rc) return rc;
    } else {
      if (cudaEventRecord(s->fork, s->stream) != cudaSuccess)
        return sfail(AC_ERR_CUDA, "fork event failed");
      for (SlabPart &p : s->part) {
        if (cudaStreamWaitEvent(p.stream, s->fork, 0) != cudaSuccess)
          return sfail(AC_ERR_CUDA, "stream wait failed");
        int rc = ac_step(p.ctx, b);
        if (rc) return rc;
        if (cudaEventRecord(p.done, p.stream) != cudaSuccess)
          return sfail(AC_ERR_CUDA, "join event failed");
      }
      for (SlabPart &p : s->part)
        if (cudaStreamWaitEvent(s->stream, p.done, 0) != cudaSuccess)
          return sfail(AC_ERR_CUDA, "stream wait failed");
      s->fresh = false;
    }
    n -= b;
  }
  return AC_OK;
}

extern "C" int ac_slab_step(ac_slab *s, int64_t n) {
  if (!s) return sfail(AC_ERR_INVALID, "slab is NULL");
  if (n < 0) return sfail(AC_ERR_INVALID, "n must be >= 0");
  if (n == 0) return AC_OK;
  if (!s->use_graph || s->stream == nullptr) return slab_issue(s, n);
  // the whole sequence (blocks, halo copies) as one graph, captured once per
  // (n, whether the halos are fresh at the start)
  if (!s->graph || s->graph_n != n || s->graph_fresh != s->fresh) {
    slab_release_graph(s);
    const bool fresh0 = s->fresh;
    const int64_t copies0 = s->copies;
    std::vector<int64_t> launches0;
    for (SlabPart &p : s->part) {
      int64_t c = 0;
      ac_launch_count(p.ctx, &c);
      launches0.push_back(c);
    }
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return sfail(AC_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    int rc = slab_issue(s, n);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->stream, &g);
    s->graph_copies = s->copies - copies0;
    s->copies = copies0;
    s->fresh = fresh0;  // the capture only recorded the sequence
    if (rc == AC_OK && e != cudaSuccess) rc = sfail(AC_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    if (rc == AC_OK && cudaGraphInstantiate(&s->graph, g, 0) != cudaSuccess) {
      s->graph = nullptr;
      rc = sfail(AC_ERR_CUDA, "graph instantiate failed");
    }
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    s->graph_n = n;
    s->graph_fresh = fresh0;
    // the part contexts counted their captured kernels as launched: the
    // replays below count them instead
    for (size_t i = 0; i < s->part.size(); ++i) {
      int64_t c = 0;
      ac_launch_count(s->part[i].ctx, &c);
      s->part[i].graph_kernels = c - launches0[i];
      s->part[i].extra -= s->part[i].graph_kernels;
    }
  }
  cudaError_t e = cudaGraphLaunch(s->graph, s->stream);
  if (e != cudaSuccess) return sfail(AC_ERR_CUDA, "graph launch failed: %s", cudaGetErrorString(e));
  for (SlabPart &p : s->part) p.extra += p.graph_kernels;
  s->copies += s->graph_copies;
  if (s->parts > 1) s->fresh = false;
  return AC_OK;
}

extern "C" int ac_slab_set_graph(ac_slab *s, int32_t enable) {
  if (!s) return sfail(AC_ERR_INVALID, "slab is NULL");
  if (enable && s->stream == nullptr)
    return sfail(AC_ERR_UNSUPPORTED, "graph replay needs a non-default stream");
  s->use_graph = enable != 0;
  if (!s->use_graph) slab_release_graph(s);
  return AC_OK;
}

extern "C" int ac_slab_set_schedule(ac_slab *s, int32_t variant, int32_t k) {
  if (!s) return sfail(AC_ERR_INVALID, "slab is NULL");
  slab_release_graph(s);
  for (SlabPart &p : s->part) {
    int rc = ac_set_schedule(p.ctx, variant, k);
    if (rc) return rc;
  }
  return AC_OK;
}

extern "C" int ac_slab_get_part(ac_slab *s, int32_t part, ac_slab_part *plan, int32_t *halo, void **phi_dev) {
  if (!s) return sfail(AC_ERR_INVALID, "slab is NULL");
  if (part < 0 || part >= s->parts) return sfail(AC_ERR_INVALID, "part %d out of range", part);
  if (plan) *plan = s->part[part].plan;
  if (halo) *halo = s->halo;
  if (phi_dev) *phi_dev = s->part[part].phi;
  return AC_OK;
}

extern "C" int ac_slab_launch_count(ac_slab *s, int64_t *kernels, int64_t *copies) {
  if (!s) return sfail(AC_ERR_INVALID, "slab is NULL");
  int64_t k = 0;
  for (SlabPart &p : s->part) {
    int64_t c = 0;
    ac_launch_count(p.ctx, &c);
    k += c + p.extra;
  }
  if (kernels) *kernels = k;
  if (copies) *copies = s->copies;
  return AC_OK;
}

extern "C" int ac_slab_destroy(ac_slab *s) {
  if (!s) return AC_OK;
  cudaStreamSynchronize(s->stream);
  slab_free(s);
  return AC_OK;
}
