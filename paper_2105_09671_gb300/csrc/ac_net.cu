// C ABI of the learned 16-step jump network: parameters, forward pass,
// loss and gradients, Adam, and the guarded learned advance of a context.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.h"
#include "net.cuh"

using namespace ac;

static int nfail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return set_error(code, buf);
}

#define NC_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return nfail(AC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

struct ShapeBufs {
  bool valid = false;
  bool train = false;
  NetShape sh{};
  NetBuffers nb;  // activation / gradient pointers for this shape
  float *phihat = nullptr;
};

struct ac_net {
  int ndim = 2;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 1;
  NetBuffers base;  // params, grads, moments, packed weights, status, loss
  ShapeBufs infer, train;
  int adam_step = 0;
  bool grads_valid = false;
  unsigned int *guard = nullptr;  // 2 words: guard maxima
  // spot check of the guard: box scratch, per-box partials, result, and a
  // pinned host copy of one jump's guard quantities
  float *spot_scratch = nullptr;
  size_t spot_floats = 0;
  double *spot_partials = nullptr;
  int spot_cap = 0;
  double *spot_out = nullptr;  // 4 doubles
  double *h_res = nullptr;     // pinned: [0..1] guard words, [2..5] observe, [6..9] spot
  int64_t launches = 0;
};

static int ensure_spot(ac_net *net, size_t floats, int samples) {
  if (net->spot_floats < floats) {
    cudaFree(net->spot_scratch);
    net->spot_scratch = nullptr;
    net->spot_floats = 0;
    NC_CUDA(cudaMalloc(&net->spot_scratch, floats * sizeof(float)));
    net->spot_floats = floats;
  }
  if (net->spot_cap < samples) {
    cudaFree(net->spot_partials);
    net->spot_partials = nullptr;
    net->spot_cap = 0;
    NC_CUDA(cudaMalloc(&net->spot_partials, (size_t)samples * 4 * sizeof(double)));
    net->spot_cap = samples;
  }
  return AC_OK;
}

static void spot_settings(int ndim, const ac_guard *g, int *samples, int *size) {
  *samples = g->spot_samples > 0 ? g->spot_samples : (ndim == 3 ? 16 : 64);
  *size = g->spot_size > 0 ? g->spot_size : (ndim == 3 ? 8 : 32);
}

static double rel_from(double d2, double r2) {
  if (!(d2 == d2)) return INFINITY;
  if (r2 > 0) return std::sqrt(d2 / r2);
  return d2 > 0 ? INFINITY : 0.0;
}

static void free_shape(ShapeBufs &s) {
  for (int i = 0; i < 5; ++i) {
    cudaFree(s.nb.a[i]);
    cudaFree(s.nb.z[i]);
    cudaFree(s.nb.gz[i]);
    s.nb.a[i] = s.nb.z[i] = s.nb.gz[i] = nullptr;
  }
  cudaFree(s.nb.raw);
  cudaFree(s.nb.g6);
  cudaFree(s.phihat);
  s.nb.raw = s.nb.g6 = s.phihat = nullptr;
  s.valid = false;
}

static bool same_shape(const NetShape &a, const NetShape &b) {
  return a.ndim == b.ndim && a.batch == b.batch && a.nx == b.nx && a.ny == b.ny && a.nz == b.nz;
}

// Per-shape buffers: inference keeps two padded activations; training keeps
// all five, the pre-activations, the padded gradients (zero ghost ring, set
// once here) and the FP32 scratch.
static int ensure_shape(ShapeBufs &s, const NetShape &sh, bool train) {
  if (s.valid && same_shape(s.sh, sh) && s.train == train) return AC_OK;
  free_shape(s);
  const size_t act = (size_t)sh.padded_cells() * kNetC * sizeof(bf16);
  const size_t zb = (size_t)sh.cells() * kNetC * sizeof(bf16);
  const int na = train ? 5 : 2;
  for (int i = 0; i < na; ++i) NC_CUDA(cudaMalloc(&s.nb.a[i], act));
  if (train) {
    for (int i = 0; i < 5; ++i) {
      NC_CUDA(cudaMalloc(&s.nb.z[i], zb));
      NC_CUDA(cudaMalloc(&s.nb.gz[i], act));
      NC_CUDA(cudaMemset(s.nb.gz[i], 0, act));
    }
    NC_CUDA(cudaMalloc(&s.nb.raw, (size_t)sh.cells() * kNetC * sizeof(float)));
    NC_CUDA(cudaMalloc(&s.nb.g6, (size_t)sh.cells() * sizeof(float)));
    NC_CUDA(cudaMalloc(&s.phihat, (size_t)sh.cells() * sizeof(float)));
  }
  s.sh = sh;
  s.train = train;
  s.valid = true;
  return AC_OK;
}

static NetBuffers merged(const ac_net *net, const ShapeBufs &s) {
  NetBuffers nb = net->base;
  for (int i = 0; i < 5; ++i) {
    nb.a[i] = s.nb.a[i];
    nb.z[i] = s.nb.z[i];
    nb.gz[i] = s.nb.gz[i];
  }
  nb.raw = s.nb.raw;
  nb.g6 = s.nb.g6;
  return nb;
}

static int check_shape(int ndim, int32_t batch, int64_t nx, int64_t ny, int64_t nz, NetShape *sh) {
  if (batch < 1 || nx < 1 || ny < 1 || nz < 1) return nfail(AC_ERR_INVALID, "batch and sizes must be >= 1");
  if (ndim == 2 && nz != 1) return nfail(AC_ERR_INVALID, "2D networks need nz == 1");
  if (nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
    return nfail(AC_ERR_INVALID, "grid extent too large");
  sh->ndim = ndim;
  sh->batch = batch;
  sh->nx = (int)nx;
  sh->ny = (int)ny;
  sh->nz = (int)nz;
  return AC_OK;
}

// He-normal initial weights (std sqrt(2 / fan_in)) from a SplitMix64 stream
// and Box-Muller; the last layer starts at zero, so the initial jump is the
// identity; biases start at zero.
static void he_init(const NetLayout &L, uint64_t seed, std::vector<float> &p) {
  p.assign((size_t)L.total, 0.0f);
  uint64_t state = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  auto next_u = [&]() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((double)(z >> 11) + 0.5) * 0x1.0p-53;  // (0, 1)
  };
  for (int l = 0; l < kNetLayers - 1; ++l) {
    const int64_t count = (int64_t)L.T * NetLayout::cin(l) * NetLayout::cout(l);
    const double sd = std::sqrt(2.0 / ((double)L.T * NetLayout::cin(l)));
    for (int64_t i = 0; i < count; ++i) {
      const double u1 = next_u(), u2 = next_u();
      p[L.w[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
}

extern "C" int ac_net_param_count(int32_t ndim, int64_t *out) {
  if ((ndim != 2 && ndim != 3) || !out) return nfail(AC_ERR_INVALID, "ndim must be 2 or 3");
  *out = net_layout(ndim).total;
  return AC_OK;
}

extern "C" int ac_net_create(int32_t ndim, void *cuda_stream, ac_net **out) {
  if (!out) return nfail(AC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return nfail(AC_ERR_INVALID, "ndim must be 2 or 3");
  ac_net *net = new (std::nothrow) ac_net();
  if (!net) return nfail(AC_ERR_NOMEM, "out of host memory");
  net->ndim = ndim;
  net->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&net->device);
  cudaDeviceGetAttribute(&net->num_sms, cudaDevAttrMultiProcessorCount, net->device);
  NetBuffers &b = net->base;
  b.layout = net_layout(ndim);
  const size_t pbytes = (size_t)b.layout.total * sizeof(float);
  const size_t wbytes = (size_t)4 * kNetC * b.layout.T * kNetC * sizeof(bf16);
  cudaError_t e = cudaMalloc(&b.params, pbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b.grads, pbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b.m, pbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b.v, pbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b.wf, wbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b.wd, wbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b.loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b.status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&net->guard, 2 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&net->spot_out, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&net->h_res, 10 * sizeof(double));
  std::vector<float> init;
  he_init(b.layout, 0, init);
  if (e == cudaSuccess) e = cudaMemcpy(b.params, init.data(), pbytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b.m, 0, pbytes);
  if (e == cudaSuccess) e = cudaMemset(b.v, 0, pbytes);
  if (e == cudaSuccess) e = cudaMemset(b.status, 0, sizeof(int));
  if (e == cudaSuccess) e = net_pack(b, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  if (e != cudaSuccess) {
    cudaFree(b.params); cudaFree(b.grads); cudaFree(b.m); cudaFree(b.v);
    cudaFree(b.wf); cudaFree(b.wd); cudaFree(b.loss); cudaFree(b.status); cudaFree(net->guard);
    cudaFree(net->spot_out); cudaFreeHost(net->h_res);
    delete net;
    cudaGetLastError();
    return nfail(AC_ERR_NOMEM, "network allocation failed: %s", cudaGetErrorString(e));
  }
  *out = net;
  return AC_OK;
}

extern "C" int ac_net_destroy(ac_net *net) {
  if (!net) return AC_OK;
  cudaStreamSynchronize(net->stream);
  free_shape(net->infer);
  free_shape(net->train);
  NetBuffers &b = net->base;
  cudaFree(b.params); cudaFree(b.grads); cudaFree(b.m); cudaFree(b.v);
  cudaFree(b.wf); cudaFree(b.wd); cudaFree(b.loss); cudaFree(b.status); cudaFree(net->guard);
  cudaFree(net->spot_out); cudaFreeHost(net->h_res);
  cudaFree(net->spot_scratch); cudaFree(net->spot_partials);
  delete net;
  return AC_OK;
}

extern "C" int ac_net_set_params(ac_net *net, const float *host_params, int64_t count) {
  if (!net || !host_params) return nfail(AC_ERR_INVALID, "NULL argument");
  if (count != net->base.layout.total)
    return nfail(AC_ERR_INVALID, "expected %lld parameters, got %lld",
                 (long long)net->base.layout.total, (long long)count);
  NC_CUDA(cudaStreamSynchronize(net->stream));
  NC_CUDA(cudaMemcpy(net->base.params, host_params, count * sizeof(float), cudaMemcpyHostToDevice));
  const size_t pbytes = (size_t)count * sizeof(float);
  NC_CUDA(cudaMemset(net->base.m, 0, pbytes));
  NC_CUDA(cudaMemset(net->base.v, 0, pbytes));
  net->adam_step = 0;
  net->grads_valid = false;
  NC_CUDA(net_pack(net->base, net->stream));
  ++net->launches;
  NC_CUDA(cudaStreamSynchronize(net->stream));
  return AC_OK;
}

extern "C" int ac_net_init_params(ac_net *net, uint64_t seed) {
  if (!net) return nfail(AC_ERR_INVALID, "net is NULL");
  std::vector<float> init;
  he_init(net->base.layout, seed, init);
  return ac_net_set_params(net, init.data(), (int64_t)init.size());
}

extern "C" int ac_net_get_params(ac_net *net, float *host_params, int64_t count) {
  if (!net || !host_params) return nfail(AC_ERR_INVALID, "NULL argument");
  if (count != net->base.layout.total) return nfail(AC_ERR_INVALID, "wrong parameter count");
  NC_CUDA(cudaStreamSynchronize(net->stream));
  NC_CUDA(cudaMemcpy(host_params, net->base.params, count * sizeof(float), cudaMemcpyDeviceToHost));
  return AC_OK;
}

extern "C" int ac_net_forward(ac_net *net, const float *phi_dev, float *out_dev, int32_t batch,
                              int64_t nx, int64_t ny, int64_t nz, double scale) {
  if (!net || !phi_dev || !out_dev) return nfail(AC_ERR_INVALID, "NULL argument");
  NetShape sh;
  int rc = check_shape(net->ndim, batch, nx, ny, nz, &sh);
  if (rc) return rc;
  rc = ensure_shape(net->infer, sh, false);
  if (rc) return rc;
  cudaError_t e = net_forward(merged(net, net->infer), sh, phi_dev, (float)scale, out_dev, nullptr,
                              false, net->num_sms, net->stream);
  if (e != cudaSuccess) return nfail(AC_ERR_CUDA, "network forward failed: %s", cudaGetErrorString(e));
  net->launches += 6;
  return AC_OK;
}

extern "C" int ac_net_loss_grads(ac_net *net, const float *phi_dev, const float *target_dev,
                                 int32_t batch, int64_t nx, int64_t ny, int64_t nz, double scale,
                                 double *loss, float *grads_host) {
  if (!net || !phi_dev || !target_dev || !loss) return nfail(AC_ERR_INVALID, "NULL argument");
  if (!(scale > 0)) return nfail(AC_ERR_INVALID, "scale must be > 0");
  NetShape sh;
  int rc = check_shape(net->ndim, batch, nx, ny, nz, &sh);
  if (rc) return rc;
  rc = ensure_shape(net->train, sh, true);
  if (rc) return rc;
  const NetBuffers nb = merged(net, net->train);
  NC_CUDA(cudaMemsetAsync(nb.loss, 0, sizeof(double), net->stream));
  NC_CUDA(cudaMemsetAsync(nb.grads, 0, (size_t)nb.layout.total * sizeof(float), net->stream));
  cudaError_t e = net_forward(nb, sh, phi_dev, (float)scale, net->train.phihat, target_dev, true,
                              net->num_sms, net->stream);
  if (e == cudaSuccess) e = net_backward(nb, sh, phi_dev, net->num_sms, net->stream);
  if (e != cudaSuccess) return nfail(AC_ERR_CUDA, "network training pass failed: %s", cudaGetErrorString(e));
  net->launches += 6 + 1 + 4 * 3 + 1;
  double h = 0.0;
  NC_CUDA(cudaMemcpyAsync(&h, nb.loss, sizeof(double), cudaMemcpyDeviceToHost, net->stream));
  NC_CUDA(cudaStreamSynchronize(net->stream));
  *loss = h / (double)sh.cells();
  int st = 0;
  NC_CUDA(cudaMemcpy(&st, nb.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    NC_CUDA(cudaMemset(nb.status, 0, sizeof(int)));
    return nfail(AC_ERR_TIMEOUT, "a bounded tensor-core wait expired");
  }
  if (grads_host)
    NC_CUDA(cudaMemcpy(grads_host, nb.grads, (size_t)nb.layout.total * sizeof(float), cudaMemcpyDeviceToHost));
  net->grads_valid = true;
  return AC_OK;
}

extern "C" int ac_net_adam(ac_net *net, double lr, double beta1, double beta2, double eps) {
  if (!net) return nfail(AC_ERR_INVALID, "net is NULL");
  if (!net->grads_valid) return nfail(AC_ERR_INVALID, "no gradients: call ac_net_loss_grads first");
  if (!(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return nfail(AC_ERR_INVALID, "invalid Adam hyper-parameters");
  ++net->adam_step;
  cudaError_t e = net_adam(net->base, (float)lr, (float)beta1, (float)beta2, (float)eps,
                           net->adam_step, net->stream);
  if (e != cudaSuccess) return nfail(AC_ERR_CUDA, "Adam update failed: %s", cudaGetErrorString(e));
  net->launches += 2;
  return AC_OK;
}

extern "C" int ac_net_train_step(ac_net *net, const float *phi_dev, const float *target_dev,
                                 int32_t batch, int64_t nx, int64_t ny, int64_t nz, double scale,
                                 double lr, double *loss) {
  int rc = ac_net_loss_grads(net, phi_dev, target_dev, batch, nx, ny, nz, scale, loss, nullptr);
  if (rc) return rc;
  return ac_net_adam(net, lr, 0.9, 0.999, 1e-8);
}

extern "C" int ac_net_launch_count(ac_net *net, int64_t *out) {
  if (!net || !out) return nfail(AC_ERR_INVALID, "NULL argument");
  *out = net->launches;
  return AC_OK;
}

// ------------------------------------------------------ guarded advance ----
extern "C" int ac_jump_residual(ac_ctx *c, const float *phat_dev, int32_t steps, double out[2]) {
  if (!c || !phat_dev || !out) return nfail(AC_ERR_INVALID, "NULL argument");
  if (c->d.dtype != AC_F32 || c->d.pitch_x != c->d.nx)
    return nfail(AC_ERR_UNSUPPORTED, "needs an FP32 context with pitch_x == nx");
  if (steps < 1) return nfail(AC_ERR_INVALID, "steps must be >= 1");
  unsigned int *buf = reinterpret_cast<unsigned int *>(c->d_out);
  cudaError_t e = launch_guard(static_cast<const float *>(c->phi), phat_dev, c->gp, c->d.ndim, steps, buf, c->stream);
  if (e != cudaSuccess) return nfail(AC_ERR_CUDA, "guard launch failed: %s", cudaGetErrorString(e));
  ++c->launches;
  unsigned int h[2];
  NC_CUDA(cudaMemcpyAsync(h, buf, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  NC_CUDA(cudaStreamSynchronize(c->stream));
  float f[2];
  memcpy(f, h, sizeof f);
  out[0] = f[0];
  out[1] = f[1];
  return AC_OK;
}

extern "C" int ac_jump_spot_check(ac_ctx *c, const float *phat_dev, int32_t steps, int32_t samples,
                                  int32_t size, uint64_t seed, double out[3]) {
  if (!c || !phat_dev || !out) return nfail(AC_ERR_INVALID, "NULL argument");
  if (c->d.dtype != AC_F32) return nfail(AC_ERR_UNSUPPORTED, "needs an FP32 context");
  if (steps < 1 || samples < 0 || size < 0) return nfail(AC_ERR_INVALID, "steps >= 1, samples and size >= 0");
  ac_guard gd{};
  gd.spot_samples = samples;
  gd.spot_size = size;
  int ns, sz;
  spot_settings(c->d.ndim, &gd, &ns, &sz);
  const size_t floats = spot_scratch_floats(c->gp, c->d.ndim, steps, ns, sz);
  float *scratch = nullptr;
  double *part = nullptr, *dout = nullptr;
  cudaError_t e = cudaMalloc(&scratch, floats * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)ns * 4 * sizeof(double) + 4 * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(scratch);
    cudaGetLastError();
    return nfail(AC_ERR_NOMEM, "spot-check scratch allocation failed");
  }
  dout = part + (size_t)ns * 4;
  e = launch_spot_check(static_cast<const float *>(c->phi), phat_dev, c->gp, c->d.ndim, steps, ns, sz,
                        seed, scratch, part, dout, c->stream);
  double h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(scratch);
  cudaFree(part);
  if (e != cudaSuccess) return nfail(AC_ERR_CUDA, "spot check failed: %s", cudaGetErrorString(e));
  c->launches += 2;
  out[0] = h[0];
  out[1] = rel_from(h[1], h[2]);
  out[2] = h[3];
  return AC_OK;
}

extern "C" int ac_learned_advance(ac_ctx *c, ac_net *net, int64_t jumps, const ac_guard *guard,
                                  int64_t *fallbacks, ac_learned_report *report) {
  if (!c || !net || !guard) return nfail(AC_ERR_INVALID, "NULL argument");
  if (jumps < 0) return nfail(AC_ERR_INVALID, "jumps must be >= 0");
  if (c->d.dtype != AC_F32) return nfail(AC_ERR_UNSUPPORTED, "the learned stepper runs on FP32 fields");
  if (c->d.ndim != net->ndim) return nfail(AC_ERR_INVALID, "network and grid dimensions differ");
  if (c->d.pitch_x != c->d.nx) return nfail(AC_ERR_UNSUPPORTED, "the learned stepper needs pitch_x == nx");
  if (guard->steps_per_jump < 1) return nfail(AC_ERR_INVALID, "steps_per_jump must be >= 1");
  if (guard->spot_samples < 0 || guard->spot_size < 0)
    return nfail(AC_ERR_INVALID, "spot_samples and spot_size must be >= 0");
  if (c->stream != net->stream) return nfail(AC_ERR_INVALID, "context and network must share a stream");
  const int n = guard->steps_per_jump;
  const double scale = n * c->gp.alpha;  // s = n dt / eps^2
  float *phi = static_cast<float *>(c->phi);
  float *phat = static_cast<float *>(c->ws);
  const bool use_spot = guard->spot_rtol > 0;
  int ns = 0, sz = 0;
  spot_settings(c->d.ndim, guard, &ns, &sz);
  if (use_spot) {
    const int rc = ensure_spot(net, spot_scratch_floats(c->gp, c->d.ndim, n, ns, sz), ns);
    if (rc) return rc;
  }
  ac_learned_report rep{};
  int64_t fb = 0;
  double obs[3];
  int rc = ac_observe(c, obs);
  if (rc) return rc;
  double e_cur = obs[0];
  const double hd = c->d.ndim == 3 ? c->d.h * c->d.h * c->d.h : c->d.h * c->d.h;
  double *hr = net->h_res;
  for (int64_t j = 0; j < jumps; ++j) {
    rc = ac_net_forward(net, phi, phat, 1, c->d.nx, c->d.ny, c->d.nz, scale);
    if (rc) return rc;
    cudaError_t e = launch_guard(phi, phat, c->gp, c->d.ndim, n, net->guard, c->stream);
    if (e == cudaSuccess)  // energy of phi_hat (FP64 reduction over the workspace)
      e = launch_observe(c->d.dtype, c->gp, phat, c->d_partials, c->d_out, c->stream);
    if (e == cudaSuccess && use_spot)
      e = launch_spot_check(phi, phat, c->gp, c->d.ndim, n, ns, sz, guard->spot_seed + (uint64_t)j,
                            net->spot_scratch, net->spot_partials, net->spot_out, c->stream);
    if (e != cudaSuccess) return nfail(AC_ERR_CUDA, "guard launch failed: %s", cudaGetErrorString(e));
    NC_CUDA(cudaMemcpyAsync(hr, net->guard, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream));
    NC_CUDA(cudaMemcpyAsync(hr + 2, c->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (use_spot)
      NC_CUDA(cudaMemcpyAsync(hr + 6, net->spot_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NC_CUDA(cudaStreamSynchronize(c->stream));
    c->launches += 3 + (use_spot ? 2 : 0);
    unsigned int gw[2];
    memcpy(gw, hr, sizeof gw);
    float mabs, mres;
    memcpy(&mabs, &gw[0], 4);
    memcpy(&mres, &gw[1], 4);
    const double e_new = hd * (hr[2] / (c->d.eps * c->d.eps) + 0.5 * hr[3] / (c->d.h * c->d.h));
    const bool finite = hr[5] == 0.0 && std::isfinite(e_new) && std::isfinite(mres);
    const bool ok_e = e_new <= e_cur * (1.0 + guard->energy_rtol) + 1e-300;
    const bool ok_m = mabs <= guard->max_abs;
    const bool ok_r = guard->residual_tol <= 0 || mres <= guard->residual_tol;
    double spot_rel = 0.0, spot_abs = 0.0;
    if (use_spot) {
      spot_abs = hr[6];
      spot_rel = rel_from(hr[7], hr[8]);
    }
    const bool ok_s = !use_spot || spot_rel <= guard->spot_rtol;
    ++rep.jumps;
    rep.rejected_nonfinite += !finite;
    rep.rejected_energy += !ok_e;
    rep.rejected_max_abs += !ok_m;
    rep.rejected_residual += !ok_r;
    rep.rejected_spot += !ok_s;
    rep.max_residual = std::max(rep.max_residual, (double)mres);
    rep.max_spot_rel = std::max(rep.max_spot_rel, spot_rel);
    rep.max_spot_abs = std::max(rep.max_spot_abs, spot_abs);
    if (finite && ok_e && ok_m && ok_r && ok_s) {
      const size_t bytes = (size_t)c->d.nx * c->d.ny * c->d.nz * sizeof(float);
      NC_CUDA(cudaMemcpyAsync(phi, phat, bytes, cudaMemcpyDeviceToDevice, c->stream));
      e_cur = e_new;
    } else {
      ++fb;
      rc = ac_step(c, n);  // the plain stepper takes over for this jump
      if (rc) return rc;
      rc = ac_observe(c, obs);
      if (rc) return rc;
      e_cur = obs[0];
    }
  }
  rep.fallbacks = fb;
  if (fallbacks) *fallbacks = fb;
  if (report) *report = rep;
  return AC_OK;
}

// ---------------------------------------------------------------- training --
// Training data come from the plain stepper itself: a pool of `pool`
// trajectories on n^d grids (h = 1/n, dt = 0.1 h^2, eps = eps_cells h),
// staggered in age so that every phase of the dynamics is in each batch.
// Each iteration copies the pool, advances the copy by steps_per_jump plain
// steps (the targets), takes one Adam step on (pool, targets) and moves the
// pool to the targets.  A trajectory older than trajectory_jumps is replaced
// by a new one: alternately a random state (amplitude 0.1, Section 3.1) and a
// tanh circle / sphere of radius uniform in [0.1, 0.4] centred in the domain.
namespace {
uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Initial state number `index` of the data recipe under `seed`: even
// indices a random state of amplitude 0.1, odd ones a tanh circle / sphere
// of radius uniform in [0.1, 0.4] centred in the unit domain (Section 3.1).
cudaError_t draw_state(const GridParams &g, float *dst, uint64_t seed, int64_t index, double h,
                       double eps, cudaStream_t s) {
  const uint64_t r = mix64(seed * 0x100000001B3ull + (uint64_t)index);
  if (index % 2 == 0) return launch_init_random(AC_F32, g, dst, r, 0.1, s);
  const double r0 = 0.1 + 0.3 * (double)(r >> 11) * 0x1.0p-53;
  const double lo[3] = {0, 0, 0}, c3[3] = {0.5, 0.5, 0.5};
  return launch_init_sphere(AC_F32, g, dst, h, lo, c3, r0, eps, s);
}

int check_train_config(const ac_train_config *cfg) {
  const int n = cfg->n, B = cfg->pool, spj = cfg->steps_per_jump;
  if (n < 8 || n > 4096 || n % 4) return nfail(AC_ERR_INVALID, "n must be a multiple of 4 in [8, 4096]");
  if (B < 1 || B > 4096 || cfg->iterations < 1 || spj < 1 || cfg->trajectory_jumps < 1)
    return nfail(AC_ERR_INVALID, "pool, iterations, steps_per_jump, trajectory_jumps must be >= 1");
  if (!(cfg->eps_cells > 0) || !(cfg->lr > 0) || !(cfg->lr_final >= 0))
    return nfail(AC_ERR_INVALID, "eps_cells and lr must be > 0");
  return AC_OK;
}
}  // namespace

extern "C" int ac_net_train(ac_net *net, const ac_train_config *cfg, double *loss_history,
                            int64_t *trajectories_used) {
  if (!net || !cfg) return nfail(AC_ERR_INVALID, "NULL argument");
  const int nd = net->ndim, n = cfg->n, B = cfg->pool, spj = cfg->steps_per_jump;
  if (int rc0 = check_train_config(cfg)) return rc0;
  const int64_t cells = nd == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const double h = 1.0 / n, eps = cfg->eps_cells * h, dt = 0.1 * h * h;
  const double scale = spj * dt / (eps * eps);
  cudaStream_t s = net->stream;

  float *states = nullptr, *targets = nullptr, *ws = nullptr;
  ac_batch *batch = nullptr;
  std::vector<ac_ctx *> ctxs;
  int rc = AC_OK;
  auto cleanup = [&]() {
    if (batch) ac_batch_destroy(batch);
    for (ac_ctx *c : ctxs) ac_destroy(c);
    cudaFree(states);
    cudaFree(targets);
    cudaFree(ws);
  };
  const size_t fbytes = (size_t)cells * sizeof(float);
  if (cudaMalloc(&states, fbytes * B) != cudaSuccess || cudaMalloc(&targets, fbytes * B) != cudaSuccess ||
      cudaMalloc(&ws, (fbytes + 256) * B) != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    return nfail(AC_ERR_NOMEM, "training buffers do not fit");
  }
  ac_grid_desc d{};
  d.ndim = nd;
  d.dtype = AC_F32;
  d.nx = n;
  d.ny = n;
  d.nz = nd == 3 ? n : 1;
  d.pitch_x = n;
  d.h = h;
  d.eps = eps;
  d.dt = dt;
  if (nd == 2) {
    std::vector<ac_grid_desc> descs(B, d);
    std::vector<void *> ptrs(B);
    for (int i = 0; i < B; ++i) ptrs[i] = targets + (size_t)i * cells;
    rc = ac_batch_create(descs.data(), ptrs.data(), B, ws, s, &batch);
  } else {
    for (int i = 0; i < B && rc == AC_OK; ++i) {
      ac_ctx *c = nullptr;
      rc = ac_create(&d, targets + (size_t)i * cells, reinterpret_cast<char *>(ws) + (fbytes + 256) * i / 256 * 256, s, &c);
      if (rc == AC_OK) ctxs.push_back(c);
    }
  }
  if (rc) { cleanup(); return rc; }

  GridParams g{};
  g.nx = n; g.ny = n; g.nz = d.nz; g.pitch = n;
  g.alpha = dt / (eps * eps); g.beta = dt / (h * h); g.status = nullptr;
  int64_t used = 0;
  auto new_trajectory = [&](int slot) -> int {
    float *dst = states + (size_t)slot * cells;
    const cudaError_t e = draw_state(g, dst, cfg->seed, used, h, eps, s);
    ++used;
    ++net->launches;
    return e == cudaSuccess ? AC_OK : nfail(AC_ERR_CUDA, "init launch failed: %s", cudaGetErrorString(e));
  };
  // advance the pool (in `targets`) by `steps` plain steps
  auto step_targets = [&](int64_t steps) -> int {
    if (steps <= 0) return AC_OK;
    if (batch) {
      std::vector<int64_t> nv(B, steps);
      return ac_batch_step(batch, nv.data());
    }
    for (ac_ctx *c : ctxs) {
      int r2 = ac_step(c, steps);
      if (r2) return r2;
    }
    return AC_OK;
  };
  // staggered start: slot i begins i * L / B jumps into its trajectory
  std::vector<int> age(B);
  for (int i = 0; i < B && rc == AC_OK; ++i) rc = new_trajectory(i);
  if (rc == AC_OK && cudaMemcpyAsync(targets, states, fbytes * B, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    rc = nfail(AC_ERR_CUDA, "copy failed");
  // different pre-advance per slot: run the plain stepper slot by slot
  for (int i = 0; i < B && rc == AC_OK; ++i) {
    age[i] = (int)((int64_t)i * cfg->trajectory_jumps / B);
    if (age[i] == 0) continue;
    ac_ctx *c = nullptr;
    rc = ac_create(&d, targets + (size_t)i * cells, ws, s, &c);
    if (rc == AC_OK) rc = ac_step(c, (int64_t)age[i] * spj);
    if (c) ac_destroy(c);
  }
  if (rc == AC_OK && cudaMemcpyAsync(states, targets, fbytes * B, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    rc = nfail(AC_ERR_CUDA, "copy failed");

  const double kPi = 3.14159265358979323846;
  for (int it = 0; it < cfg->iterations && rc == AC_OK; ++it) {
    if (cudaMemcpyAsync(targets, states, fbytes * B, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      rc = nfail(AC_ERR_CUDA, "copy failed");
      break;
    }
    rc = step_targets(spj);
    if (rc) break;
    const double f = cfg->iterations > 1 ? (double)it / (cfg->iterations - 1) : 1.0;
    const double lr = cfg->lr_final + 0.5 * (cfg->lr - cfg->lr_final) * (1.0 + std::cos(kPi * f));
    double loss = 0.0;
    rc = ac_net_train_step(net, states, targets, B, n, n, d.nz, scale, lr, &loss);
    if (rc) break;
    if (loss_history) loss_history[it] = loss;
    if (cudaMemcpyAsync(states, targets, fbytes * B, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      rc = nfail(AC_ERR_CUDA, "copy failed");
      break;
    }
    for (int i = 0; i < B && rc == AC_OK; ++i)
      if (++age[i] >= cfg->trajectory_jumps) {
        rc = new_trajectory(i);
        age[i] = 0;
      }
  }
  if (rc == AC_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = nfail(AC_ERR_CUDA, "training failed");
  if (trajectories_used) *trajectories_used = used;
  cleanup();
  return rc;
}

// ------------------------------------------------------------- calibration --
extern "C" int ac_net_calibrate_guard(ac_net *net, const ac_train_config *cfg, double residual_factor,
                                      ac_guard *guard, ac_guard_calibration *report) {
  if (!net || !cfg || !guard) return nfail(AC_ERR_INVALID, "NULL argument");
  if (int rc0 = check_train_config(cfg)) return rc0;
  if (!(residual_factor > 0)) return nfail(AC_ERR_INVALID, "residual_factor must be > 0");
  if (guard->spot_samples < 0 || guard->spot_size < 0)
    return nfail(AC_ERR_INVALID, "spot_samples and spot_size must be >= 0");
  const int nd = net->ndim, n = cfg->n, states = cfg->pool, spj = cfg->steps_per_jump;
  const int64_t cells = nd == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const double h = 1.0 / n, eps = cfg->eps_cells * h, dt = 0.1 * h * h;
  const double scale = spj * dt / (eps * eps);
  cudaStream_t s = net->stream;
  const size_t fbytes = (size_t)cells * sizeof(float);
  float *phi = nullptr, *tgt = nullptr, *ws = nullptr, *phat = nullptr;
  ac_ctx *cphi = nullptr, *ctgt = nullptr;
  auto cleanup = [&]() {
    if (cphi) ac_destroy(cphi);
    if (ctgt) ac_destroy(ctgt);
    cudaFree(phi);
    cudaFree(tgt);
    cudaFree(ws);
    cudaFree(phat);
  };
  if (cudaMalloc(&phi, fbytes) != cudaSuccess || cudaMalloc(&tgt, fbytes) != cudaSuccess ||
      cudaMalloc(&ws, fbytes) != cudaSuccess || cudaMalloc(&phat, fbytes) != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    return nfail(AC_ERR_NOMEM, "calibration fields do not fit");
  }
  ac_grid_desc d{};
  d.ndim = nd;
  d.dtype = AC_F32;
  d.nx = n;
  d.ny = n;
  d.nz = nd == 3 ? n : 1;
  d.pitch_x = n;
  d.h = h;
  d.eps = eps;
  d.dt = dt;
  int rc = ac_create(&d, phi, ws, s, &cphi);
  if (rc == AC_OK) rc = ac_create(&d, tgt, ws, s, &ctgt);
  int ns = 0, sz = 0;
  spot_settings(nd, guard, &ns, &sz);
  if (rc == AC_OK) rc = ensure_spot(net, spot_scratch_floats(cphi->gp, nd, spj, ns, sz), ns);
  if (rc) { cleanup(); return rc; }
  GridParams g = cphi->gp;
  double plain_max = 0.0, net_max = 0.0, spot_max = 0.0;
  std::vector<double> rel;
  for (int i = 0; i < states && rc == AC_OK; ++i) {
    // a held-out state: drawn as the training data are, at a staggered age
    cudaError_t e = draw_state(g, phi, cfg->seed, i, h, eps, s);
    if (e != cudaSuccess) { rc = nfail(AC_ERR_CUDA, "init failed: %s", cudaGetErrorString(e)); break; }
    const int64_t age = (int64_t)i * cfg->trajectory_jumps / states;
    rc = ac_step(cphi, age * spj);
    if (rc) break;
    // the plain stepper's jump P(phi) and its residual
    if (cudaMemcpyAsync(tgt, phi, fbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      rc = nfail(AC_ERR_CUDA, "copy failed");
      break;
    }
    rc = ac_step(ctgt, spj);
    double r2[2];
    if (rc == AC_OK) rc = ac_jump_residual(cphi, tgt, spj, r2);
    if (rc) break;
    plain_max = std::max(plain_max, r2[1]);
    // the network's jump: its residual, its error against P over the whole
    // field and the spot check's estimate of that error
    rc = ac_net_forward(net, phi, phat, 1, n, n, d.nz, scale);
    if (rc == AC_OK) rc = ac_jump_residual(cphi, phat, spj, r2);
    if (rc) break;
    net_max = std::max(net_max, r2[1]);
    double *hr = net->h_res;
    e = launch_diff_norms(phat, tgt, cells, cphi->d_partials, cphi->d_out, s);
    if (e == cudaSuccess)
      e = launch_spot_check(phi, phat, g, nd, spj, ns, sz, guard->spot_seed + (uint64_t)i, net->spot_scratch,
                            net->spot_partials, net->spot_out, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr + 2, cphi->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr + 6, net->spot_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rc = nfail(AC_ERR_CUDA, "calibration reduction failed: %s", cudaGetErrorString(e)); break; }
    net->launches += 4;
    rel.push_back(rel_from(hr[3], hr[4]));
    spot_max = std::max(spot_max, rel_from(hr[7], hr[8]));
  }
  cleanup();
  if (rc) return rc;
  std::sort(rel.begin(), rel.end());
  guard->residual_tol = residual_factor * plain_max;
  if (report) {
    report->states = states;
    report->plain_residual_max = plain_max;
    report->net_residual_max = net_max;
    report->net_rel_err_median = rel.empty() ? 0.0 : rel[rel.size() / 2];
    report->net_rel_err_max = rel.empty() ? 0.0 : rel.back();
    report->spot_rel_err_max = spot_max;
  }
  return AC_OK;
}
