// api.cu -- context management, error reporting, and the ph_eval_jac /
// ph_mgs_solve entry points of the C ABI (include/ph.h).
#include <atomic>
#include <cstdio>
#include <cstring>

#include "ctrl.h"
#include "internal.h"

ph_status ph_fail(ph_ctx *ctx, ph_status st, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return st;
}

ph_status ph_cuda_fail(ph_ctx *ctx, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return ph_fail(ctx, e == cudaErrorMemoryAllocation ? PH_ENOMEM : PH_ECUDA, m);
}

bool ph_is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" const char *ph_version(void) { return "libph 0.2 (sm_103a)"; }

// ---- device memory accounting ---------------------------------------------------

static std::atomic<int64_t> g_dev_used{0};
static std::atomic<int64_t> g_dev_limit{0};        // 0: no cap

cudaError_t ph_dev_alloc(void **p, size_t bytes) {
  const int64_t lim = g_dev_limit.load();
  const int64_t now = g_dev_used.fetch_add((int64_t)bytes) + (int64_t)bytes;
  if (lim > 0 && now > lim) {
    g_dev_used.fetch_sub((int64_t)bytes);
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) g_dev_used.fetch_sub((int64_t)bytes);
  return e;
}

void ph_dev_free(void *p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  g_dev_used.fetch_sub((int64_t)bytes);
}

extern "C" ph_status ph_set_memory_limit(int64_t bytes, int64_t *in_use) {
  if (bytes < 0) return PH_EINVAL;
  g_dev_limit.store(bytes);
  if (in_use) *in_use = g_dev_used.load();
  return PH_OK;
}

extern "C" ph_status ph_set_wait_limit(ph_ctx *ctx, double ms) {
  if (!ctx) return PH_EINVAL;
  if (!(ms > 0.0) || ms > 600000.0) return ph_fail(ctx, PH_EINVAL, "ph_set_wait_limit: out of range");
  ctx->wait_ns = (unsigned long long)(ms * 1e6);
  return PH_OK;
}

void ph_track_release(ph_ctx *ctx);

extern "C" ph_status ph_debug_withhold_pivot(ph_ctx *ctx, int k) {
  if (!ctx) return PH_EINVAL;
  ctx->withhold = k < 0 ? -1 : k;
  ph_track_release(ctx);                            // captured graphs hold the old value
  return PH_OK;
}

extern "C" ph_status ph_init(ph_ctx **out, int device, void *cuda_stream) {
  if (!out) return PH_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return PH_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return PH_ECUDA;
  }
  ph_ctx *c = new (std::nothrow) ph_ctx();
  if (!c) return PH_ENOMEM;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return PH_OK;
}

extern "C" ph_status ph_destroy(ph_ctx *c) {
  if (!c) return PH_EINVAL;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  ph_track_release(c);
  DevBuf *bufs[] = {&c->in_x, &c->in_gamma, &c->in_t, &c->in_J, &c->in_rhs, &c->out_h,
                    &c->out_J, &c->out_dx, &c->slots, &c->ptab, &c->scal, &c->A, &c->R,
                    &c->nrm2, &c->irkk, &c->dxv, &c->state, &c->hist, &c->xw, &c->logbuf,
                    &c->ystage, &c->flags, &c->spow, &c->bws, &c->bq, &c->bx0, &c->bxo,
                    &c->bstats, &c->blog, &c->btune, &c->tuneA, &c->tuneW, &c->tuneN,
                    &c->tuneF, &c->tuneX, &c->tuneS, &c->mgs_part};
  for (DevBuf *b : bufs) b->release();
  delete c;
  return PH_OK;
}

extern "C" const char *ph_last_error(ph_ctx *c) { return c ? c->err.c_str() : "no context"; }

// ---- staging of host or device arrays --------------------------------------------

// Returns a device pointer holding `bytes` of src: src itself when it already is
// device memory, else a copy in `buf`.
static ph_status stage_in(ph_ctx *ctx, DevBuf &buf, const void *src, size_t bytes,
                          const double **dev) {
  if (ph_is_device_ptr(src)) {
    *dev = (const double *)src;
    return PH_OK;
  }
  PH_CUDA(ctx, buf.ensure(bytes));
  PH_CUDA(ctx, cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *dev = buf.as<const double>();
  return PH_OK;
}

static ph_status stage_out(ph_ctx *ctx, DevBuf &buf, void *dst, size_t bytes, double **dev,
                           bool *host) {
  *host = !ph_is_device_ptr(dst);
  if (!*host) {
    *dev = (double *)dst;
    return PH_OK;
  }
  PH_CUDA(ctx, buf.ensure(bytes));
  *dev = buf.as<double>();
  return PH_OK;
}

static ph_status reset_state(ph_ctx *ctx, PathState **st) {
  PH_CUDA(ctx, ctx->state.ensure(sizeof(PathState)));
  PH_CUDA(ctx, cudaMemsetAsync(ctx->state.p, 0, sizeof(PathState), ctx->stream));
  *st = ctx->state.as<PathState>();
  return PH_OK;
}

static ph_status read_state(ph_ctx *ctx, PathState *h) {
  PH_CUDA(ctx, cudaMemcpyAsync(h, ctx->state.p, sizeof(PathState), cudaMemcpyDeviceToHost,
                               ctx->stream));
  PH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PH_OK;
}

extern "C" ph_status ph_eval_jac(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                 const double *gamma, int k, const double *t, const double *x,
                                 double *h, double *J) {
  if (!ctx) return PH_EINVAL;
  if (!f || f->ctx != ctx) return ph_fail(ctx, PH_EINVAL, "ph_eval_jac: f missing or from another context");
  if (g && (g->ctx != ctx || g->L != f->L || g->N != f->N || g->n != f->n))
    return ph_fail(ctx, PH_EINVAL, "ph_eval_jac: g does not match f");
  if (!x || !h || !J) return ph_fail(ctx, PH_EINVAL, "ph_eval_jac: NULL array");
  if (gamma) {
    if (!t) return ph_fail(ctx, PH_EINVAL, "ph_eval_jac: t is NULL");
    if (k < 1 || k > 64) return ph_fail(ctx, PH_EINVAL, "ph_eval_jac: k must be in [1, 64]");
    if (!g) {
      if (f->N != f->n) return ph_fail(ctx, PH_EINVAL, "ph_eval_jac: the total-degree start system needs N == n");
      if (f->max_deg < 1) return ph_fail(ctx, PH_EINVAL, "ph_eval_jac: f has a constant polynomial");
      for (int d : f->h_deg)
        if (d < 1) return ph_fail(ctx, PH_EINVAL, "ph_eval_jac: f has a constant polynomial");
    }
  }
  cudaSetDevice(ctx->device);
  const int L = f->L, n = f->n, N = f->N;
  const double *dx_ = nullptr, *dg = nullptr, *dt = nullptr;
  ph_status s;
  if ((s = stage_in(ctx, ctx->in_x, x, sizeof(double) * 2 * L * n, &dx_)) != PH_OK) return s;
  if (gamma) {
    if ((s = stage_in(ctx, ctx->in_gamma, gamma, sizeof(double) * 2 * L, &dg)) != PH_OK) return s;
    if ((s = stage_in(ctx, ctx->in_t, t, sizeof(double) * L, &dt)) != PH_OK) return s;
  }
  double *dh, *dJ;
  bool hh, hJ;
  const size_t hbytes = sizeof(double) * 2 * L * N, Jbytes = sizeof(double) * 2 * L * (size_t)n * N;
  if ((s = stage_out(ctx, ctx->out_h, h, hbytes, &dh, &hh)) != PH_OK) return s;
  if ((s = stage_out(ctx, ctx->out_J, J, Jbytes, &dJ, &hJ)) != PH_OK) return s;
  PH_CUDA(ctx, ph_eval_launch(ctx, f, g, dg, k, dt, dx_, dh, dJ, N, (long)n * N, nullptr, 0,
                              nullptr, nullptr));
  if (hh) PH_CUDA(ctx, cudaMemcpyAsync(h, dh, hbytes, cudaMemcpyDeviceToHost, ctx->stream));
  if (hJ) PH_CUDA(ctx, cudaMemcpyAsync(J, dJ, Jbytes, cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PH_OK;
}

long ph_lda(int N) { return ((long)N + 31) / 32 * 32; }

extern "C" ph_status ph_mgs_solve(ph_ctx *ctx, ph_prec prec, int N, int n, const double *J,
                                  const double *rhs, double *dx, double *resid_norm) {
  if (!ctx) return PH_EINVAL;
  if (prec != PH_D && prec != PH_DD && prec != PH_QD)
    return ph_fail(ctx, PH_EINVAL, "ph_mgs_solve: bad precision");
  if (n < 1 || N < n) return ph_fail(ctx, PH_EINVAL, "ph_mgs_solve: need N >= n >= 1");
  if ((long)N * (n + 1) > (1L << 28)) return ph_fail(ctx, PH_EINVAL, "ph_mgs_solve: matrix too large");
  if (!J || !rhs || !dx) return ph_fail(ctx, PH_EINVAL, "ph_mgs_solve: NULL array");
  cudaSetDevice(ctx->device);
  const int L = (int)prec, nc = n + 1;
  const long ldA = ph_lda(N), Ap = (long)nc * ldA;
  PH_CUDA(ctx, ctx->A.ensure(sizeof(double) * 2 * L * (size_t)Ap));
  double *A = ctx->A.as<double>();
  // A = [J | rhs]: one pitched copy per limb/part plane
  for (int c = 0; c < 2 * L; ++c) {
    PH_CUDA(ctx, cudaMemcpy2DAsync(A + c * Ap, ldA * sizeof(double), J + (long)c * n * N,
                                   N * sizeof(double), N * sizeof(double), n, cudaMemcpyDefault,
                                   ctx->stream));
  }
  PH_CUDA(ctx, cudaMemcpy2DAsync(A + (long)n * ldA, Ap * sizeof(double), rhs, N * sizeof(double),
                                 N * sizeof(double), 2 * L, cudaMemcpyDefault, ctx->stream));
  PathState *st;
  ph_status s;
  if ((s = reset_state(ctx, &st)) != PH_OK) return s;
  double *ddx;
  bool hdx;
  const size_t dxbytes = sizeof(double) * 2 * L * n;
  if ((s = stage_out(ctx, ctx->out_dx, dx, dxbytes, &ddx, &hdx)) != PH_OK) return s;
  PH_CUDA(ctx, ctx->ystage.ensure(sizeof(double)));
  double *dres = ctx->ystage.as<double>();
  PH_CUDA(ctx, ctx->flags.ensure(sizeof(int) * (size_t)(n + 1)));
  PH_CUDA(ctx, cudaMemsetAsync(ctx->flags.p, 0, sizeof(int) * (size_t)(n + 1), ctx->stream));
  PH_CUDA(ctx, ph_mgs_launch(ctx, L, N, n, A, ldA, ddx, st, nullptr, dres));
  if (hdx) PH_CUDA(ctx, cudaMemcpyAsync(dx, ddx, dxbytes, cudaMemcpyDeviceToHost, ctx->stream));
  double rn = 0.0;
  PH_CUDA(ctx, cudaMemcpyAsync(&rn, dres, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PathState hs;
  if ((s = read_state(ctx, &hs)) != PH_OK) return s;
  if (hs.timeout) return ph_fail(ctx, PH_TIMEOUT, "ph_mgs_solve: a grid barrier timed out");
  if (hs.mgs_status != PH_OK)
    return ph_fail(ctx, (ph_status)hs.mgs_status, "ph_mgs_solve: a column of [J | rhs] became zero");
  if (resid_norm) *resid_norm = rn;
  return PH_OK;
}

// ---- host-exported step-size controller -----------------------------------------

extern "C" void ph_ctrl_init(ph_ctrl_state *c, const ph_track_params *p) { ctrl_init(c, p); }
extern "C" double ph_ctrl_next_t(ph_ctrl_state *c, const ph_track_params *p) { return ctrl_next_t(c, p); }
extern "C" void ph_ctrl_report(ph_ctrl_state *c, const ph_track_params *p, double t_new, int success) {
  ctrl_report(c, p, t_new, success);
}
extern "C" int ph_ctrl_linear_contraction(double d2, double d1, double d0) {
  return linear_contraction(d2, d1, d0) ? 1 : 0;
}
