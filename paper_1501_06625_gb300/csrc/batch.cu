// batch.cu -- ph_track_paths: many solution paths of one homotopy at once.
//
// The paper accelerates the tracking of a single path (Introduction; the
// many-path case is its companion work).  A single path of a few dozen
// variables cannot fill a GB300: its predictor-corrector step is a chain of
// dependent FP64 operations (~64 cycles each on this GPU).  Here one persistent
// kernel tracks many paths, one block per path: a block takes the next
// unstarted path from a counter, tracks it to its end entirely with its own
// threads (pathblock.cuh: predictor, evaluation, MGS, back substitution,
// update, step control, separated by __syncthreads only), stores the end point
// and takes the next path.  Blocks never wait for one another, paths of uneven
// length balance themselves, and with two blocks per SM every FP64 unit has work.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pathblock.cuh"

using namespace ph;

long ph_lda(int N);

namespace {

struct BatchArgs {
  Job base;                       // the homotopy, the parameters, the layout
  int npaths;
  const double *x0;               // [npaths][2L][n]
  double *x_out;                  // [npaths][2L][n]
  ph_path_stats *stats;           // [npaths]
  ph_step_record *log;            // [npaths][log_cap] or null
  unsigned int *next;             // work queue counter
  double *ws;                     // per-block workspaces
  long ws_stride;
};

template <class P>
__global__ void __launch_bounds__(kBT) k_paths(BatchArgs a) {
  extern __shared__ double smem[];
  __shared__ int s_path;
  const long pt = 2L * P::L * a.base.n;
  Job j = a.base;
  j.ws = a.ws + (long)blockIdx.x * a.ws_stride;
  for (;;) {
    if (threadIdx.x == 0) s_path = (int)atomicAdd(a.next, 1u);
    __syncthreads();
    const int path = s_path;
    __syncthreads();
    if (path >= a.npaths) return;
    j.x0 = a.x0 + (long)path * pt;
    j.x_out = a.x_out + (long)path * pt;
    j.stats = a.stats + path;
    j.log = a.log ? a.log + (long)path * a.base.log_cap : nullptr;
    track_job<P>(j, smem);
  }
}

template <class P>
cudaError_t launch_paths(const BatchArgs &args, int grid, size_t smem, cudaStream_t st) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_paths<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_paths<P><<<grid, kBT, smem, st>>>(args);
  return cudaGetLastError();
}

template <class P>
int blocks_per_sm(size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_paths<P>, kBT, smem) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < 1 ? 1 : (nb > 2 ? 2 : nb);
}

template <class P>
cudaError_t launch_any(int L, const BatchArgs &args, int grid, size_t smem, cudaStream_t st) {
  return L == 1 ? launch_paths<F64>(args, grid, smem, st)
       : L == 2 ? launch_paths<DD>(args, grid, smem, st) : launch_paths<QD>(args, grid, smem, st);
}

// The summation's lanes per output inside the per-block kernel (the paper's
// threads per sum, Section 3.3), chosen by timing: `grid` copies of one start
// point (a full GPU of blocks, each the same work), one corrector iteration
// each (a fixed step with one update), for 1, 2, 4, 8, 16 and 32 lanes after
// one untimed launch; the fastest is kept on the system.
static cudaError_t tune_block_lanes(ph_ctx *ctx, const ph_system *f, const BatchArgs &base,
                                   int grid, size_t smem, const double *x0_first) {
  const int L = f->L;
  const long pt = 2L * L * f->n;
  BatchArgs t = base;
  cudaError_t e = ctx->btune.ensure(sizeof(double) * pt * 2 * grid + sizeof(ph_path_stats) * grid);
  if (e != cudaSuccess) return e;
  double *tx0 = ctx->btune.as<double>(), *txo = tx0 + pt * grid;
  for (int q = 0; q < grid && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(tx0 + pt * q, x0_first, sizeof(double) * pt, cudaMemcpyDeviceToDevice,
                        ctx->stream);
  t.npaths = grid;
  t.x0 = tx0;
  t.x_out = txo;
  t.stats = (ph_path_stats *)(txo + pt * grid);
  t.log = nullptr;
  t.base.log_cap = 0;
  t.base.p.fixed_steps = 1;
  t.base.p.max_newton = 1;
  t.base.p.lin_prec = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  static const int lanes[6] = {1, 2, 4, 8, 16, 32};
  float best = 1e30f;
  int choice = kSG;
  for (int v = -1; v < 6 && e == cudaSuccess; ++v) {
    t.base.sum_lanes = lanes[v < 0 ? 2 : v];          // v = -1: warm-up
    e = cudaMemsetAsync(t.next, 0, sizeof(unsigned int), ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    if (e == cudaSuccess) e = launch_any<DD>(L, t, grid, smem, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && v >= 0) {
      f->block_ms[v] = ms;
      if (ms < best) {
        best = ms;
        choice = lanes[v];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) f->block_lanes = choice;
  return e;
}

}  // namespace

// the system part of a job (shared with the serving form)
void ph_job_fill_system(Job &j, const ph_system *f, const ph_system *g) {
  j.L = f->L; j.N = f->N; j.n = f->n; j.nout = f->nout;
  j.emax = std::max(f->emax, g ? g->emax : 1);
  j.Mf = f->M; j.Mpf = f->Mp; j.maxvf = f->maxv;
  j.nvf = f->nv.as<int32_t>(); j.vidxf = f->vidx.as<int32_t>(); j.vexpf = f->vexp.as<int32_t>();
  j.optrf = f->out_ptr.as<int32_t>(); j.oslotf = f->out_slot.as<int32_t>();
  j.coeff_f = f->coeff.as<double>(); j.deg = f->deg.as<int32_t>();
  j.nsf = (long)(f->maxv + 1) * f->Mp;
  if (g) {
    j.Mg = g->M; j.Mpg = g->Mp; j.maxvg = g->maxv;
    j.nvg = g->nv.as<int32_t>(); j.vidxg = g->vidx.as<int32_t>(); j.vexpg = g->vexp.as<int32_t>();
    j.optrg = g->out_ptr.as<int32_t>(); j.oslotg = g->out_slot.as<int32_t>();
    j.coeff_g = g->coeff.as<double>();
    j.zrows_g = g->zero_rows.as<uint8_t>();
    j.nsg = (long)(g->maxv + 1) * g->Mp;
  }
  j.ldA = ph_lda(f->N);
  j.sum_lanes = f->block_lanes > 0 ? f->block_lanes : kSG;
  JobLayout o = job_layout(j.L, j.n, j.ldA, j.emax, j.nsf, j.nsg);
  j.o_x = o.o_x; j.o_dx = o.o_dx; j.o_hist = o.o_hist; j.o_ptab = o.o_ptab; j.o_spow = o.o_spow;
  j.o_A = o.o_A; j.o_W = o.o_W; j.o_fslots = o.o_fslots; j.o_gslots = o.o_gslots;
  j.o_scal = o.o_scal; j.o_t = o.o_t; j.o_g = o.o_g; j.o_h = o.o_h;
}

long ph_job_ws_doubles(const Job &j) {
  return job_layout(j.L, j.n, j.ldA, j.emax, j.nsf, j.nsg).stride;
}

extern "C" ph_status ph_block_lanes(ph_ctx *ctx, const ph_system *f, int *lanes, double *ms) {
  if (!ctx) return PH_EINVAL;
  if (!f || f->ctx != ctx || !lanes) return ph_fail(ctx, PH_EINVAL, "ph_block_lanes: invalid argument");
  *lanes = f->block_lanes > 0 ? f->block_lanes : kSG;
  if (ms)
    for (int q = 0; q < 6; ++q) ms[q] = f->block_ms[q];
  return PH_OK;
}

extern "C" ph_status ph_set_block_lanes(ph_ctx *ctx, const ph_system *f, int lanes) {
  if (!ctx) return PH_EINVAL;
  if (!f || f->ctx != ctx || (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 &&
                              lanes != 8 && lanes != 16 && lanes != 32))
    return ph_fail(ctx, PH_EINVAL, "ph_set_block_lanes: invalid argument");
  f->block_lanes = lanes;
  if (lanes == 0)
    for (int q = 0; q < 6; ++q) f->block_ms[q] = -1.0f;
  return PH_OK;
}

extern "C" ph_status ph_track_paths(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                    const double *gamma, int npaths, const double *x0,
                                    const ph_track_params *params, double *x_out,
                                    ph_path_stats *stats, ph_step_record *log, int log_cap) {
  if (!ctx) return PH_EINVAL;
  if (!f || f->ctx != ctx) return ph_fail(ctx, PH_EINVAL, "ph_track_paths: f missing or from another context");
  if (g && (g->ctx != ctx || g->L != f->L || g->N != f->N || g->n != f->n))
    return ph_fail(ctx, PH_EINVAL, "ph_track_paths: g does not match f");
  if (!gamma || !x0 || !params || !x_out || npaths < 0)
    return ph_fail(ctx, PH_EINVAL, "ph_track_paths: invalid argument");
  const ph_track_params p = *params;
  if (p.max_newton < 1 || p.max_newton > 64 || p.pred_order < 0 || p.pred_order > 8 ||
      p.relax_k < 1 || p.relax_k > 64 || p.max_steps < 0 || p.lin_prec < 0 || p.lin_prec > 3 ||
      p.fixed_rows < 0 || p.fixed_rows > 1 || (p.fixed_rows && !g) ||
      (p.fixed_steps <= 0 && !(p.max_dt > 0.0 && p.min_dt > 0.0 && p.min_dt <= p.max_dt)))
    return ph_fail(ctx, PH_EINVAL, "ph_track_paths: invalid parameters");
  if (!g) {
    if (f->N != f->n) return ph_fail(ctx, PH_EINVAL, "ph_track_paths: the total-degree start system needs N == n");
    for (int d : f->h_deg)
      if (d < 1) return ph_fail(ctx, PH_EINVAL, "ph_track_paths: f has a constant polynomial");
  }
  if (log_cap < 0 || (log_cap > 0 && !log)) return ph_fail(ctx, PH_EINVAL, "ph_track_paths: bad log");
  if (npaths == 0) return PH_OK;
  cudaSetDevice(ctx->device);
  const int L = f->L, n = f->n;
  const long pt = 2L * L * n;
  BatchArgs a;
  memset(&a, 0, sizeof a);
  ph_job_fill_system(a.base, f, g);
  a.ws_stride = ph_job_ws_doubles(a.base);
  const size_t smem = job_smem_bytes(L, n);
  const int bps = L == 1 ? blocks_per_sm<F64>(smem)
                : L == 2 ? blocks_per_sm<DD>(smem) : blocks_per_sm<QD>(smem);
  int grid = ctx->sm_count * bps;
  if (grid > npaths) grid = npaths;
  PH_CUDA(ctx, ctx->bws.ensure(sizeof(double) * (size_t)a.ws_stride * grid));
  PH_CUDA(ctx, ctx->bq.ensure(sizeof(unsigned int)));
  PH_CUDA(ctx, cudaMemsetAsync(ctx->bq.p, 0, sizeof(unsigned int), ctx->stream));

  // paths in and out (staged when they are host arrays)
  const size_t xbytes = sizeof(double) * pt * npaths;
  const double *dx0 = x0;
  if (!ph_is_device_ptr(x0)) {
    PH_CUDA(ctx, ctx->bx0.ensure(xbytes));
    PH_CUDA(ctx, cudaMemcpyAsync(ctx->bx0.p, x0, xbytes, cudaMemcpyHostToDevice, ctx->stream));
    dx0 = ctx->bx0.as<double>();
  }
  double *dxo = x_out;
  const bool host_out = !ph_is_device_ptr(x_out);
  if (host_out) {
    PH_CUDA(ctx, ctx->bxo.ensure(xbytes));
    dxo = ctx->bxo.as<double>();
  }
  PH_CUDA(ctx, ctx->bstats.ensure(sizeof(ph_path_stats) * (size_t)npaths));
  ph_step_record *dlog = nullptr;
  if (log_cap > 0) {
    PH_CUDA(ctx, ctx->blog.ensure(sizeof(ph_step_record) * (size_t)npaths * log_cap));
    dlog = ctx->blog.as<ph_step_record>();
  }
  PH_CUDA(ctx, ctx->in_gamma.ensure(sizeof(double) * 2 * L));
  PH_CUDA(ctx, cudaMemcpyAsync(ctx->in_gamma.p, gamma, sizeof(double) * 2 * L, cudaMemcpyDefault,
                               ctx->stream));

  a.base.gamma = ctx->in_gamma.as<double>();
  a.base.p = p;
  a.base.log_cap = log_cap;
  a.npaths = npaths;
  a.x0 = dx0;
  a.x_out = dxo;
  a.stats = ctx->bstats.as<ph_path_stats>();
  a.log = dlog;
  a.next = ctx->bq.as<unsigned int>();
  a.ws = ctx->bws.as<double>();
  // a batch that fills the GPU times the summation's lanes per output once
  // per system (the first time), before the paths run
  if (f->block_lanes == 0 && npaths >= ctx->sm_count) {
    PH_CUDA(ctx, tune_block_lanes(ctx, f, a, grid, smem, dx0));
    PH_CUDA(ctx, cudaMemsetAsync(ctx->bq.p, 0, sizeof(unsigned int), ctx->stream));
  }
  a.base.sum_lanes = f->block_lanes > 0 ? f->block_lanes : kSG;
  PH_CUDA(ctx, launch_any<DD>(L, a, grid, smem, ctx->stream));
  if (host_out) PH_CUDA(ctx, cudaMemcpyAsync(x_out, dxo, xbytes, cudaMemcpyDeviceToHost, ctx->stream));
  if (stats)
    PH_CUDA(ctx, cudaMemcpyAsync(stats, a.stats, sizeof(ph_path_stats) * (size_t)npaths,
                                 cudaMemcpyDefault, ctx->stream));
  if (log_cap > 0)
    PH_CUDA(ctx, cudaMemcpyAsync(log, dlog, sizeof(ph_step_record) * (size_t)npaths * log_cap,
                                 cudaMemcpyDefault, ctx->stream));
  PH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PH_OK;
}
