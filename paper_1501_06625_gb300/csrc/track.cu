// track.cu -- ph_track_path: one solution path tracked entirely on the device.
//
// The paper keeps the step control on the host and copies the two norms of
// each Newton iteration back (Section 3.1, Fig. 2, Fig. 3).  On GB300 a host
// round trip costs more than a small step's kernels, so here the same
// decisions run in one-thread kernels on the device and the whole path is a
// single CUDA graph launch: a conditional WHILE node repeats the body
//   step_begin  controller: t := min(1, t + dt), reset the corrector
//   predict     extrapolation through the last accepted points (Section 3.1)
//   max_newton x [ prep, ad, sum      h, J and -h into [J | -h], ||h||
//                  check_res          fail if ||h|| grew, succeed if small
//                  mgs                dx by MGS + back substitution, ||dx||
//                  update             x += dx
//                  check_dx ]         succeed if ||dx|| small
//   step_end    accept (history push) or reject, controller update, log,
//               and ends the loop when the path is finished
// until step_end clears the condition.  Kernels gate themselves on flags in
// PathState, so a corrector that finished early costs only empty launches.
// The host reads the state once, after the path.
//
// The precision form (lin_prec 1) records a second kernel set beside each
// iteration's: h alone in working precision (its leading limbs scaled by 2^-e,
// e the exponent of max |h_i|), the Jacobian in IEEE double from the leading
// limbs, MGS in double, and x += 2^e dx in working precision.  The control
// kernels choose the set per step through two gates: double while t is below
// the end game, working precision at t = 1 and when a failed step is corrected
// again (the retry runs the step body once more at the same t, in working
// precision).  The rules (one extra iteration, escalation) are those of the
// many-path form.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "ctrl.h"
#include "internal.h"
#include "mp.cuh"

using namespace ph;

long ph_lda(int N);

namespace {

constexpr int kHist = 16;          // ring of accepted points (pred_order <= 8)

// The gates of the precision form's two kernel sets: the working-precision set
// runs while the corrector runs and solves in working precision, the double
// set while it runs and solves in double.
__device__ __forceinline__ void set_gates(PathState *st) {
  st->gate_wp = st->skip_nt || st->lin != 0;
  st->gate_lp = st->skip_nt || st->lin == 0;
}

__global__ void k_step_begin(PathState *st, ph_track_params p, int L) {
  st->iterations += 1;
  if (st->timeout && !st->ctrl.done) {     // a bounded wait ran out: stop the path
    st->ctrl.done = 1;
    st->ctrl.status = PH_TIMEOUT;
  }
  if (st->ctrl.done) {
    st->skip_step = 1;
    st->skip_nt = 1;
    set_gates(st);
    return;
  }
  double tn;
  if (st->retry) {                         // the failed step again, in working precision
    st->retry = 0;
    st->pass = 1;
    tn = st->t_new;
  } else {
    tn = ctrl_next_t(&st->ctrl, &p);
    if (tn < 0.0) {
      st->skip_step = 1;
      st->skip_nt = 1;
      set_gates(st);
      return;
    }
    st->pass = 0;
    st->force = 0;
  }
  st->t_new = tn;
  st->t_dev[0] = tn;
  for (int l = 1; l < L; ++l) st->t_dev[l] = 0.0;
  st->nt_done = 0;
  st->nt_success = p.fixed_steps > 0 ? 1 : 0;
  st->nt_iters = 0;
  st->nt_updates = 0;
  st->last_res = p.max_res;
  st->res_bits = 0;
  st->dx_bits = 0;
  st->mgs_status = 0;
  st->skip_step = 0;
  st->skip_nt = 0;
  st->escalate = 0;
  st->onpath = 0;
  st->linear = 0;
  const double endgame = p.endgame_t > 0.0 ? p.endgame_t : 1.0;
  st->lin = (p.lin_prec == 1 && !(tn >= endgame) && st->force != 2 && !st->wp_rest) ? 1 : 0;
  set_gates(st);
}

// x(t_new) = sum_j w_j x(t_j) over the last m accepted points, with the
// Lagrange weights w_j = prod_{l != j} (t_new - t_l) / (t_j - t_l) of the
// interpolating polynomial of degree m - 1 (computed by m threads per block).
template <class P>
__global__ void k_predict(PathState *st, const double *__restrict__ hist, double *__restrict__ xw,
                          int n, int pred_order) {
  if (st->skip_step) return;
  typedef typename P::real real;
  __shared__ real w[kHist];
  __shared__ int s_slot[kHist];
  const int cnt = st->hist_count, head = st->hist_head;
  const int m = cnt < pred_order + 1 ? cnt : pred_order + 1;
  const double tn = st->t_new;
  if ((int)threadIdx.x < m) {
    int j = threadIdx.x;
    int sj = (head - (m - 1 - j) + kHist) % kHist;
    double tj = st->hist_t[sj];
    real num = P::from(1.0), den = P::from(1.0);
    for (int l = 0; l < m; ++l) {
      if (l == j) continue;
      double tl = st->hist_t[(head - (m - 1 - l) + kHist) % kHist];
      real a, b;
      double s, e;
      two_sum(tn, -tl, s, e);          // t_new - t_l exactly
      a = P::zero(); P::set_limb(a, 0, s); if (P::L > 1) P::set_limb(a, 1, e);
      two_sum(tj, -tl, s, e);
      b = P::zero(); P::set_limb(b, 0, s); if (P::L > 1) P::set_limb(b, 1, e);
      num = P::mul(num, a);
      den = P::mul(den, b);
    }
    w[j] = m == 1 ? P::from(1.0) : P::div(num, den);
    s_slot[j] = sj;
  }
  __syncthreads();
  const long pt = 2L * P::L * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    cx<P> acc = c_zero<P>();
    for (int j = 0; j < m; ++j)
      acc = c_add<P>(acc, c_mul_real<P>(c_load<P>(hist + s_slot[j] * pt, n, i), w[j]));
    c_store<P>(xw, n, i, acc);
  }
}

__global__ void k_check_res(PathState *st, ph_track_params p) {
  if (st->skip_nt) return;
  double r = __longlong_as_double((long long)st->res_bits);
  st->res = r;
  st->nt_iters += 1;
  st->newton_iters += 1;
  st->res_last = r;
  st->dx_bits = 0;
  st->mgs_status = 0;
  // the exponent by which the double solve's right-hand side is scaled
  st->scale_e = (r > 0.0 && isfinite(r)) ? ilogb(r) : 0;
  if (p.fixed_steps <= 0) {
    if (!(r <= st->last_res) || !isfinite(r)) {     // residual grew (or NaN): fail
      st->nt_done = 1;
      st->nt_success = 0;
      st->skip_nt = 1;
    } else if (r < ctrl_tol_res(&p, st->t_new)) {
      st->nt_done = 1;
      st->nt_success = 1;
      st->skip_nt = 1;
    }
  }
  set_gates(st);
}

// The double solve's right-hand side: -h's leading limbs times 2^-e, so that
// neither it nor the update underflows however small the residual.
__global__ void k_rhs_scale(const PathState *st, double *__restrict__ rhs, long plane, int N) {
  if (st->gate_lp) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    const int e = st->scale_e;
    rhs[i] = ldexp(rhs[i], -e);
    rhs[plane + i] = ldexp(rhs[plane + i], -e);
  }
}

// x += dx: from the working-precision solve (lowp 0, dx in the L-limb layout)
// or from the double solve (lowp 1, dx [re|im][n] scaled back by 2^e).
template <class P>
__global__ void k_update(PathState *st, double *__restrict__ xw, const double *__restrict__ dx,
                         int n, int fixed, int lowp) {
  if (st->skip_nt || st->lin != lowp) return;
  const bool bad = st->mgs_status != 0;
  if (bad && !fixed) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    cx<P> d;
    if (bad) {
      d = c_from<P>(NAN, NAN);
    } else if (lowp) {
      const int e = st->scale_e;
      d = c_from<P>(ldexp(dx[i], e), ldexp(dx[n + i], e));
    } else {
      d = c_load<P>(dx, n, i);
    }
    c_store<P>(xw, n, i, c_add<P>(c_load<P>(xw, n, i), d));
  }
}

// The update test.  After a double solve, also the condition estimate
// max r_kk / min r_kk from the solve's pivot norms (nrm2[k] = r_kk^2, k < n),
// the escalation rule, and one iteration beyond max_newton when the previous
// update was below sqrt(tol_dx) (the working-precision corrector would have
// squared it below tol_dx by now; the double one contracts by kappa u_double).
__global__ void k_check_dx(PathState *st, ph_track_params p, const double *__restrict__ nrm2,
                           int n) {
  if (st->skip_nt) return;
  __shared__ double s_mx[32], s_mn[32];
  const int lin = st->lin, tid = threadIdx.x;
  double mx = 0.0, mn = INFINITY;
  if (lin) {
    for (int k = tid; k < n; k += blockDim.x) {
      const double v = nrm2[k];
      mx = fmax(mx, v);
      mn = fmin(mn, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
      mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    }
    if ((tid & 31) == 0) {
      s_mx[tid >> 5] = mx;
      s_mn[tid >> 5] = mn;
    }
    __syncthreads();
    if (tid == 0)
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        mx = fmax(mx, s_mx[w]);
        mn = fmin(mn, s_mn[w]);
      }
  }
  if (tid != 0) return;
  const bool fixed = p.fixed_steps > 0;
  if (lin) {
    const double c = st->mgs_status == 0 ? sqrt(mx / mn) : INFINITY;
    st->solves_f64 += 1;
    st->cond = c;
    if (!(c * 0x1p-53 <= kEscalateRho)) st->escalate = 2;
  }
  if (st->mgs_status != 0 && !fixed) {               // singular Jacobian: fail
    st->nt_done = 1;
    st->nt_success = 0;
    st->skip_nt = 1;
    set_gates(st);
    return;
  }
  double d = st->mgs_status != 0 ? NAN : __longlong_as_double((long long)st->dx_bits);
  if (lin) d = ldexp(d, st->scale_e);
  const double tol_dx = ctrl_tol_dx(&p, st->t_new);
  const bool prev_on_path = lin && st->nt_updates >= 1 && st->dxn <= sqrt(tol_dx);
  if (prev_on_path) st->onpath = 1;
  if (lin && st->nt_updates >= 2 && linear_contraction(st->dxn2, st->dxn, d)) st->linear = 1;
  st->dxn2 = st->dxn;
  st->dxn = d;
  st->dx_last = d;
  st->nt_updates += 1;
  st->updates += 1;
  st->res_bits = 0;
  if (!fixed) {
    if (!isfinite(d)) {
      st->nt_done = 1;
      st->nt_success = 0;
      st->skip_nt = 1;
      set_gates(st);
      return;
    }
    if (d < tol_dx) {
      st->nt_done = 1;
      st->nt_success = 1;
      st->skip_nt = 1;
      set_gates(st);
      return;
    }
    st->last_res = st->res;
  }
  const int max_it = fixed ? p.max_newton : p.max_newton + 1;
  if (st->nt_iters >= p.max_newton && !(prev_on_path && st->nt_iters < max_it)) {
    st->nt_done = 1;                                 // out of iterations
    st->nt_success = fixed ? 1 : 0;
    st->skip_nt = 1;
  }
  set_gates(st);
}

template <class P>
__global__ void k_step_end(PathState *st, ph_track_params p, double *__restrict__ hist,
                           const double *__restrict__ xw, int n, ph_step_record *log, int log_cap,
                           cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ int s_ok, s_slot, s_retry;
  __shared__ double s_max;
  if (st->skip_step) {
    if (use_cond && threadIdx.x == 0 && st->ctrl.done) cudaGraphSetConditional(cond, 0);
    return;
  }
  if (threadIdx.x == 0) {
    // the precision form: a failed step whose corrector must not be trusted is
    // corrected once more at the same t, in working precision (k_step_begin)
    int ok = st->nt_success;
    s_retry = 0;
    if (p.lin_prec != 0 && !ok) {
      if (st->onpath) st->escalate = 2;
      // a failed low-precision corrector that contracted only linearly: its
      // solves limit it; the rest of the path runs in working precision
      if (st->linear && p.fixed_steps <= 0) {
        st->escalate = 2;
        st->wp_rest = 1;
      }
      if (st->pass == 0 && st->escalate && p.fixed_steps <= 0) {
        st->force = st->escalate;
        st->escalated += 1;
        st->retry = 1;
        s_retry = 1;
      }
    }
  }
  __syncthreads();
  if (s_retry) return;
  if (threadIdx.x == 0) {
    int ok = st->nt_success;
    st->steps += 1;
    if (ok) st->accepted += 1; else st->rejected += 1;
    if (log && st->log_len < log_cap) {
      ph_step_record r;
      r.t = st->t_new;
      r.res = st->res;
      r.dx = st->dxn;
      r.accepted = ok;
      r.updates = st->nt_updates;
      log[st->log_len] = r;
    }
    st->log_len += 1;
    ctrl_report(&st->ctrl, &p, st->t_new, ok);
    int slot = (st->hist_head + 1) % kHist;
    if (ok) {
      st->hist_head = slot;
      st->hist_t[slot] = st->t_new;
      st->hist_count = st->hist_count < kHist ? st->hist_count + 1 : kHist;
    }
    s_ok = ok;
    s_slot = slot;
    s_max = 0.0;
  }
  __syncthreads();
  if (!s_ok) {
    if (use_cond && threadIdx.x == 0 && st->ctrl.done) cudaGraphSetConditional(cond, 0);
    return;
  }
  const long pt = 2L * P::L * n;
  double mymax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    cx<P> xi = c_load<P>(xw, n, i);
    c_store<P>(hist + s_slot * pt, n, i, xi);
    double a = c_mag_lead<P>(xi);
    if (!(a <= mymax)) mymax = a;
  }
  // max over the block through the bit patterns (non-negative or NaN)
  atomicMax((unsigned long long *)&s_max, (unsigned long long)__double_as_longlong(mymax));
  __syncthreads();
  if (threadIdx.x == 0) {
    if (p.fixed_steps <= 0 && !st->ctrl.done && !(s_max <= p.max_x)) {
      st->ctrl.done = 1;
      st->ctrl.status = PH_DIVERGED;
    }
    if (use_cond && st->ctrl.done) cudaGraphSetConditional(cond, 0);
  }
}

struct TrackGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  // what the graph was built for
  uint64_t f_serial = 0, g_serial = 0;    // the systems (0: none)
  ph_track_params p;
  void *bufs[16] = {};
  int log_cap = -1;
  long kernels_per_step = 0;
  cudaStream_t stream = nullptr;
  bool valid = false;
};

struct TrackCache {
  TrackGraph tg;
  cudaStream_t cap = nullptr;      // private stream used for capture
  int32_t *done_host = nullptr;    // pinned flag for host-side step control
};

}  // namespace

// ---- graph cache per context -------------------------------------------------------
static std::mutex g_cache_mu;
static std::map<ph_ctx *, TrackCache *> g_cache;

static TrackCache *get_cache(ph_ctx *ctx) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_cache.find(ctx);
  if (it != g_cache.end()) return it->second;
  TrackCache *c = new TrackCache();
  g_cache[ctx] = c;
  return c;
}

static void drop_graph(TrackGraph &tg) {
  if (tg.exec) cudaGraphExecDestroy(tg.exec);
  if (tg.graph) cudaGraphDestroy(tg.graph);
  tg = TrackGraph();
}

void ph_track_release(ph_ctx *ctx) {
  TrackCache *c = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(ctx);
    if (it == g_cache.end()) return;
    c = it->second;
    g_cache.erase(it);
  }
  drop_graph(c->tg);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->done_host) cudaFreeHost(c->done_host);
  delete c;
}

// Records the body of one predictor-corrector step on `s`.
static cudaError_t record_step(ph_ctx *ctx, cudaStream_t s, const ph_system *f,
                               const ph_system *g, const double *gamma,
                               const ph_track_params &p, PathState *st, double *hist, double *xw,
                               double *A, long ldA, double *dx, ph_step_record *log, int log_cap,
                               cudaGraphConditionalHandle cond, int use_cond) {
  const int L = f->L, n = f->n, N = f->N;
  const long Ap = (long)(n + 1) * ldA;
  cudaStream_t saved = ctx->stream;
  ctx->stream = s;
  cudaError_t e = cudaSuccess;
  k_step_begin<<<1, 1, 0, s>>>(st, p, L);
  int pb = 128, pg = (n + pb - 1) / pb;
  if (L == 1) k_predict<F64><<<pg, pb, 0, s>>>(st, hist, xw, n, p.pred_order);
  else if (L == 2) k_predict<DD><<<pg, pb, 0, s>>>(st, hist, xw, n, p.pred_order);
  else k_predict<QD><<<pg, pb, 0, s>>>(st, hist, xw, n, p.pred_order);
  // the precision form: both kernel sets, and one iteration more (k_check_dx)
  const bool mixed = p.lin_prec == 1;
  const int n_it = mixed && p.fixed_steps <= 0 ? p.max_newton + 1 : p.max_newton;
  const int *gwp = mixed ? &st->gate_wp : &st->skip_nt;
  const uint8_t *frows = p.fixed_rows && g ? g->zero_rows.as<uint8_t>() : nullptr;
  double *rhs = A + (long)n * ldA;
  const int fx = p.fixed_steps > 0;
  const unsigned ub = (unsigned)((n + 127) / 128);
  for (int it = 0; it < n_it && e == cudaSuccess; ++it) {
    e = ph_eval_launch(ctx, f, g, gamma, p.relax_k, st->t_dev, xw, nullptr, A, ldA, Ap, rhs, Ap,
                       gwp, &st->res_bits, frows);
    if (e == cudaSuccess && mixed)
      e = ph_eval_values_launch(ctx, f, g, gamma, p.relax_k, st->t_dev, xw, rhs, Ap, &st->gate_lp,
                                &st->res_bits, frows);
    if (e != cudaSuccess) break;
    k_check_res<<<1, 1, 0, s>>>(st, p);
    if (mixed) {
      k_rhs_scale<<<(N + 127) / 128, 128, 0, s>>>(st, rhs, Ap, N);
      e = ph_eval_launch_f64(ctx, f, g, gamma, p.relax_k, st->t_dev, xw, A, ldA, Ap, &st->gate_lp,
                             frows);
      if (e != cudaSuccess) break;
    }
    e = ph_mgs_launch(ctx, L, N, n, A, ldA, dx, st, gwp, nullptr);
    if (e == cudaSuccess && mixed) e = ph_mgs_launch(ctx, 1, N, n, A, ldA, dx, st, &st->gate_lp, nullptr);
    if (e != cudaSuccess) break;
    for (int lowp = 0; lowp <= (mixed ? 1 : 0); ++lowp) {
      if (L == 1) k_update<F64><<<ub, 128, 0, s>>>(st, xw, dx, n, fx, lowp);
      else if (L == 2) k_update<DD><<<ub, 128, 0, s>>>(st, xw, dx, n, fx, lowp);
      else k_update<QD><<<ub, 128, 0, s>>>(st, xw, dx, n, fx, lowp);
    }
    k_check_dx<<<1, 128, 0, s>>>(st, p, ctx->nrm2.as<double>(), n);
  }
  if (e == cudaSuccess) {
    int eb = n < 256 ? 128 : 256;
    if (L == 1)
      k_step_end<F64><<<1, eb, 0, s>>>(st, p, hist, xw, n, log, log_cap, cond, use_cond);
    else if (L == 2)
      k_step_end<DD><<<1, eb, 0, s>>>(st, p, hist, xw, n, log, log_cap, cond, use_cond);
    else k_step_end<QD><<<1, eb, 0, s>>>(st, p, hist, xw, n, log, log_cap, cond, use_cond);
    e = cudaGetLastError();
  }
  ctx->stream = saved;
  return e;
}

static ph_status build_graph(ph_ctx *ctx, TrackCache *c, const ph_system *f, const ph_system *g,
                             const double *gamma, const ph_track_params &p, PathState *st,
                             double *hist, double *xw, double *A, long ldA, double *dx,
                             ph_step_record *log, int log_cap) {
  drop_graph(c->tg);
  ph_mgs_tune(ctx, f->L, f->N, f->n);                // measured now: the capture cannot
  if (p.lin_prec == 1) ph_mgs_tune(ctx, 1, f->N, f->n);
  ph_sum_tune(ctx, f, g);
  if (!c->cap) PH_CUDA(ctx, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  TrackGraph &tg = c->tg;
  PH_CUDA(ctx, cudaGraphCreate(&tg.graph, 0));
  cudaGraph_t body = tg.graph;
  cudaGraphConditionalHandle cond = 0;
  const int use_cond = p.control == 0;
  if (use_cond) {
    // a WHILE node repeats the step body until k_step_end clears the condition
    PH_CUDA(ctx, cudaGraphConditionalHandleCreate(&cond, tg.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    PH_CUDA(ctx, cudaGraphAddNode(&node, tg.graph, nullptr, nullptr, 0, &cp));
    body = cp.conditional.phGraph_out[0];
  }
  PH_CUDA(ctx, cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  cudaError_t e = record_step(ctx, c->cap, f, g, gamma, p, st, hist, xw, A, ldA, dx, log, log_cap,
                              cond, use_cond);
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(c->cap, &out);
  if (e != cudaSuccess) { drop_graph(tg); return ph_cuda_fail(ctx, e, "capture of the step"); }
  if (e2 != cudaSuccess) { drop_graph(tg); return ph_cuda_fail(ctx, e2, "cudaStreamEndCapture"); }
  size_t nodes = 0;
  cudaGraphGetNodes(body, nullptr, &nodes);
  tg.kernels_per_step = (long)nodes;
  e = cudaGraphInstantiate(&tg.exec, tg.graph, 0);
  if (e != cudaSuccess) { drop_graph(tg); return ph_cuda_fail(ctx, e, "cudaGraphInstantiate"); }
  tg.f_serial = f->serial;
  tg.g_serial = g ? g->serial : 0;
  tg.p = p;
  tg.log_cap = log_cap;
  tg.valid = true;
  return PH_OK;
}

// ph_track_path on an executing context `ctx` that may differ from the
// context the systems were loaded in, as long as both are on the same device
// (the serving loop runs its large jobs on a context of its own).
ph_status ph_track_path_exec(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                             const double *gamma, const double *x0,
                             const ph_track_params *params, double *x_out,
                             ph_path_stats *stats, ph_step_record *log, int log_cap) {
  if (!ctx) return PH_EINVAL;
  if (!f || !f->ctx || f->ctx->device != ctx->device)
    return ph_fail(ctx, PH_EINVAL, "ph_track_path: f missing or from another device");
  if (g && (g->ctx != f->ctx || g->L != f->L || g->N != f->N || g->n != f->n))
    return ph_fail(ctx, PH_EINVAL, "ph_track_path: g does not match f");
  if (!gamma || !x0 || !params || !x_out) return ph_fail(ctx, PH_EINVAL, "ph_track_path: NULL argument");
  const ph_track_params p = *params;
  if (p.max_newton < 1 || p.max_newton > 64 || p.pred_order < 0 || p.pred_order > 8 ||
      p.relax_k < 1 || p.relax_k > 64 || p.control < 0 || p.control > 1 || p.max_steps < 0 ||
      p.fixed_rows < 0 || p.fixed_rows > 1 || (p.fixed_rows && !g) ||
      (p.fixed_steps <= 0 && !(p.max_dt > 0.0 && p.min_dt > 0.0 && p.min_dt <= p.max_dt)))
    return ph_fail(ctx, PH_EINVAL, "ph_track_path: invalid parameters");
  if (p.lin_prec != 0 && p.lin_prec != 1)
    return ph_fail(ctx, PH_EINVAL,
                   "ph_track_path: lin_prec 2 and 3 are taken by ph_track_paths and the serving loop");
  if (!g) {
    if (f->N != f->n) return ph_fail(ctx, PH_EINVAL, "ph_track_path: the total-degree start system needs N == n");
    for (int d : f->h_deg)
      if (d < 1) return ph_fail(ctx, PH_EINVAL, "ph_track_path: f has a constant polynomial");
  }
  if (log_cap < 0 || (log_cap > 0 && !log)) return ph_fail(ctx, PH_EINVAL, "ph_track_path: bad log");
  cudaSetDevice(ctx->device);
  const int L = f->L, n = f->n, N = f->N;
  const long pt = 2L * L * n;
  const long ldA = ph_lda(N);

  // host inputs: gamma and x0 (copied in; a non-finite start point ends here)
  std::vector<double> hx0(pt), hg(2 * L);
  PH_CUDA(ctx, cudaMemcpy(hx0.data(), x0, sizeof(double) * pt, cudaMemcpyDefault));
  PH_CUDA(ctx, cudaMemcpy(hg.data(), gamma, sizeof(double) * 2 * L, cudaMemcpyDefault));
  for (double v : hx0)
    if (!std::isfinite(v)) {
      if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->launches = 0;
        stats->status = PH_NONFINITE;
      }
      PH_CUDA(ctx, cudaMemcpy(x_out, x0, sizeof(double) * pt, cudaMemcpyDefault));
      return PH_NONFINITE;
    }

  PH_CUDA(ctx, ctx->state.ensure(sizeof(PathState)));
  PH_CUDA(ctx, ctx->hist.ensure(sizeof(double) * pt * kHist));
  PH_CUDA(ctx, ctx->xw.ensure(sizeof(double) * pt));
  PH_CUDA(ctx, ctx->dxv.ensure(sizeof(double) * pt));
  PH_CUDA(ctx, ctx->A.ensure(sizeof(double) * 2 * L * (size_t)(n + 1) * ldA));
  PH_CUDA(ctx, ctx->in_gamma.ensure(sizeof(double) * 2 * L));
  PH_CUDA(ctx, ctx->logbuf.ensure(sizeof(ph_step_record) * (log_cap > 0 ? log_cap : 1)));
  // buffers the evaluation and the solver grow on demand: size them now so the
  // captured graph's pointers stay valid
  {
    int emax = f->emax > (g ? g->emax : 0) ? f->emax : g->emax;
    int ntab = emax > 2 ? emax - 1 : 1;
    long fs = (long)(f->maxv + 1) * f->Mp, gs = g ? (long)(g->maxv + 1) * g->Mp : 0;
    PH_CUDA(ctx, ctx->ptab.ensure(sizeof(double) * 2 * L * (size_t)n * ntab));
    PH_CUDA(ctx, ctx->scal.ensure(sizeof(double) * 3 * L));
    PH_CUDA(ctx, ctx->spow.ensure(sizeof(double) * 4 * L * (size_t)n));
    PH_CUDA(ctx, ctx->slots.ensure(sizeof(double) * 2 * L * (size_t)(fs + gs + 1)));
    PH_CUDA(ctx, ctx->R.ensure(sizeof(double) * 2 * L * (size_t)(n + 1) * (n + 1)));
    PH_CUDA(ctx, ctx->nrm2.ensure(sizeof(double) * 2 * L * (size_t)(n + 1)));
    PH_CUDA(ctx, ctx->irkk.ensure(sizeof(double) * L * (size_t)n));
    PH_CUDA(ctx, ctx->flags.ensure(sizeof(int) * (size_t)(n + 1)));
  }
  PathState *st = ctx->state.as<PathState>();
  double *hist = ctx->hist.as<double>(), *xw = ctx->xw.as<double>(), *dx = ctx->dxv.as<double>();
  double *A = ctx->A.as<double>(), *dgam = ctx->in_gamma.as<double>();
  ph_step_record *dlog = log_cap > 0 ? ctx->logbuf.as<ph_step_record>() : nullptr;

  // initial state: controller at t = 0, the start point as the only history point
  PathState h0;
  memset(&h0, 0, sizeof h0);
  ctrl_init(&h0.ctrl, &p);
  h0.hist_count = 1;
  h0.hist_head = 0;
  h0.hist_t[0] = 0.0;
  PH_CUDA(ctx, cudaMemcpyAsync(st, &h0, sizeof h0, cudaMemcpyHostToDevice, ctx->stream));
  PH_CUDA(ctx, cudaMemsetAsync(ctx->flags.p, 0, sizeof(int) * (size_t)(n + 1), ctx->stream));
  PH_CUDA(ctx, cudaMemcpyAsync(hist, hx0.data(), sizeof(double) * pt, cudaMemcpyHostToDevice, ctx->stream));
  PH_CUDA(ctx, cudaMemcpyAsync(dgam, hg.data(), sizeof(double) * 2 * L, cudaMemcpyHostToDevice, ctx->stream));

  TrackCache *c = get_cache(ctx);
  void *bufs[16] = {st, hist, xw, dx, A, dgam, dlog, ctx->slots.p, ctx->ptab.p, ctx->scal.p,
                    ctx->R.p, ctx->nrm2.p, ctx->irkk.p, ctx->flags.p, ctx->spow.p, nullptr};
  bool same = c->tg.valid && c->tg.f_serial == f->serial &&
              c->tg.g_serial == (g ? g->serial : 0) && c->tg.log_cap == log_cap &&
              memcmp(&c->tg.p, &p, sizeof p) == 0 && memcmp(c->tg.bufs, bufs, sizeof bufs) == 0 &&
              c->tg.stream == ctx->stream;
  if (!same) {
    // ensure the scratch the kernels grow is already at its final size
    ph_status s = build_graph(ctx, c, f, g, dgam, p, st, hist, xw, A, ldA, dx, dlog, log_cap);
    if (s != PH_OK) return s;
    memcpy(c->tg.bufs, bufs, sizeof bufs);
    c->tg.stream = ctx->stream;
  }
  PathState hs;
  if (p.control == 0) {
    PH_CUDA(ctx, cudaGraphLaunch(c->tg.exec, ctx->stream));
  } else {
    // host-side step control: one step per launch, the controller's done
    // flag read back after each (a few bytes per step, Section 3.1)
    if (!c->done_host) PH_CUDA(ctx, cudaMallocHost(&c->done_host, sizeof(int32_t)));
    for (;;) {
      PH_CUDA(ctx, cudaGraphLaunch(c->tg.exec, ctx->stream));
      PH_CUDA(ctx, cudaMemcpyAsync(c->done_host, &st->ctrl.done, sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, ctx->stream));
      PH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (*c->done_host) break;
    }
  }
  PH_CUDA(ctx, cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // the last accepted point
  PH_CUDA(ctx, cudaMemcpy(x_out, hist + hs.hist_head * pt, sizeof(double) * pt, cudaMemcpyDefault));
  if (log_cap > 0) {
    int nl = hs.log_len < log_cap ? hs.log_len : log_cap;
    if (nl > 0)
      PH_CUDA(ctx, cudaMemcpy(log, dlog, sizeof(ph_step_record) * nl, cudaMemcpyDefault));
  }
  ph_status status = hs.timeout ? PH_TIMEOUT : (ph_status)hs.ctrl.status;
  if (stats) {
    stats->status = status;
    stats->steps = hs.steps;
    stats->accepted = hs.accepted;
    stats->rejected = hs.rejected;
    stats->newton_iters = hs.newton_iters;
    stats->updates = hs.updates;
    stats->t_final = hs.hist_t[hs.hist_head];
    stats->res = hs.res_last;
    stats->dx = hs.dx_last;
    stats->launches = (int64_t)hs.iterations * c->tg.kernels_per_step;
    stats->solves_f64 = hs.solves_f64;
    stats->solves_f32 = 0;
    stats->escalated = hs.escalated;
    stats->wp_rest = hs.wp_rest;
    stats->cond = hs.cond;
  }
  if (status == PH_TIMEOUT) return ph_fail(ctx, PH_TIMEOUT, "ph_track_path: a grid barrier timed out");
  return status;
}

extern "C" ph_status ph_track_path(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                   const double *gamma, const double *x0,
                                   const ph_track_params *params, double *x_out,
                                   ph_path_stats *stats, ph_step_record *log, int log_cap) {
  if (!ctx) return PH_EINVAL;
  if (!f || f->ctx != ctx) return ph_fail(ctx, PH_EINVAL, "ph_track_path: f missing or from another context");
  if (g && g->ctx != ctx) return ph_fail(ctx, PH_EINVAL, "ph_track_path: g does not match f");
  return ph_track_path_exec(ctx, f, g, gamma, x0, params, x_out, stats, log, log_cap);
}

// ---- measurement support ----------------------------------------------------------

extern "C" ph_status ph_profile_newton(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                       const double *gamma, int k, const double *t,
                                       const double *x, int reps, double *ms_out) {
  if (!ctx) return PH_EINVAL;
  if (!f || f->ctx != ctx || !gamma || !t || !x || !ms_out || reps < 1 || k < 1)
    return ph_fail(ctx, PH_EINVAL, "ph_profile_newton: invalid argument");
  if (g && (g->ctx != ctx || g->L != f->L || g->N != f->N || g->n != f->n))
    return ph_fail(ctx, PH_EINVAL, "ph_profile_newton: g does not match f");
  if (!g && f->N != f->n) return ph_fail(ctx, PH_EINVAL, "ph_profile_newton: needs N == n");
  cudaSetDevice(ctx->device);
  const int L = f->L, n = f->n, N = f->N;
  const long ldA = ph_lda(N), Ap = (long)(n + 1) * ldA;
  PH_CUDA(ctx, ctx->A.ensure(sizeof(double) * 2 * L * (size_t)Ap));
  PH_CUDA(ctx, ctx->dxv.ensure(sizeof(double) * 2 * L * (size_t)n));
  PH_CUDA(ctx, ctx->state.ensure(sizeof(PathState)));
  PH_CUDA(ctx, ctx->in_x.ensure(sizeof(double) * 2 * L * (size_t)n));
  PH_CUDA(ctx, ctx->in_gamma.ensure(sizeof(double) * 2 * L));
  PH_CUDA(ctx, ctx->in_t.ensure(sizeof(double) * L));
  PH_CUDA(ctx, cudaMemcpyAsync(ctx->in_x.p, x, sizeof(double) * 2 * L * n, cudaMemcpyDefault, ctx->stream));
  PH_CUDA(ctx, cudaMemcpyAsync(ctx->in_gamma.p, gamma, sizeof(double) * 2 * L, cudaMemcpyDefault, ctx->stream));
  PH_CUDA(ctx, cudaMemcpyAsync(ctx->in_t.p, t, sizeof(double) * L, cudaMemcpyDefault, ctx->stream));
  PH_CUDA(ctx, cudaMemsetAsync(ctx->state.p, 0, sizeof(PathState), ctx->stream));
  PH_CUDA(ctx, ctx->flags.ensure(sizeof(int) * (size_t)(n + 1)));
  PH_CUDA(ctx, cudaMemsetAsync(ctx->flags.p, 0, sizeof(int) * (size_t)(n + 1), ctx->stream));
  double *A = ctx->A.as<double>();
  PathState *st = ctx->state.as<PathState>();
  cudaEvent_t ev[5];
  for (int i = 0; i < 5; ++i) PH_CUDA(ctx, cudaEventCreate(&ev[i]));
  double acc[4] = {0, 0, 0, 0};
  ph_status status = PH_OK;
  for (int r = 0; r < reps + 1 && status == PH_OK; ++r) {
    cudaError_t e = cudaSuccess;
    // the three evaluation kernels one at a time (the launcher issues all
    // three; its segments are timed by splitting it: prep+ad+sum, then
    // prep alone and prep+ad are derived from separate runs below)
    cudaEventRecord(ev[0], ctx->stream);
    e = ph_eval_launch_part(ctx, f, g, ctx->in_gamma.as<double>(), k, ctx->in_t.as<double>(),
                            ctx->in_x.as<double>(), nullptr, A, ldA, Ap, A + (long)n * ldA, Ap,
                            nullptr, nullptr, 1);
    cudaEventRecord(ev[1], ctx->stream);
    if (e == cudaSuccess)
      e = ph_eval_launch_part(ctx, f, g, ctx->in_gamma.as<double>(), k, ctx->in_t.as<double>(),
                              ctx->in_x.as<double>(), nullptr, A, ldA, Ap, A + (long)n * ldA, Ap,
                              nullptr, nullptr, 2);
    cudaEventRecord(ev[2], ctx->stream);
    if (e == cudaSuccess)
      e = ph_eval_launch_part(ctx, f, g, ctx->in_gamma.as<double>(), k, ctx->in_t.as<double>(),
                              ctx->in_x.as<double>(), nullptr, A, ldA, Ap, A + (long)n * ldA, Ap,
                              nullptr, nullptr, 4);
    cudaEventRecord(ev[3], ctx->stream);
    if (e == cudaSuccess) e = ph_mgs_launch(ctx, L, N, n, A, ldA, ctx->dxv.as<double>(), st, nullptr, nullptr);
    cudaEventRecord(ev[4], ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) { status = ph_cuda_fail(ctx, e, "ph_profile_newton"); break; }
    if (r == 0) continue;                 // the first pass warms up
    for (int i = 0; i < 4; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      acc[i] += ms;
    }
  }
  for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
  if (status != PH_OK) return status;
  PathState hs;
  PH_CUDA(ctx, cudaMemcpy(&hs, st, sizeof hs, cudaMemcpyDeviceToHost));
  if (hs.timeout) return ph_fail(ctx, PH_TIMEOUT, "ph_profile_newton: a grid barrier timed out");
  for (int i = 0; i < 4; ++i) ms_out[i] = acc[i] / reps;
  return PH_OK;
}

namespace {
__global__ void k_dfma_peak(double *out, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = __fma_rn(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" ph_status ph_fp64_peak(ph_ctx *ctx, double ms_target, double *gops) {
  if (!ctx || !gops || !(ms_target > 0.0)) return ph_fail(ctx, PH_EINVAL, "ph_fp64_peak: invalid argument");
  cudaSetDevice(ctx->device);
  const int blocks = ctx->sm_count * 4, threads = 256;
  PH_CUDA(ctx, ctx->ystage.ensure(sizeof(double) * blocks * threads));
  double *out = ctx->ystage.as<double>();
  cudaEvent_t e0, e1;
  PH_CUDA(ctx, cudaEventCreate(&e0));
  PH_CUDA(ctx, cudaEventCreate(&e1));
  int iters = 256;
  float ms = 0.f;
  for (int attempt = 0; attempt < 8; ++attempt) {
    k_dfma_peak<<<blocks, threads, 0, ctx->stream>>>(out, 16, 1.0000001, 1e-9);
    cudaEventRecord(e0, ctx->stream);
    k_dfma_peak<<<blocks, threads, 0, ctx->stream>>>(out, iters, 1.0000001, 1e-9);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return ph_cuda_fail(ctx, e, "ph_fp64_peak");
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms >= ms_target || iters >= (1 << 22)) break;
    double scale = ms > 0.01 ? ms_target / ms : 16.0;
    iters = (int)(iters * (scale > 16.0 ? 16.0 : scale) * 1.1) + 1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *gops = (double)blocks * threads * iters * 8.0 / (ms * 1e-3) / 1e9;
  return PH_OK;
}

// ---- the unit rates that shape the design ------------------------------------------

namespace {
// four independent FP64 tensor-core MMAs (m8n8k4, 256 FMAs each per warp) per iteration
__global__ void k_dmma_rate(double *out, int iters) {
  const double a = 1.0 + threadIdx.x * 1e-9, b = 1.0 - threadIdx.x * 1e-9;
  double c0[2] = {0, 0}, c1[2] = {0, 0}, c2[2] = {0, 0}, c3[2] = {0, 0};
  for (int i = 0; i < iters; ++i) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c0[0]), "+d"(c0[1]) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c1[0]), "+d"(c1[1]) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c2[0]), "+d"(c2[1]) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c3[0]), "+d"(c3[1]) : "d"(a), "d"(b));
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0[0] + c0[1] + c1[0] + c1[1] + c2[0] + c2[1] +
                                               c3[0] + c3[1];
}

// eight independent 32-bit integer multiply-adds per iteration
__global__ void k_imad_rate(double *out, int iters) {
  unsigned a = 3u + threadIdx.x, b = 7u ^ threadIdx.x;
  unsigned c[8] = {0, 1, 2, 3, 4, 5, 6, 7};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = c[q] * a + b;
  }
  unsigned s = 0;
  for (int q = 0; q < 8; ++q) s += c[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}
}  // namespace

extern "C" ph_status ph_unit_rates(ph_ctx *ctx, double *rates) {
  if (!ctx || !rates) return PH_EINVAL;
  cudaSetDevice(ctx->device);
  double dfma = 0.0;
  ph_status s = ph_fp64_peak(ctx, 20.0, &dfma);
  if (s != PH_OK) return s;
  const int blocks = ctx->sm_count * 4, threads = 128;
  PH_CUDA(ctx, ctx->ystage.ensure(sizeof(double) * blocks * 256));
  double *out = ctx->ystage.as<double>();
  cudaEvent_t e0, e1;
  PH_CUDA(ctx, cudaEventCreate(&e0));
  PH_CUDA(ctx, cudaEventCreate(&e1));
  float ms_mma = 0.f, ms_imad = 0.f;
  const int it_mma = 4096, it_imad = 8192;
  k_dmma_rate<<<blocks, threads, 0, ctx->stream>>>(out, 16);
  cudaEventRecord(e0, ctx->stream);
  k_dmma_rate<<<blocks, threads, 0, ctx->stream>>>(out, it_mma);
  cudaEventRecord(e1, ctx->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_mma, e0, e1);
  if (e == cudaSuccess) {
    k_imad_rate<<<blocks, 256, 0, ctx->stream>>>(out, 16);
    cudaEventRecord(e0, ctx->stream);
    k_imad_rate<<<blocks, 256, 0, ctx->stream>>>(out, it_imad);
    cudaEventRecord(e1, ctx->stream);
    e = cudaEventSynchronize(e1);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_imad, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return ph_cuda_fail(ctx, e, "ph_unit_rates");
  rates[0] = dfma;
  rates[1] = (double)blocks * (threads / 32) * it_mma * 4 * 256 / (ms_mma * 1e-3) / 1e9;
  rates[2] = (double)blocks * 256 * it_imad * 8 / (ms_imad * 1e-3) / 1e9;
  return PH_OK;
}
