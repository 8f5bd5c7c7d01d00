// batch.cu -- ph_track_paths: many solution paths of one homotopy at once.
//
// The paper accelerates the tracking of a single path (Introduction; the
// many-path case is its companion work).  A single path of a few dozen
// variables cannot fill a GB300: its predictor-corrector step is a chain of
// dependent FP64 operations (~64 cycles each on this GPU).  Here one persistent
// kernel tracks many paths, one block per path: a block takes the next
// unstarted path from a counter, tracks it to its end entirely with its own
// threads (predictor, evaluation, MGS, back substitution, update, step
// control, all separated by __syncthreads only), stores the end point and takes
// the next path.  Blocks never wait for one another, paths of uneven length
// balance themselves, and with two blocks per SM every FP64 unit has work.
//
// The step follows the same definitions as the single-path kernels (the same
// controller code, the same Newton tests, the same reverse-mode evaluation);
// the MGS inside a block is the unnormalised right-looking form with one warp
// per column in turn (columns dealt round-robin to the 8 warps), the pivot
// norms kept in shared memory, and a block barrier per column step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctrl.h"
#include "internal.h"
#include "mp.cuh"
#include "pathdev.cuh"

using namespace ph;

long ph_lda(int N);

namespace {

constexpr int BT = 256;           // threads per block: 8 warps, 2 per SM sub-partition
constexpr int NW = BT / 32;
constexpr int kHist = 16;         // accepted points kept for the predictor
constexpr int SG = 4;             // lanes per output in the summation

struct BatchArgs {
  // target system f (and start system g, optional)
  int N, n, Mf, Mpf, maxvf, Mg, Mpg, maxvg, emax, nout;
  const int32_t *nvf, *vidxf, *vexpf, *optrf, *oslotf, *deg;
  const double *coeff_f;
  const int32_t *nvg, *vidxg, *vexpg, *optrg, *oslotg;
  const double *coeff_g;
  const double *gamma;            // [2L]
  ph_track_params p;
  int npaths;
  const double *x0;               // [npaths][2L][n]
  double *x_out;                  // [npaths][2L][n]
  ph_path_stats *stats;           // [npaths]
  ph_step_record *log;            // [npaths][log_cap] or null
  int log_cap;
  unsigned int *next;             // work queue counter
  // per-block workspace (doubles)
  double *ws;
  long ws_stride, o_x, o_dx, o_hist, o_ptab, o_spow, o_A, o_W, o_fslots, o_gslots, o_scal, o_t;
  long ldA, nsf, nsg;
};

// one part (0 = real, 1 = imaginary) of element i of a complex array laid out
// [limb][re|im][...] with `plane` doubles between planes
template <class P>
PHD typename P::real rp_load(const double *v, long plane, int part, long i) {
  return r_load<P>(v + part * plane, 2 * plane, i);
}
template <class P>
PHD void rp_store(double *v, long plane, int part, long i, const typename P::real &z) {
  r_store<P>(v + part * plane, 2 * plane, i, z);
}

template <class P>
__device__ typename P::real warp_sum_part(typename Part<P>::acc a) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) a = Part<P>::combine(a, Part<P>::shfl(a, m));
  return Part<P>::value(a);
}

// MGS of [J | -h] (A, in this block's workspace) and back substitution.
// Returns the status (PH_OK or PH_NONFINITE); dx and max |dx_i| on success.
template <class P>
__device__ int block_mgs(const BatchArgs &a, double *A, double *W, double *dx, double *s_nrm,
                         double *s_y, double *s_dxmax) {
  typedef typename P::real real;
  typedef Part<P> PO;
  __shared__ int s_bad;
  const int N = a.N, n = a.n, nc = n + 1;
  const long ldA = a.ldA, Ap = (long)nc * ldA, Wp = (long)nc * nc;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  if (tid == 0) s_bad = 0;
  if (w == 0) {                                    // ||a_0||^2
    typename PO::acc ar = PO::zero(), ai = PO::zero();
    for (int i = lane; i < N; i += 32) {
      PO::sq(ar, rp_load<P>(A, Ap, 0, i));
      PO::sq(ai, rp_load<P>(A, Ap, 1, i));
    }
    real s = P::add(warp_sum_part<P>(ar), warp_sum_part<P>(ai));
    if (lane == 0) r_store<P>(s_nrm, nc, 0, s);
  }
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    const real r2 = r_load<P>(s_nrm, nc, k);
    const double lead = P::lead(r2);
    if (!(lead > 0.0) || !isfinite(lead)) {        // the same value in every thread
      if (tid == 0) s_bad = 1;
      break;
    }
    const real inv2 = P::recip(r2);
    const double *ak = A + (long)k * ldA;
    for (int j = k + 1 + (((w - (k + 1)) % NW) + NW) % NW; j <= n; j += NW) {
      double *aj = A + (long)j * ldA;
      typename PO::acc dr = PO::zero(), di = PO::zero();
      for (int i = lane; i < N; i += 32) {
        real akr = rp_load<P>(ak, Ap, 0, i), aki = rp_load<P>(ak, Ap, 1, i);
        real ajr = rp_load<P>(aj, Ap, 0, i), aji = rp_load<P>(aj, Ap, 1, i);
        PO::dot2(dr, akr, ajr, aki, aji, 1.0);
        PO::dot2(di, akr, aji, aki, ajr, -1.0);
      }
      const real alr = P::mul(warp_sum_part<P>(dr), inv2);
      const real ali = P::mul(warp_sum_part<P>(di), inv2);
      if (lane == 0) {
        rp_store<P>(W + (long)j * nc, Wp, 0, k, alr);
        rp_store<P>(W + (long)j * nc, Wp, 1, k, ali);
      }
      typename PO::acc nr = PO::zero(), ni = PO::zero();
      for (int i = lane; i < N; i += 32) {
        real akr = rp_load<P>(ak, Ap, 0, i), aki = rp_load<P>(ak, Ap, 1, i);
        real ajr = PO::upd(rp_load<P>(aj, Ap, 0, i), alr, akr, ali, aki, 1.0);
        real aji = PO::upd(rp_load<P>(aj, Ap, 1, i), alr, aki, ali, akr, -1.0);
        rp_store<P>(aj, Ap, 0, i, ajr);
        rp_store<P>(aj, Ap, 1, i, aji);
        if (j == k + 1) {
          PO::sq(nr, ajr);
          PO::sq(ni, aji);
        }
      }
      if (j == k + 1) {
        real s = P::add(warp_sum_part<P>(nr), warp_sum_part<P>(ni));
        if (lane == 0) r_store<P>(s_nrm, nc, j, s);
      }
    }
  }
  __syncthreads();
  if (s_bad) return PH_NONFINITE;
  // back substitution on y = alpha_{., n} by warp 0: dx_k = y_k, y_i -= alpha_ik dx_k
  if (w == 0) {
    const double *yc = W + (long)n * nc;
    for (int i = lane; i < n; i += 32) c_store<P>(s_y, n, i, c_load<P>(yc, Wp, i));
    __syncwarp();
    for (int k = n - 1; k >= 1; --k) {
      const real xr = rp_load<P>(s_y, n, 0, k), xi = rp_load<P>(s_y, n, 1, k);
      const double *Wk = W + (long)k * nc;
      for (int i = lane; i < k; i += 32) {
        real wr = rp_load<P>(Wk, Wp, 0, i), wi = rp_load<P>(Wk, Wp, 1, i);
        rp_store<P>(s_y, n, 0, i, PO::upd(rp_load<P>(s_y, n, 0, i), wr, xr, wi, xi, 1.0));
        rp_store<P>(s_y, n, 1, i, PO::upd(rp_load<P>(s_y, n, 1, i), wr, xi, wi, xr, -1.0));
      }
      __syncwarp();
    }
    double m = 0.0;
    for (int i = lane; i < n; i += 32) {
      cx<P> v = c_load<P>(s_y, n, i);
      c_store<P>(dx, n, i, v);
      double mg = c_mag_lead<P>(v);
      if (!(mg <= m)) m = mg;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_xor_sync(0xffffffffu, m, off);
      if (!(o <= m)) m = o;
    }
    if (lane == 0) *s_dxmax = m;
  }
  __syncthreads();
  return PH_OK;
}

template <class P>
__global__ void __launch_bounds__(BT) k_paths(BatchArgs a) {
  typedef typename P::real real;
  extern __shared__ double smem[];
  double *s_y = smem;                                   // [2L][n]
  double *s_nrm = smem + 2 * P::L * a.n;                // [L][n+1]
  __shared__ ph_ctrl_state s_ctrl;
  __shared__ real s_w[kHist];
  __shared__ double s_t[kHist];
  __shared__ int s_path, s_head, s_count, s_dec, s_ok, s_upd, s_iters, s_bad;
  __shared__ double s_tn, s_last, s_res, s_dxn, s_dxmax, s_xmax;
  __shared__ unsigned long long s_resbits;
  __shared__ ph_path_stats s_st;

  const int n = a.n, N = a.N, tid = threadIdx.x;
  const long pt = 2L * P::L * n;
  double *ws = a.ws + (long)blockIdx.x * a.ws_stride;
  double *x = ws + a.o_x, *dx = ws + a.o_dx, *hist = ws + a.o_hist, *ptab = ws + a.o_ptab;
  double *spow = ws + a.o_spow, *A = ws + a.o_A, *W = ws + a.o_W, *fslots = ws + a.o_fslots;
  double *gslots = ws + a.o_gslots, *scal = ws + a.o_scal, *tl = ws + a.o_t;
  const bool fixed = a.p.fixed_steps > 0;
  const long Ap = (long)(n + 1) * a.ldA;
  const bool total_degree = a.optrg == nullptr;

  for (;;) {
    if (tid == 0) s_path = (int)atomicAdd(a.next, 1u);
    __syncthreads();
    const int path = s_path;
    if (path >= a.npaths) return;
    // start: the start point is the only accepted point
    const double *x0 = a.x0 + (long)path * pt;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (long e = tid; e < pt; e += BT) {
      double v = x0[e];
      hist[e] = v;
      if (!isfinite(v)) s_bad = 1;
    }
    if (tid == 0) {
      ctrl_init(&s_ctrl, &a.p);
      memset(&s_st, 0, sizeof s_st);
      s_head = 0;
      s_count = 1;
      s_t[0] = 0.0;
    }
    __syncthreads();
    if (s_bad) {
      for (long e = tid; e < pt; e += BT) a.x_out[(long)path * pt + e] = x0[e];
      if (tid == 0 && a.stats) {
        s_st.status = PH_NONFINITE;
        a.stats[path] = s_st;
      }
      __syncthreads();
      continue;
    }
    for (;;) {
      if (tid == 0) s_tn = ctrl_next_t(&s_ctrl, &a.p);
      __syncthreads();
      const double tn = s_tn;
      if (tn < 0.0) break;
      // predictor: Lagrange weights of the last m accepted points at tn
      const int m = s_count < a.p.pred_order + 1 ? s_count : a.p.pred_order + 1;
      if (tid < m) {
        const int sj = (s_head - (m - 1 - tid) + kHist) % kHist;
        const double tj = s_t[sj];
        real num = P::from(1.0), den = P::from(1.0);
        for (int l = 0; l < m; ++l) {
          if (l == tid) continue;
          const double tq = s_t[(s_head - (m - 1 - l) + kHist) % kHist];
          double s1, e1;
          real u = P::zero(), v = P::zero();
          two_sum(tn, -tq, s1, e1);
          P::set_limb(u, 0, s1);
          P::set_limb(u, 1, e1);
          two_sum(tj, -tq, s1, e1);
          P::set_limb(v, 0, s1);
          P::set_limb(v, 1, e1);
          num = P::mul(num, u);
          den = P::mul(den, v);
        }
        s_w[tid] = m == 1 ? P::from(1.0) : P::div(num, den);
      }
      if (tid == 0) {
        tl[0] = tn;
        for (int l = 1; l < P::L; ++l) tl[l] = 0.0;
        s_last = a.p.max_res;
        s_dec = 0;
        s_ok = fixed ? 1 : 0;
        s_upd = 0;
        s_iters = 0;
      }
      __syncthreads();
      for (int i = tid; i < n; i += BT) {
        cx<P> acc = c_zero<P>();
        for (int j = 0; j < m; ++j) {
          const int sj = (s_head - (m - 1 - j) + kHist) % kHist;
          acc = c_add<P>(acc, c_mul_real<P>(c_load<P>(hist + sj * pt, n, i), s_w[j]));
        }
        c_store<P>(x, n, i, acc);
      }
      // corrector
      for (int it = 0; it < a.p.max_newton; ++it) {
        __syncthreads();
        for (int j = tid; j < n; j += BT)
          prep_variable<P>(j, x, n, a.emax, ptab, a.deg, total_degree ? spow : nullptr);
        if (tid == 0) {
          prep_factors<P>(tl, a.gamma, a.p.relax_k, scal);
          s_resbits = 0ull;
        }
        __syncthreads();
        for (int s = tid; s < a.Mf; s += BT)
          ad_term<P>(s, a.Mpf, a.nvf, a.vidxf, a.vexpf, a.coeff_f, ptab, n, a.maxvf, fslots, a.nsf);
        for (int s = tid; s < a.Mg; s += BT)
          ad_term<P>(s, a.Mpg, a.nvg, a.vidxg, a.vexpg, a.coeff_g, ptab, n, a.maxvg, gslots, a.nsg);
        __syncthreads();
        double mymax = 0.0;
        for (int o0 = 0; o0 < a.nout; o0 += BT / SG) {
          const int o = o0 + tid / SG, lane = tid % SG;
          const bool act = o < a.nout;
          cx<P> val = sum_output<P, SG>(act, o, lane, N, n, a.optrf, a.oslotf, fslots, a.nsf,
                                        a.optrg, a.oslotg, gslots, a.nsg, spow, scal, 1);
          if (act && lane == 0) {
            if (o < n * N) {
              const int j = o / N, i = o - j * N;
              c_store<P>(A + (long)j * a.ldA, Ap, i, val);
            } else {
              const int i = o - n * N;
              c_store<P>(A + (long)n * a.ldA, Ap, i, c_neg<P>(val));
              double mg = c_mag_lead<P>(val);
              if (!(mg <= mymax)) mymax = mg;
            }
          }
        }
        atomicMax(&s_resbits, (unsigned long long)__double_as_longlong(mymax));
        __syncthreads();
        if (tid == 0) {                            // residual test (Fig. "An accelerated Newton's method")
          const double r = __longlong_as_double((long long)s_resbits);
          s_res = r;
          s_iters += 1;
          s_st.newton_iters += 1;
          s_st.res = r;
          if (!fixed) {
            if (!(r <= s_last) || !isfinite(r)) { s_dec = 1; s_ok = 0; }
            else if (r < a.p.tol_res) { s_dec = 1; s_ok = 1; }
          }
        }
        __syncthreads();
        if (s_dec) break;
        const int ms = block_mgs<P>(a, A, W, dx, s_nrm, s_y, &s_dxmax);
        if (ms != PH_OK && !fixed) {
          if (tid == 0) { s_dec = 1; s_ok = 0; }
          __syncthreads();
          break;
        }
        for (int i = tid; i < n; i += BT) {
          cx<P> d = ms != PH_OK ? c_from<P>(NAN, NAN) : c_load<P>(dx, n, i);
          c_store<P>(x, n, i, c_add<P>(c_load<P>(x, n, i), d));
        }
        if (tid == 0) {                            // update test
          const double d = ms != PH_OK ? NAN : s_dxmax;
          s_dxn = d;
          s_st.dx = d;
          s_upd += 1;
          s_st.updates += 1;
          if (!fixed) {
            if (!isfinite(d)) { s_dec = 1; s_ok = 0; }
            else if (d < a.p.tol_dx) { s_dec = 1; s_ok = 1; }
            else s_last = s_res;
          }
          if (!s_dec && s_iters >= a.p.max_newton) { s_dec = 1; s_ok = fixed ? 1 : 0; }
        }
        __syncthreads();
        if (s_dec) break;
      }
      __syncthreads();
      // step control (Fig. "Accelerated tracking of one single path")
      if (tid == 0) {
        const int ok = s_ok;
        s_st.steps += 1;
        if (ok) s_st.accepted += 1; else s_st.rejected += 1;
        if (a.log && s_st.steps <= a.log_cap) {
          ph_step_record r;
          r.t = tn;
          r.res = s_res;
          r.dx = s_dxn;
          r.accepted = ok;
          r.updates = s_upd;
          a.log[(long)path * a.log_cap + s_st.steps - 1] = r;
        }
        ctrl_report(&s_ctrl, &a.p, tn, ok);
        if (ok) {
          s_head = (s_head + 1) % kHist;
          s_t[s_head] = tn;
          s_count = s_count < kHist ? s_count + 1 : kHist;
        }
        s_xmax = 0.0;
      }
      __syncthreads();
      if (s_ok) {
        double mymax = 0.0;
        for (int i = tid; i < n; i += BT) {
          cx<P> xi = c_load<P>(x, n, i);
          c_store<P>(hist + s_head * pt, n, i, xi);
          double mg = c_mag_lead<P>(xi);
          if (!(mg <= mymax)) mymax = mg;
        }
        atomicMax((unsigned long long *)&s_xmax, (unsigned long long)__double_as_longlong(mymax));
        __syncthreads();
        if (tid == 0 && !fixed && !s_ctrl.done && !(s_xmax <= a.p.max_x)) {
          s_ctrl.done = 1;
          s_ctrl.status = PH_DIVERGED;
        }
      }
      __syncthreads();
      if (s_ctrl.done) break;
    }
    // end point: the last accepted point
    for (long e = tid; e < pt; e += BT) a.x_out[(long)path * pt + e] = hist[(long)s_head * pt + e];
    if (tid == 0 && a.stats) {
      s_st.status = s_ctrl.status;
      s_st.t_final = s_t[s_head];
      s_st.launches = 0;
      a.stats[path] = s_st;
    }
    __syncthreads();
  }
}

template <class P>
cudaError_t launch_paths(const BatchArgs &args, int grid, size_t smem, cudaStream_t st) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_paths<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_paths<P><<<grid, BT, smem, st>>>(args);
  return cudaGetLastError();
}

template <class P>
int blocks_per_sm(size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_paths<P>, BT, smem) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < 1 ? 1 : (nb > 2 ? 2 : nb);
}

}  // namespace

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
      p.relax_k < 1 || p.relax_k > 64 || p.max_steps < 0 ||
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
  const int L = f->L, n = f->n, N = f->N, nc = n + 1;
  const long pt = 2L * L * n, ldA = ph_lda(N);
  const int emax = std::max(f->emax, g ? g->emax : 1);
  const long ntab = emax > 2 ? emax - 1 : 1;
  const long nsf = (long)(f->maxv + 1) * f->Mp, nsg = g ? (long)(g->maxv + 1) * g->Mp : 0;
  auto up = [](long v) { return (v + 31) / 32 * 32; };      // 256-byte aligned regions
  BatchArgs a;
  memset(&a, 0, sizeof a);
  a.o_x = 0;
  a.o_dx = a.o_x + up(pt);
  a.o_hist = a.o_dx + up(pt);
  a.o_ptab = a.o_hist + up(pt * kHist);
  a.o_spow = a.o_ptab + up(pt * ntab);
  a.o_A = a.o_spow + up(2 * pt);
  a.o_W = a.o_A + up(2L * L * nc * ldA);
  a.o_fslots = a.o_W + up(2L * L * nc * nc);
  a.o_gslots = a.o_fslots + up(2L * L * nsf);
  a.o_scal = a.o_gslots + up(2L * L * nsg);
  a.o_t = a.o_scal + up(3L * L);
  a.ws_stride = a.o_t + up(L);
  const size_t smem = sizeof(double) * (2L * L * n + (long)L * nc);
  const int bps = L == 2 ? blocks_per_sm<DD>(smem) : blocks_per_sm<QD>(smem);
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

  a.N = N; a.n = n; a.emax = emax; a.nout = f->nout;
  a.Mf = f->M; a.Mpf = f->Mp; a.maxvf = f->maxv;
  a.nvf = f->nv.as<int32_t>(); a.vidxf = f->vidx.as<int32_t>(); a.vexpf = f->vexp.as<int32_t>();
  a.optrf = f->out_ptr.as<int32_t>(); a.oslotf = f->out_slot.as<int32_t>();
  a.coeff_f = f->coeff.as<double>(); a.deg = f->deg.as<int32_t>();
  if (g) {
    a.Mg = g->M; a.Mpg = g->Mp; a.maxvg = g->maxv;
    a.nvg = g->nv.as<int32_t>(); a.vidxg = g->vidx.as<int32_t>(); a.vexpg = g->vexp.as<int32_t>();
    a.optrg = g->out_ptr.as<int32_t>(); a.oslotg = g->out_slot.as<int32_t>();
    a.coeff_g = g->coeff.as<double>();
  }
  a.gamma = ctx->in_gamma.as<double>();
  a.p = p;
  a.npaths = npaths;
  a.x0 = dx0;
  a.x_out = dxo;
  a.stats = ctx->bstats.as<ph_path_stats>();
  a.log = dlog;
  a.log_cap = log_cap;
  a.next = ctx->bq.as<unsigned int>();
  a.ws = ctx->bws.as<double>();
  a.ldA = ldA;
  a.nsf = nsf;
  a.nsg = nsg;
  PH_CUDA(ctx, L == 2 ? launch_paths<DD>(a, grid, smem, ctx->stream)
                      : launch_paths<QD>(a, grid, smem, ctx->stream));
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
