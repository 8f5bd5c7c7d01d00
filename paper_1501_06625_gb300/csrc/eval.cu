// eval.cu -- values and Jacobian of h(x,t) = gamma (1-t)^k g(x) + t^k f(x)
// (Section 2, Eq. (1)) by reverse-mode differentiation of every monomial
// (Section 3.2) and segmented summation (Section 3.3).
//
// Three kernels per evaluation:
//  k_prep  power table x_j^e (e < largest exponent) and the homotopy factors
//          t^k and gamma (1-t)^k;
//  k_ad    one thread (or T lanes, k_ad_split) per monomial c x^a with v distinct variables: the common
//          factor CF = prod x_j^{a_j - 1} from the power table is folded into
//          the coefficient, then the Speelpenning product of the v variables is
//          differentiated in the reverse mode (forward prefix products, backward
//          suffix and cross products, Section 3.2, Table 1):
//            d/dx_j (c x^a) = a_j * (c CF x_1..x_{j-1}) * (x_{j+1}..x_v).
//          Monomials are sorted by v so a warp runs monomials of equal length,
//          and the instructions are stored position-major so lanes read
//          consecutive addresses (Section 3.2).  Results go to "slots".
//  k_sum   G lanes per output (the paper's #Th, Section 3.3) add the output's
//          slots in a fixed order (no atomics: the result is deterministic),
//          scale by the homotopy factors, add the start system and write J, h,
//          -h (the right-hand side of the Newton system) and max |h_i|.
#include "internal.h"
#include "mp.cuh"
#include "pathdev.cuh"

using namespace ph;

namespace {

template <class P>
__global__ void k_prep(const double *__restrict__ x, int n, int emax, double *__restrict__ ptab,
                       const int32_t *__restrict__ deg, double *__restrict__ spow,
                       const double *__restrict__ t, const double *__restrict__ gamma, int k,
                       double *__restrict__ scal, const int *__restrict__ skip) {
  if (skip && *skip) return;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) prep_variable<P>(j, x, n, emax, ptab, deg, spow);
  if (gamma && blockIdx.x == 0 && threadIdx.x == 0) prep_factors<P>(t, gamma, k, scal);
}

template <class P>
__global__ void __launch_bounds__(128) k_ad(int M, int Mp, const int32_t *__restrict__ nv,
                                            const int32_t *__restrict__ vidx,
                                            const int32_t *__restrict__ vexp,
                                            const double *__restrict__ coeff,
                                            const double *__restrict__ ptab, int n, int maxv,
                                            double *__restrict__ slots, long nslots,
                                            const int *__restrict__ skip, int s0) {
  if (skip && *skip) return;
  int s = s0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  ad_term<P>(s, Mp, nv, vidx, vexp, coeff, ptab, n, maxv, slots, nslots);
}

// The value c x^a of term s alone (no derivatives): the residual of the
// precision form, where the Jacobian is evaluated in a lower precision.
template <class P>
__global__ void __launch_bounds__(128) k_val(int M, int Mp, const int32_t *__restrict__ nv,
                                             const int32_t *__restrict__ vidx,
                                             const int32_t *__restrict__ vexp,
                                             const double *__restrict__ coeff,
                                             const double *__restrict__ ptab, int n, int emax,
                                             int maxv, double *__restrict__ slots, long nslots,
                                             const int *__restrict__ skip) {
  if (skip && *skip) return;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  val_term<P>(s, Mp, nv, vidx, vexp, coeff, ptab, n, emax, maxv, slots, nslots);
}

template <class P>
PHD cx<P> shfl_up_c(const cx<P> &a, int d, int width) {
  cx<P> z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) {
    P::set_limb(z.re, l, __shfl_up_sync(0xffffffffu, P::limb(a.re, l), d, width));
    P::set_limb(z.im, l, __shfl_up_sync(0xffffffffu, P::limb(a.im, l), d, width));
  }
  return z;
}

// T lanes per monomial (T = 2, 4, 8): lane q owns a chunk of c = ceil(v/T)
// consecutive variable positions.  Each lane forms its chunk's factor
// B_q = (c if q = 0) * CF_q * prod_{own} x_j, where CF_q collects the common
// factor x_j^{a_j - 1} of its own positions; shuffle scans give the products
// of the other chunks' factors to the left and right, and the lane finishes
// its positions with a local reverse sweep:
//   d/dx_j = a_j * (left * right * CF_q) * prod_{own l != j} x_l.
// The critical path drops from ~3v to ~3v/T + 2 log2(T) + 2 complex products.
template <class P, int T>
__global__ void __launch_bounds__(128) k_ad_split(int s0, int s1, int Mp,
                                                  const int32_t *__restrict__ nv,
                                                  const int32_t *__restrict__ vidx,
                                                  const int32_t *__restrict__ vexp,
                                                  const double *__restrict__ coeff,
                                                  const double *__restrict__ ptab, int n, int maxv,
                                                  double *__restrict__ slots, long nslots,
                                                  const int *__restrict__ skip) {
  if (skip && *skip) return;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = s0 + (int)(gt / T);
  const int q = (int)(gt % T);
  const bool active = s < s1;                    // every lane still joins the shuffles
  const long pl = 2L * P::L * n;
  const int v = active ? nv[s] : 0;
  const int c = (v + T - 1) / T;
  const int p0 = q * c < v ? q * c : v;
  const int p1 = p0 + c < v ? p0 + c : v;
  const cx<P> one = c_from<P>(1.0, 0.0);
  // the chunk's common factor and full factor
  cx<P> cf = one;
  bool has_cf = false;
  for (int p = p0; p < p1; ++p) {
    int a = vexp[(long)p * Mp + s];
    if (a >= 2) {
      cx<P> w = c_load<P>(ptab + (a - 2) * pl, n, vidx[(long)p * Mp + s]);
      cf = has_cf ? c_mul_ad<P>(cf, w) : w;
      has_cf = true;
    }
  }
  const cx<P> c0 = (active && q == 0) ? c_load<P>(coeff, Mp, s) : one;
  cx<P> B = c0;
  bool b_one = !(active && q == 0);
  if (has_cf) { B = b_one ? cf : c_mul_ad<P>(B, cf); b_one = false; }
  for (int p = p0; p < p1; ++p) {
    cx<P> xj = c_load<P>(ptab, n, vidx[(long)p * Mp + s]);
    B = b_one ? xj : c_mul_ad<P>(B, xj);
    b_one = false;
  }
  // inclusive prefix and suffix products over the T lanes of this monomial
  cx<P> I = B, S = B;
#pragma unroll
  for (int d = 1; d < T; d <<= 1) {
    cx<P> y = shfl_up_c<P>(I, d, T);
    if (q >= d) I = c_mul_ad<P>(y, I);
    cx<P> z = shfl_down_c<P>(S, d, T);
    if (q + d < T) S = c_mul_ad<P>(S, z);
  }
  cx<P> left = shfl_up_c<P>(I, 1, T);
  cx<P> right = shfl_down_c<P>(S, 1, T);
  if (!active) return;
  if (q == T - 1) c_store<P>(slots, nslots, (long)maxv * Mp + s, I);   // the value
  if (p0 == p1) return;
  // outer factor of this chunk (lane 0 carries the coefficient itself)
  cx<P> outer;
  bool o_one = true;
  if (q > 0) { outer = left; o_one = false; }
  else { outer = c0; o_one = false; }
  if (q < T - 1) { outer = o_one ? right : c_mul_ad<P>(outer, right); o_one = false; }
  if (has_cf) { outer = o_one ? cf : c_mul_ad<P>(outer, cf); o_one = false; }
  if (o_one) outer = one;
  // local reverse sweep over the chunk (prefixes parked in the slots)
  cx<P> pre = outer;
  for (int p = p0; p < p1; ++p) {
    c_store<P>(slots, nslots, (long)p * Mp + s, pre);
    if (p + 1 < p1) pre = c_mul_ad<P>(pre, c_load<P>(ptab, n, vidx[(long)p * Mp + s]));
  }
  cx<P> suf = one;
  for (int p = p1 - 1; p >= p0; --p) {
    cx<P> d = c_load<P>(slots, nslots, (long)p * Mp + s);
    if (p < p1 - 1) d = c_mul_ad<P>(d, suf);
    d = c_mul_int<P>(d, vexp[(long)p * Mp + s]);
    c_store<P>(slots, nslots, (long)p * Mp + s, d);
    if (p > p0) {
      cx<P> xj = c_load<P>(ptab, n, vidx[(long)p * Mp + s]);
      suf = (p == p1 - 1) ? xj : c_mul_ad<P>(suf, xj);
    }
  }
}

template <class P, int G>
__global__ void __launch_bounds__(256) k_sum(
    int N, int n, int nout, const int32_t *__restrict__ optr, const int32_t *__restrict__ oslot,
    const double *__restrict__ slots, long nslots, const int32_t *__restrict__ goptr,
    const int32_t *__restrict__ goslot, const double *__restrict__ gslots, long gnslots,
    const double *__restrict__ spow, const double *__restrict__ scal, int homotopy,
    double *__restrict__ J, long ldJ, long Jplane, double *__restrict__ h,
    double *__restrict__ rhs, long rhs_plane, unsigned long long *__restrict__ res_bits,
    const int *__restrict__ skip, int o0, int lead_rhs, const uint8_t *__restrict__ fixed) {
  if (skip && *skip) return;
  long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int o = o0 + (int)(gt / G);
  int lane = (int)(gt % G);
  bool active = o < nout;
  cx<P> val = sum_output<P, G>(active, o, lane, N, n, optr, oslot, slots, nslots, goptr, goslot,
                               gslots, gnslots, spow, scal, homotopy, fixed);
  if (!active || lane != 0) return;
  const int nN = n * N;
  if (o < nN) {
    int j = o / N, i = o - j * N;
    c_store<P>(J + (long)j * ldJ, Jplane, i, val);
  } else {
    int i = o - nN;
    if (h) c_store<P>(h, N, i, val);
    if (rhs && lead_rhs) {                     // the leading limbs of -h, [re|im]
      rhs[i] = -P::lead(val.re);
      rhs[rhs_plane + i] = -P::lead(val.im);
    } else if (rhs) {
      c_store<P>(rhs, rhs_plane, i, c_neg<P>(val));
    }
    if (res_bits) atomicMax(res_bits, (unsigned long long)__double_as_longlong(c_mag_lead<P>(val)));
  }
}

// One launch per bucket of monomials sharing a lane count (the buckets are
// contiguous because the terms are sorted by their number of variables).
template <class P>
void ad_launch(const ph_system *sy, const double *ptab, int n, double *slots, long ns,
               const int *skip, cudaStream_t st) {
  for (const ph_system::Bucket &b : sy->buckets) {
    const long threads = (long)(b.s1 - b.s0) * b.lanes;
    const unsigned grid = (unsigned)((threads + 127) / 128);
    const int32_t *nv = sy->nv.as<int32_t>(), *vi = sy->vidx.as<int32_t>(), *ve = sy->vexp.as<int32_t>();
    const double *co = sy->coeff.as<double>();
    switch (b.lanes) {
      case 1:
        k_ad<P><<<grid, 128, 0, st>>>(b.s1, sy->Mp, nv, vi, ve, co, ptab, n, sy->maxv, slots, ns, skip, b.s0);
        break;
      case 2:
        k_ad_split<P, 2><<<grid, 128, 0, st>>>(b.s0, b.s1, sy->Mp, nv, vi, ve, co, ptab, n, sy->maxv, slots, ns, skip);
        break;
      case 4:
        k_ad_split<P, 4><<<grid, 128, 0, st>>>(b.s0, b.s1, sy->Mp, nv, vi, ve, co, ptab, n, sy->maxv, slots, ns, skip);
        break;
      default:
        k_ad_split<P, 8><<<grid, 128, 0, st>>>(b.s0, b.s1, sy->Mp, nv, vi, ve, co, ptab, n, sy->maxv, slots, ns, skip);
        break;
    }
  }
}

// the summation kernel with G lanes per output
template <class P, int G>
void sum_launch_g(const ph_system *f, const ph_system *g, int N, int n, const double *fslots,
                  long fs, const double *gslots, long gs, const double *spow, const double *scal,
                  int homotopy, double *J, long ldJ, long Jplane, double *h, double *rhs,
                  long rhs_plane, unsigned long long *res_bits, const int *skip, cudaStream_t st,
                  int o0, int lead_rhs, const uint8_t *fixed) {
  const long threads = (long)(f->nout - o0) * G;
  k_sum<P, G><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      N, n, f->nout, f->out_ptr.as<int32_t>(), f->out_slot.as<int32_t>(), fslots, fs,
      g ? g->out_ptr.as<int32_t>() : nullptr, g ? g->out_slot.as<int32_t>() : nullptr, gslots, gs,
      spow, scal, homotopy, J, ldJ, Jplane, h, rhs, rhs_plane, res_bits, skip, o0, lead_rhs, fixed);
}

constexpr int kSumLanes[6] = {1, 2, 4, 8, 16, 32};

template <class P>
void sum_launch(int G, const ph_system *f, const ph_system *g, int N, int n, const double *fslots,
                long fs, const double *gslots, long gs, const double *spow, const double *scal,
                int homotopy, double *J, long ldJ, long Jplane, double *h, double *rhs,
                long rhs_plane, unsigned long long *res_bits, const int *skip, cudaStream_t st,
                int o0 = 0, int lead_rhs = 0, const uint8_t *fixed = nullptr) {
#define PH_SUM_CASE(g_)                                                                          \
  case g_:                                                                                       \
    sum_launch_g<P, g_>(f, g, N, n, fslots, fs, gslots, gs, spow, scal, homotopy, J, ldJ,        \
                        Jplane, h, rhs, rhs_plane, res_bits, skip, st, o0, lead_rhs, fixed);      \
    break;
  switch (G) {
    PH_SUM_CASE(1)
    PH_SUM_CASE(2)
    PH_SUM_CASE(4)
    PH_SUM_CASE(16)
    PH_SUM_CASE(32)
    default:
      sum_launch_g<P, 8>(f, g, N, n, fslots, fs, gslots, gs, spow, scal, homotopy, J, ldJ, Jplane,
                         h, rhs, rhs_plane, res_bits, skip, st, o0, lead_rhs, fixed);
  }
#undef PH_SUM_CASE
}

// Times the summation with each lane count on the context's buffers (their
// contents do not matter for the time; the outputs go to a scratch matrix) and
// keeps the fastest on f.  Nothing is measured during a stream capture.
template <class P>
void tune_sum(ph_ctx *ctx, const ph_system *f, const ph_system *g) {
  if (f->sum_lanes > 0) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  const int L = P::L, n = f->n, N = f->N;
  const long fs = (long)(f->maxv + 1) * f->Mp;
  const long gs = g ? (long)(g->maxv + 1) * g->Mp : 0;
  cudaError_t e = ctx->slots.ensure(sizeof(double) * 2 * L * (size_t)(fs + gs + 1));
  if (e == cudaSuccess) e = ctx->spow.ensure(sizeof(double) * 4 * L * (size_t)n);
  if (e == cudaSuccess) e = ctx->scal.ensure(sizeof(double) * 3 * L);
  const long ldJ = N, Jplane = (long)n * N;
  if (e == cudaSuccess) e = ctx->tuneA.ensure(sizeof(double) * 2 * L * (size_t)Jplane);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double *fslots = ctx->slots.as<double>(), *gslots = fslots + 2 * L * fs;
  float best = 1e30f;
  int choice = 8;
  for (int v = 0; v < 6 && e == cudaSuccess; ++v) {
    float tmin = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {     // rep 0 warms up
      e = cudaEventRecord(e0, ctx->stream);
      sum_launch<P>(kSumLanes[v], f, g, N, n, fslots, fs, gslots, gs, ctx->spow.as<double>(),
                    ctx->scal.as<double>(), 1, ctx->tuneA.as<double>(), ldJ, Jplane, nullptr,
                    nullptr, 0, nullptr, nullptr, ctx->stream);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && rep > 0 && ms < tmin) tmin = ms;
    }
    if (e == cudaSuccess) {
      f->sum_ms[v] = tmin;
      if (tmin < best) {
        best = tmin;
        choice = kSumLanes[v];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  f->sum_lanes = e == cudaSuccess ? choice : 8;
}

template <class P>
cudaError_t eval_impl(ph_ctx *ctx, const ph_system *f, const ph_system *g, const double *gamma,
                      int k, const double *t, const double *x, double *h, double *J, long ldJ,
                      long Jplane, double *rhs, long rhs_plane, const int *skip,
                      unsigned long long *res_bits, int parts, const uint8_t *fixed) {
  const int L = P::L, n = f->n, N = f->N;
  int emax = f->emax;
  if (g && g->emax > emax) emax = g->emax;
  const int ntab = emax > 2 ? emax - 1 : 1;
  cudaError_t e;
  if ((e = ctx->ptab.ensure(sizeof(double) * 2 * L * (size_t)n * ntab)) != cudaSuccess) return e;
  if ((e = ctx->scal.ensure(sizeof(double) * 3 * L)) != cudaSuccess) return e;
  if ((e = ctx->spow.ensure(sizeof(double) * 4 * L * (size_t)n)) != cudaSuccess) return e;
  // the total-degree start system's powers are needed only with a homotopy and no g
  double *spow = (gamma && !g) ? ctx->spow.as<double>() : nullptr;
  const long fs = (long)(f->maxv + 1) * f->Mp;
  const long gs = g ? (long)(g->maxv + 1) * g->Mp : 0;
  if ((e = ctx->slots.ensure(sizeof(double) * 2 * L * (size_t)(fs + gs + 1))) != cudaSuccess) return e;
  double *ptab = ctx->ptab.as<double>(), *scal = ctx->scal.as<double>();
  double *fslots = ctx->slots.as<double>(), *gslots = fslots + 2 * L * fs;
  cudaStream_t st = ctx->stream;

  if (parts & 1)
    k_prep<P><<<(n + 127) / 128, 128, 0, st>>>(x, n, emax, ptab, f->deg.as<int32_t>(), spow, t,
                                               gamma, k, scal, skip);
  if (parts & 2) {
    if (f->M > 0) ad_launch<P>(f, ptab, n, fslots, fs, skip, st);
    if (g && g->M > 0) ad_launch<P>(g, ptab, n, gslots, gs, skip, st);
  }
  if (parts & 4) {
    tune_sum<P>(ctx, f, g);
    sum_launch<P>(f->sum_lanes > 0 ? f->sum_lanes : 8, f, g, N, n, fslots, fs, gslots, gs, spow,
                  scal, gamma != nullptr, J, ldJ, Jplane, h, rhs, rhs_plane, res_bits, skip, st,
                  0, 0, fixed);
  }
  return cudaGetLastError();
}

// h(x, t) alone in the working precision: the power table and the factors,
// the value of every term, and the summation of the N outputs of h only; the
// leading limbs of -h go to rhs ([re|im], planes rhs_plane apart) and
// max_i |h_i| to *res_bits.
template <class P>
cudaError_t eval_values_impl(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                             const double *gamma, int k, const double *t, const double *x,
                             double *rhs, long rhs_plane, const int *skip,
                             unsigned long long *res_bits, const uint8_t *fixed) {
  const int L = P::L, n = f->n, N = f->N;
  int emax = f->emax;
  if (g && g->emax > emax) emax = g->emax;
  const int ntab = emax > 2 ? emax - 1 : 1;
  cudaError_t e;
  if ((e = ctx->ptab.ensure(sizeof(double) * 2 * L * (size_t)n * ntab)) != cudaSuccess) return e;
  if ((e = ctx->scal.ensure(sizeof(double) * 3 * L)) != cudaSuccess) return e;
  if ((e = ctx->spow.ensure(sizeof(double) * 4 * L * (size_t)n)) != cudaSuccess) return e;
  double *spow = (gamma && !g) ? ctx->spow.as<double>() : nullptr;
  const long fs = (long)(f->maxv + 1) * f->Mp;
  const long gs = g ? (long)(g->maxv + 1) * g->Mp : 0;
  if ((e = ctx->slots.ensure(sizeof(double) * 2 * L * (size_t)(fs + gs + 1))) != cudaSuccess) return e;
  double *ptab = ctx->ptab.as<double>(), *scal = ctx->scal.as<double>();
  double *fslots = ctx->slots.as<double>(), *gslots = fslots + 2 * L * fs;
  cudaStream_t st = ctx->stream;
  k_prep<P><<<(n + 127) / 128, 128, 0, st>>>(x, n, emax, ptab, f->deg.as<int32_t>(), spow, t,
                                             gamma, k, scal, skip);
  if (f->M > 0)
    k_val<P><<<(f->M + 127) / 128, 128, 0, st>>>(f->M, f->Mp, f->nv.as<int32_t>(),
                                                 f->vidx.as<int32_t>(), f->vexp.as<int32_t>(),
                                                 f->coeff.as<double>(), ptab, n, emax, f->maxv,
                                                 fslots, fs, skip);
  if (g && g->M > 0)
    k_val<P><<<(g->M + 127) / 128, 128, 0, st>>>(g->M, g->Mp, g->nv.as<int32_t>(),
                                                 g->vidx.as<int32_t>(), g->vexp.as<int32_t>(),
                                                 g->coeff.as<double>(), ptab, n, emax, g->maxv,
                                                 gslots, gs, skip);
  tune_sum<P>(ctx, f, g);
  sum_launch<P>(f->sum_lanes > 0 ? f->sum_lanes : 8, f, g, N, n, fslots, fs, gslots, gs, spow,
                scal, gamma != nullptr, nullptr, 0, 0, nullptr, rhs, rhs_plane, res_bits, skip, st,
                n * N, 1, fixed);
  return cudaGetLastError();
}

}  // namespace

cudaError_t ph_eval_values_launch(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                  const double *gamma, int k, const double *t, const double *x,
                                  double *rhs, long rhs_plane, const int *skip,
                                  unsigned long long *res_bits, const uint8_t *fixed) {
  if (f->L == 1)
    return eval_values_impl<F64>(ctx, f, g, gamma, k, t, x, rhs, rhs_plane, skip, res_bits, fixed);
  if (f->L == 2)
    return eval_values_impl<DD>(ctx, f, g, gamma, k, t, x, rhs, rhs_plane, skip, res_bits, fixed);
  return eval_values_impl<QD>(ctx, f, g, gamma, k, t, x, rhs, rhs_plane, skip, res_bits, fixed);
}

// The evaluation in IEEE double of a system loaded with more limbs: every
// array is read through its leading limb (the limb-major layouts put limb 0
// first), the results are written in the one-limb layout.
cudaError_t ph_eval_launch_f64(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                               const double *gamma, int k, const double *t, const double *x,
                               double *J, long ldJ, long Jplane, const int *skip,
                               const uint8_t *fixed) {
  return eval_impl<F64>(ctx, f, g, gamma, k, t, x, nullptr, J, ldJ, Jplane, nullptr, 0, skip,
                        nullptr, 7, fixed);
}

cudaError_t ph_eval_launch_part(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                const double *gamma, int k, const double *t, const double *x,
                                double *h, double *J, long ldJ, long Jplane, double *rhs,
                                long rhs_plane, const int *skip, unsigned long long *res_bits,
                                int parts, const uint8_t *fixed) {
  if (f->L == 1)
    return eval_impl<F64>(ctx, f, g, gamma, k, t, x, h, J, ldJ, Jplane, rhs, rhs_plane, skip,
                          res_bits, parts, fixed);
  if (f->L == 2)
    return eval_impl<DD>(ctx, f, g, gamma, k, t, x, h, J, ldJ, Jplane, rhs, rhs_plane, skip,
                         res_bits, parts, fixed);
  return eval_impl<QD>(ctx, f, g, gamma, k, t, x, h, J, ldJ, Jplane, rhs, rhs_plane, skip,
                       res_bits, parts, fixed);
}

void ph_sum_tune(ph_ctx *ctx, const ph_system *f, const ph_system *g) {
  if (f->L == 1) tune_sum<F64>(ctx, f, g);
  else if (f->L == 2) tune_sum<DD>(ctx, f, g);
  else tune_sum<QD>(ctx, f, g);
}

extern "C" ph_status ph_sum_lanes(ph_ctx *ctx, const ph_system *f, const ph_system *g, int *lanes,
                                  double *ms) {
  if (!ctx) return PH_EINVAL;
  if (!f || f->ctx != ctx || !lanes || (g && (g->ctx != ctx || g->L != f->L || g->n != f->n)))
    return ph_fail(ctx, PH_EINVAL, "ph_sum_lanes: invalid argument");
  cudaSetDevice(ctx->device);
  ph_sum_tune(ctx, f, g);
  *lanes = f->sum_lanes > 0 ? f->sum_lanes : 8;
  if (ms)
    for (int v = 0; v < 6; ++v) ms[v] = f->sum_ms[v];
  return PH_OK;
}

cudaError_t ph_eval_launch(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                           const double *gamma, int k, const double *t, const double *x,
                           double *h, double *J, long ldJ, long Jplane, double *rhs,
                           long rhs_plane, const int *skip, unsigned long long *res_bits,
                           const uint8_t *fixed) {
  return ph_eval_launch_part(ctx, f, g, gamma, k, t, x, h, J, ldJ, Jplane, rhs, rhs_plane, skip,
                             res_bits, 7, fixed);
}
