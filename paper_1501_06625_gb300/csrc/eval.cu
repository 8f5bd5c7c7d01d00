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
//          suffix and cross products, Table "Evaluating four monomials"):
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
      cf = has_cf ? c_mul<P>(cf, w) : w;
      has_cf = true;
    }
  }
  const cx<P> c0 = (active && q == 0) ? c_load<P>(coeff, Mp, s) : one;
  cx<P> B = c0;
  bool b_one = !(active && q == 0);
  if (has_cf) { B = b_one ? cf : c_mul<P>(B, cf); b_one = false; }
  for (int p = p0; p < p1; ++p) {
    cx<P> xj = c_load<P>(ptab, n, vidx[(long)p * Mp + s]);
    B = b_one ? xj : c_mul<P>(B, xj);
    b_one = false;
  }
  // inclusive prefix and suffix products over the T lanes of this monomial
  cx<P> I = B, S = B;
#pragma unroll
  for (int d = 1; d < T; d <<= 1) {
    cx<P> y = shfl_up_c<P>(I, d, T);
    if (q >= d) I = c_mul<P>(y, I);
    cx<P> z = shfl_down_c<P>(S, d, T);
    if (q + d < T) S = c_mul<P>(S, z);
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
  if (q < T - 1) { outer = o_one ? right : c_mul<P>(outer, right); o_one = false; }
  if (has_cf) { outer = o_one ? cf : c_mul<P>(outer, cf); o_one = false; }
  if (o_one) outer = one;
  // local reverse sweep over the chunk (prefixes parked in the slots)
  cx<P> pre = outer;
  for (int p = p0; p < p1; ++p) {
    c_store<P>(slots, nslots, (long)p * Mp + s, pre);
    if (p + 1 < p1) pre = c_mul<P>(pre, c_load<P>(ptab, n, vidx[(long)p * Mp + s]));
  }
  cx<P> suf = one;
  for (int p = p1 - 1; p >= p0; --p) {
    cx<P> d = c_load<P>(slots, nslots, (long)p * Mp + s);
    if (p < p1 - 1) d = c_mul<P>(d, suf);
    d = c_mul_int<P>(d, vexp[(long)p * Mp + s]);
    c_store<P>(slots, nslots, (long)p * Mp + s, d);
    if (p > p0) {
      cx<P> xj = c_load<P>(ptab, n, vidx[(long)p * Mp + s]);
      suf = (p == p1 - 1) ? xj : c_mul<P>(suf, xj);
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
    const int *__restrict__ skip) {
  if (skip && *skip) return;
  long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  int o = (int)(gt / G);
  int lane = (int)(gt % G);
  bool active = o < nout;
  cx<P> val = sum_output<P, G>(active, o, lane, N, n, optr, oslot, slots, nslots, goptr, goslot,
                               gslots, gnslots, spow, scal, homotopy);
  if (!active || lane != 0) return;
  const int nN = n * N;
  if (o < nN) {
    int j = o / N, i = o - j * N;
    c_store<P>(J + (long)j * ldJ, Jplane, i, val);
  } else {
    int i = o - nN;
    if (h) c_store<P>(h, N, i, val);
    if (rhs) c_store<P>(rhs, rhs_plane, i, c_neg<P>(val));
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

template <class P>
cudaError_t eval_impl(ph_ctx *ctx, const ph_system *f, const ph_system *g, const double *gamma,
                      int k, const double *t, const double *x, double *h, double *J, long ldJ,
                      long Jplane, double *rhs, long rhs_plane, const int *skip,
                      unsigned long long *res_bits, int parts) {
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
  constexpr int G = 8;
  const long threads = (long)f->nout * G;
  if (parts & 4)
  k_sum<P, G><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      N, n, f->nout, f->out_ptr.as<int32_t>(), f->out_slot.as<int32_t>(), fslots, fs,
      g ? g->out_ptr.as<int32_t>() : nullptr, g ? g->out_slot.as<int32_t>() : nullptr, gslots, gs,
      spow, scal, gamma != nullptr, J, ldJ, Jplane, h, rhs, rhs_plane, res_bits, skip);
  return cudaGetLastError();
}

}  // namespace

cudaError_t ph_eval_launch_part(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                const double *gamma, int k, const double *t, const double *x,
                                double *h, double *J, long ldJ, long Jplane, double *rhs,
                                long rhs_plane, const int *skip, unsigned long long *res_bits,
                                int parts) {
  if (f->L == 1)
    return eval_impl<F64>(ctx, f, g, gamma, k, t, x, h, J, ldJ, Jplane, rhs, rhs_plane, skip,
                          res_bits, parts);
  if (f->L == 2)
    return eval_impl<DD>(ctx, f, g, gamma, k, t, x, h, J, ldJ, Jplane, rhs, rhs_plane, skip,
                         res_bits, parts);
  return eval_impl<QD>(ctx, f, g, gamma, k, t, x, h, J, ldJ, Jplane, rhs, rhs_plane, skip,
                       res_bits, parts);
}

cudaError_t ph_eval_launch(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                           const double *gamma, int k, const double *t, const double *x,
                           double *h, double *J, long ldJ, long Jplane, double *rhs,
                           long rhs_plane, const int *skip, unsigned long long *res_bits) {
  return ph_eval_launch_part(ctx, f, g, gamma, k, t, x, h, J, ldJ, Jplane, rhs, rhs_plane, skip,
                             res_bits, 7);
}
