// pathdev.cuh -- device functions of the evaluation shared by the single-path
// kernels (eval.cu) and the many-path kernel (batch.cu).
//
// Layouts (see system.cu): sorted term s at position p reads vidx/vexp[p*Mp+s];
// its partial derivative with respect to that variable goes to slot p*Mp+s and
// its value to slot maxv*Mp+s of a slot buffer [2L][nslots]; ptab holds x^e at
// [(e-1)][2L][n]; spow holds the start system's d_i x_i^{d_i-1} at [0][2L][n]
// and x_i^{d_i} - 1 at [1][2L][n].
#pragma once
#include <type_traits>

#include "mp.cuh"
#include "qfx.cuh"

namespace ph {

// The complex product of the term evaluation: in QD the 256-bit fixed-point
// form (qfx.cuh), which is faster than the FP64 form both in throughput and
// along one dependent chain (measured: ~8,900 against ~16,000 cycles for a
// QD sum of two products on one warp); the FP64 forms otherwise.  (In DD the
// fixed-point product measured slower along the AD's dependent chains.)
template <class P>
PHD cx<P> c_mul_ad(const cx<P> &a, const cx<P> &b) {
  if constexpr (std::is_same<P, QD>::value) return qf_cmul(a, b);
  else return c_mul<P>(a, b);
}

// Powers of one variable for the power table (x^1 .. x^{emax-1}) and, for the
// total-degree start system, d x^{d-1} and x^d - 1.
template <class P>
__device__ void prep_variable(int j, const double *__restrict__ x, int n, int emax,
                              double *__restrict__ ptab, const int32_t *__restrict__ deg,
                              double *__restrict__ spow) {
  const long pl = 2L * P::L * n;
  cx<P> xj = c_load<P>(x, n, j);
  c_store<P>(ptab, n, j, xj);
  cx<P> p = xj;
  for (int e = 2; e < emax; ++e) {
    p = c_mul<P>(p, xj);
    c_store<P>(ptab + (e - 1) * pl, n, j, p);
  }
  if (spow) {
    const int d = deg[j];
    cx<P> pw = c_pow<P>(xj, d - 1);                       // x^{d-1}
    c_store<P>(spow, n, j, c_mul_d<P>(pw, (double)d));
    cx<P> xd = c_mul<P>(pw, xj);
    xd.re = P::sub(xd.re, P::from(1.0));
    c_store<P>(spow + pl, n, j, xd);
  }
}

// t^k (real) and gamma (1-t)^k (complex) into scal: [L] then [2L]
template <class P>
__device__ void prep_factors(const double *__restrict__ t, const double *__restrict__ gamma,
                             int k, double *__restrict__ scal) {
  typename P::real tt = r_load<P>(t, 1, 0);
  typename P::real omt = P::sub(P::from(1.0), tt);
  typename P::real tk = P::from(1.0), ok = P::from(1.0);
  for (int e = 0; e < k; ++e) {
    tk = P::mul(tk, tt);
    ok = P::mul(ok, omt);
  }
  cx<P> g = c_load<P>(gamma, 1, 0);
  r_store<P>(scal, 1, 0, tk);
  c_store<P>(scal + P::L, 1, 0, c_mul_real<P>(g, ok));
}

// Reverse-mode differentiation of sorted term s by one thread: the common
// factor prod x_j^{a_j-1} is folded into the coefficient, then forward prefix
// products (parked in the slots), backward suffix and cross products:
//   d/dx_j (c x^a) = a_j (c CF x_1..x_{j-1}) (x_{j+1}..x_v).
template <class P>
__device__ void ad_term(int s, int Mp, const int32_t *__restrict__ nv,
                        const int32_t *__restrict__ vidx, const int32_t *__restrict__ vexp,
                        const double *__restrict__ coeff, const double *__restrict__ ptab, int n,
                        int maxv, double *__restrict__ slots, long nslots) {
  const long pl = 2L * P::L * n;
  const int v = nv[s];
  cx<P> c = c_load<P>(coeff, Mp, s);
  for (int p = 0; p < v; ++p) {
    int a = vexp[(long)p * Mp + s];
    if (a >= 2) c = c_mul_ad<P>(c, c_load<P>(ptab + (a - 2) * pl, n, vidx[(long)p * Mp + s]));
  }
  cx<P> pre = c;
  for (int p = 0; p < v; ++p) {
    c_store<P>(slots, nslots, (long)p * Mp + s, pre);
    pre = c_mul_ad<P>(pre, c_load<P>(ptab, n, vidx[(long)p * Mp + s]));
  }
  c_store<P>(slots, nslots, (long)maxv * Mp + s, pre);
  cx<P> suf = c_zero<P>();
  for (int p = v - 1; p >= 0; --p) {
    cx<P> d = c_load<P>(slots, nslots, (long)p * Mp + s);
    if (p < v - 1) d = c_mul_ad<P>(d, suf);
    d = c_mul_int<P>(d, vexp[(long)p * Mp + s]);
    c_store<P>(slots, nslots, (long)p * Mp + s, d);
    if (p > 0) {
      cx<P> xj = c_load<P>(ptab, n, vidx[(long)p * Mp + s]);
      suf = (p == v - 1) ? xj : c_mul_ad<P>(suf, xj);
    }
  }
}

// Value alone of sorted term s (c x^a) by one thread, into its value slot
// maxv*Mp+s: each variable's power from the power table, which holds x^1 ..
// x^{emax-1} (x^a, or x^{a-1} x when a = emax >= 2).  The residual of
// the mixed-precision corrector needs h(x,t) only; this is v complex products
// per term where the reverse mode takes about 3v.
template <class P>
__device__ void val_term(int s, int Mp, const int32_t *__restrict__ nv,
                         const int32_t *__restrict__ vidx, const int32_t *__restrict__ vexp,
                         const double *__restrict__ coeff, const double *__restrict__ ptab, int n,
                         int emax, int maxv, double *__restrict__ slots, long nslots) {
  const long pl = 2L * P::L * n;
  const int v = nv[s];
  cx<P> c = c_load<P>(coeff, Mp, s);
  for (int p = 0; p < v; ++p) {
    const int a = vexp[(long)p * Mp + s], j = vidx[(long)p * Mp + s];
    if (a == 1 || a < emax) {
      c = c_mul_ad<P>(c, c_load<P>(ptab + (a - 1) * pl, n, j));
    } else {
      c = c_mul_ad<P>(c, c_load<P>(ptab + (a - 2) * pl, n, j));
      c = c_mul_ad<P>(c, c_load<P>(ptab, n, j));
    }
  }
  c_store<P>(slots, nslots, (long)maxv * Mp + s, c);
}

template <class P>
PHD cx<P> shfl_down_c(const cx<P> &a, int off, int width) {
  cx<P> z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) {
    P::set_limb(z.re, l, __shfl_down_sync(0xffffffffu, P::limb(a.re, l), off, width));
    P::set_limb(z.im, l, __shfl_down_sync(0xffffffffu, P::limb(a.im, l), off, width));
  }
  return z;
}

// Summation of output o by the G lanes of a group (every lane of the warp must
// call this, active or not).  Returns the finished output on lane 0 of the
// group: the sum of its slots (in the order of the terms), times t^k when a
// homotopy is evaluated, plus gamma (1-t)^k times the start system's term
// (from g's slots, or from spow for the total-degree system).  fixed (may be
// null): rows held fixed, h_i = f_i (g_i is the zero polynomial there).
template <class P, int G>
__device__ cx<P> sum_output(bool active, int o, int lane, int N, int n,
                            const int32_t *__restrict__ optr, const int32_t *__restrict__ oslot,
                            const double *__restrict__ slots, long nslots,
                            const int32_t *__restrict__ goptr, const int32_t *__restrict__ goslot,
                            const double *__restrict__ gslots, long gnslots,
                            const double *__restrict__ spow, const double *__restrict__ scal,
                            int homotopy, const uint8_t *__restrict__ fixed = nullptr) {
  cx<P> af = c_zero<P>(), ag = c_zero<P>();
  if (active) {
    for (int q = optr[o] + lane; q < optr[o + 1]; q += G)
      af = c_add<P>(af, c_load<P>(slots, nslots, oslot[q]));
    if (goptr)
      for (int q = goptr[o] + lane; q < goptr[o + 1]; q += G)
        ag = c_add<P>(ag, c_load<P>(gslots, gnslots, goslot[q]));
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    af = c_add<P>(af, shfl_down_c<P>(af, off, G));
    if (goptr) ag = c_add<P>(ag, shfl_down_c<P>(ag, off, G));
  }
  if (!active || lane != 0 || !homotopy) return af;
  const int nN = n * N;
  if (fixed && fixed[o < nN ? o % N : o - nN]) return af;
  const typename P::real sf = r_load<P>(scal, 1, 0);
  const cx<P> sg = c_load<P>(scal + P::L, 1, 0);
  cx<P> val = c_mul_real<P>(af, sf);
  if (goptr) return c_add<P>(val, c_mul<P>(sg, ag));
  const long pl = 2L * P::L * n;
  if (o < nN) {
    int j = o / N, i = o - j * N;
    if (i == j) val = c_add<P>(val, c_mul<P>(sg, c_load<P>(spow, n, i)));
  } else {
    val = c_add<P>(val, c_mul<P>(sg, c_load<P>(spow + pl, n, o - nN)));
  }
  return val;
}

// ---- per-part arithmetic (one real component of a complex quantity) -------------
//
// acc: an accumulator of real terms; dot2(x1,y1,x2,y2,sg) adds x1 y1 + sg x2 y2;
// sq(x) adds x^2; upd(a, ar, b, ai, c, sg) = a - ar b + sg ai c.

template <class P> struct Part {
  typedef typename P::real real;
  struct acc { real v; };
  PHD static acc zero() { return {P::zero()}; }
  PHD static void dot2(acc &a, const real &x1, const real &y1, const real &x2, const real &y2,
                       double sg) {
    real t = P::mul(x2, y2);
    if (sg < 0) t = P::neg(t);
    a.v = P::add(a.v, P::add(P::mul(x1, y1), t));
  }
  PHD static void sq(acc &a, const real &x) { a.v = P::add(a.v, P::mul(x, x)); }
  PHD static acc combine(const acc &a, const acc &b) { return {P::add(a.v, b.v)}; }
  PHD static acc shfl(const acc &a, int m) {
    acc z;
#pragma unroll
    for (int l = 0; l < P::L; ++l)
      P::set_limb(z.v, l, __shfl_xor_sync(0xffffffffu, P::limb(a.v, l), m));
    return z;
  }
  PHD static real value(const acc &a) { return a.v; }
  PHD static real upd(const real &a, const real &ar, const real &b, const real &ai,
                      const real &c, double sg) {
    real t = P::mul(ai, c);
    if (sg < 0) t = P::neg(t);
    return P::add(a, P::sub(t, P::mul(ar, b)));
  }
};

// one-limb types: fused multiply-adds
template <class P> struct Part1 {
  typedef typename P::real real;
  struct acc { real v; };
  PHD static acc zero() { return {P::zero()}; }
  PHD static void dot2(acc &a, const real &x1, const real &y1, const real &x2, const real &y2,
                       double sg) {
    a.v = P::fma(x1, y1, P::fma(sg < 0 ? P::neg(x2) : x2, y2, a.v));
  }
  PHD static void sq(acc &a, const real &x) { a.v = P::fma(x, x, a.v); }
  PHD static acc combine(const acc &a, const acc &b) { return {P::add(a.v, b.v)}; }
  PHD static acc shfl(const acc &a, int m) { return {__shfl_xor_sync(0xffffffffu, a.v, m)}; }
  PHD static real value(const acc &a) { return a.v; }
  PHD static real upd(const real &a, const real &ar, const real &b, const real &ai,
                      const real &c, double sg) {
    return P::fma(P::neg(ar), b, P::fma(sg < 0 ? P::neg(ai) : ai, c, a));
  }
};
template <> struct Part<F64> : Part1<F64> {};
template <> struct Part<F32> : Part1<F32> {};

// quad-double: every dot-product term and update is one fused sum of
// products with the accumulator as addend (qd_sum_prod)
template <> struct Part<QD> {
  typedef qd real;
  struct acc { qd v; };
  PHD static acc zero() { return {QD::zero()}; }
  PHD static void dot2(acc &a, const qd &x1, const qd &y1, const qd &x2, const qd &y2, double sg) {
    const qd x[2] = {x1, sg < 0 ? QD::neg(x2) : x2}, y[2] = {y1, y2};
    a.v = qd_sum_prod<2, true>(x, y, a.v);
  }
  PHD static void sq(acc &a, const qd &v) {
    const qd x[1] = {v};
    a.v = qd_sum_prod<1, true>(x, x, a.v);
  }
  PHD static acc combine(const acc &a, const acc &b) { return {QD::add(a.v, b.v)}; }
  PHD static acc shfl(const acc &a, int m) {
    acc z;
#pragma unroll
    for (int l = 0; l < 4; ++l) z.v.x[l] = __shfl_xor_sync(0xffffffffu, a.v.x[l], m);
    return z;
  }
  PHD static qd value(const acc &a) { return a.v; }
  // a - ar b + sg ai c
  PHD static qd upd(const qd &a, const qd &ar, const qd &b, const qd &ai, const qd &c, double sg) {
    const qd x[2] = {QD::neg(ar), sg < 0 ? QD::neg(ai) : ai}, y[2] = {b, c};
    return qd_sum_prod<2, true>(x, y, a);
  }
};

// double-double: Dot2-style unnormalised (s, c) accumulation
template <> struct Part<DD> {
  typedef dd real;
  struct acc { double s, c; };
  PHD static acc zero() { return {0.0, 0.0}; }
  PHD static void add_term(acc &a, double p) {
    double s, e;
    ph::two_sum(a.s, p, s, e);
    a.s = s;
    a.c = ph::fadd(a.c, e);
  }
  PHD static void dot2(acc &a, const dd &x1, const dd &y1, const dd &x2, const dd &y2, double sg) {
    double p1, e1, p2, e2;
    ph::two_prod(x1.h, y1.h, p1, e1);
    ph::two_prod(sg * x2.h, y2.h, p2, e2);
    double lo = ph::fadd(e1, e2);
    lo = ph::ffma(x1.h, y1.l, lo);
    lo = ph::ffma(x1.l, y1.h, lo);
    lo = ph::ffma(sg * x2.h, y2.l, lo);
    lo = ph::ffma(sg * x2.l, y2.h, lo);
    add_term(a, p1);
    add_term(a, p2);
    a.c = ph::fadd(a.c, lo);
  }
  PHD static void sq(acc &a, const dd &x) {
    double p, e;
    ph::two_prod(x.h, x.h, p, e);
    e = ph::ffma(2.0 * x.h, x.l, e);
    add_term(a, p);
    a.c = ph::fadd(a.c, e);
  }
  PHD static acc combine(const acc &a, const acc &b) {
    acc z;
    double e;
    ph::two_sum(a.s, b.s, z.s, e);
    z.c = ph::fadd(ph::fadd(a.c, b.c), e);
    return z;
  }
  PHD static acc shfl(const acc &a, int m) {
    return {__shfl_xor_sync(0xffffffffu, a.s, m), __shfl_xor_sync(0xffffffffu, a.c, m)};
  }
  PHD static dd value(const acc &a) {
    double s, e;
    ph::fast_two_sum(a.s, a.c, s, e);
    return {s, e};
  }
  // a - ar b + sg ai c with one renormalisation
  PHD static dd upd(const dd &a, const dd &ar, const dd &b, const dd &ai, const dd &c, double sg) {
    double p1, e1, p2, e2, s, es1, es2;
    ph::two_prod(ar.h, b.h, p1, e1);
    ph::two_prod(sg * ai.h, c.h, p2, e2);
    ph::two_sum(a.h, -p1, s, es1);
    ph::two_sum(s, p2, s, es2);
    double lo = ph::fadd(ph::fadd(a.l, es1), es2);
    lo = ph::fsub(lo, e1);
    lo = ph::fadd(lo, e2);
    lo = ph::ffma(-ar.h, b.l, lo);
    lo = ph::ffma(-ar.l, b.h, lo);
    lo = ph::ffma(sg * ai.h, c.l, lo);
    lo = ph::ffma(sg * ai.l, c.h, lo);
    double z, zl;
    ph::fast_two_sum(s, lo, z, zl);
    return {z, zl};
  }
};


}  // namespace ph
