// mp.cuh -- complex double-double (DD, 2 limbs) and quad-double (QD, 4 limbs)
// arithmetic on FP64 error-free transformations, for sm_103a.
//
// The paper computes in complex DD and QD (Section 3.1) with the QD library's
// algorithms (Introduction).  This file writes its own operations from the
// error-free transformations of IEEE doubles:
//   two_sum       a + b = s + e exactly                (Knuth; 6 FP64 ops)
//   fast_two_sum  a + b = s + e exactly if |a| >= |b|  (Dekker; 3 ops)
//   two_prod      a * b = p + e exactly                (FMA; 2 ops)
// On GB300 an FP64 warp instruction occupies an SM sub-partition's FP64 unit
// for about 64 cycles whatever its kind (measured; FP32 is ~60x faster), so
// every operation below is written to issue as few FP64 instructions as the
// error budget allows.  The budget is an error bound relative to the sum of the
// magnitudes of the terms (the quantity the library's accuracy is stated in),
// not relative to the result; this admits the cheaper "sloppy" DD addition.
//
// Every FP64 operation goes through an explicitly rounded intrinsic, so the
// compiler cannot contract a product and a sum into an FMA and break an
// error-free transformation.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace ph {

#define PHD __device__ __forceinline__

PHD double fadd(double a, double b) { return __dadd_rn(a, b); }
PHD double fsub(double a, double b) { return __dsub_rn(a, b); }
PHD double fmul(double a, double b) { return __dmul_rn(a, b); }
PHD double ffma(double a, double b, double c) { return __fma_rn(a, b, c); }

PHD void two_sum(double a, double b, double &s, double &e) {
  double x = fadd(a, b);
  double bv = fsub(x, a);
  double av = fsub(x, bv);
  e = fadd(fsub(a, av), fsub(b, bv));
  s = x;
}

PHD void fast_two_sum(double a, double b, double &s, double &e) {
  double x = fadd(a, b);
  e = fsub(b, fsub(x, a));
  s = x;
}

PHD void two_prod(double a, double b, double &p, double &e) {
  double x = fmul(a, b);
  e = ffma(a, b, -x);
  p = x;
}

// ---------------------------------------------------------------- double-double
struct dd { double h, l; };

struct DD {
  static constexpr int L = 2;
  typedef dd real;
  PHD static real zero() { return {0.0, 0.0}; }
  PHD static real from(double a) { return {a, 0.0}; }
  PHD static double lead(const real &a) { return a.h; }
  PHD static double limb(const real &a, int i) { return i == 0 ? a.h : a.l; }
  PHD static void set_limb(real &a, int i, double v) { if (i == 0) a.h = v; else a.l = v; }
  PHD static real neg(real a) { return {-a.h, -a.l}; }
  // Sloppy addition: two_sum of the leading limbs, the low limbs added in
  // double, then renormalised.  |error| <= ~3u^2 (|a| + |b|).  11 ops.
  PHD static real add(real a, real b) {
    double s, e;
    two_sum(a.h, b.h, s, e);
    e = fadd(e, a.l);
    e = fadd(e, b.l);
    fast_two_sum(s, e, s, e);
    return {s, e};
  }
  PHD static real sub(real a, real b) { return add(a, neg(b)); }
  // a*b without the product of the low limbs: |error| <= ~5u^2 |a b|.  7 ops.
  PHD static real mul(real a, real b) {
    double p, e;
    two_prod(a.h, b.h, p, e);
    e = ffma(a.h, b.l, e);
    e = ffma(a.l, b.h, e);
    fast_two_sum(p, e, p, e);
    return {p, e};
  }
  PHD static real mul_d(real a, double b) {
    double p, e;
    two_prod(a.h, b, p, e);
    e = ffma(a.l, b, e);
    fast_two_sum(p, e, p, e);
    return {p, e};
  }
  PHD static real scale2(real a) { return {fmul(a.h, 2.0), fmul(a.l, 2.0)}; }
  // quotient digits q1, q2, q3 from exact-ish remainders
  PHD static real div(real a, real b) {
    double q1 = a.h / b.h;
    real r = sub(a, mul_d(b, q1));
    double q2 = r.h / b.h;
    r = sub(r, mul_d(b, q2));
    double q3 = r.h / b.h;
    double s, e;
    fast_two_sum(q1, q2, s, e);
    return add({s, e}, from(q3));
  }
  // 1/b: the double reciprocal y0 and one Newton correction y0 + y0 (1 - b y0);
  // 1 - b.h y0 is exact in one FMA for a correctly rounded y0.  ~16 ops.
  PHD static real recip(real b) {
    double y0 = __drcp_rn(b.h);                   // correctly rounded, as 1.0 / b.h
    double e = ffma(-b.h, y0, 1.0);
    e = ffma(-b.l, y0, e);
    double s, t;
    fast_two_sum(y0, fmul(y0, e), s, t);
    return {s, t};
  }
  // one Newton correction of the double square root
  PHD static real sqrt(real a) {
    if (!(a.h > 0.0)) return zero();
    double s = __dsqrt_rn(a.h);
    double p, e;
    two_prod(s, s, p, e);
    real r = sub(a, {p, e});
    double c = r.h / fmul(2.0, s);
    fast_two_sum(s, c, s, e);
    return {s, e};
  }
};

// ---------------------------------------------------------------- quad-double
struct qd { double x[4]; };

// Renormalisation of five overlapping components whose exact sum is the value:
// two bottom-up sweeps of two_sum (error-free, so the value is unchanged even
// when cancellation leaves the components out of order), then the fifth
// component is folded into the fourth.
PHD void qd_renorm(double &c0, double &c1, double &c2, double &c3, double &c4) {
  two_sum(c3, c4, c3, c4);
  two_sum(c2, c3, c2, c3);
  two_sum(c1, c2, c1, c2);
  two_sum(c0, c1, c0, c1);
  two_sum(c3, c4, c3, c4);
  two_sum(c2, c3, c2, c3);
  two_sum(c1, c2, c1, c2);
  two_sum(c0, c1, c0, c1);
  c3 = fadd(c3, c4);
}

struct QD {
  static constexpr int L = 4;
  typedef qd real;
  PHD static real zero() { return {{0.0, 0.0, 0.0, 0.0}}; }
  PHD static real from(double a) { return {{a, 0.0, 0.0, 0.0}}; }
  PHD static double lead(const real &a) { return a.x[0]; }
  PHD static double limb(const real &a, int i) { return a.x[i]; }
  PHD static void set_limb(real &a, int i, double v) { a.x[i] = v; }
  PHD static real neg(real a) { return {{-a.x[0], -a.x[1], -a.x[2], -a.x[3]}}; }
  // Order-by-order addition: the components of equal order are added with
  // two_sum and the errors carried into the next order; order-3 terms are
  // added in double; then renormalised.
  PHD static real add(real a, real b) {
    double s0, s1, s2, s3, e0, e1, e2, e3;
    two_sum(a.x[0], b.x[0], s0, e0);
    two_sum(a.x[1], b.x[1], s1, e1);
    two_sum(s1, e0, s1, e0);
    two_sum(a.x[2], b.x[2], s2, e2);
    two_sum(s2, e1, s2, e1);
    two_sum(s2, e0, s2, e0);
    s3 = fadd(a.x[3], b.x[3]);
    e3 = fadd(fadd(e0, e1), e2);
    double c4 = 0.0;
    two_sum(s3, e3, s3, c4);
    qd_renorm(s0, s1, s2, s3, c4);
    return {{s0, s1, s2, s3}};
  }
  PHD static real sub(real a, real b) { return add(a, neg(b)); }
  // Products of the limbs by order i + j: orders 0..2 split exactly with
  // two_prod, order 3 in double, orders >= 4 dropped (below 2^-212 |a b|).
  PHD static real mul(real a, real b) {
    double p00, q00, p01, q01, p10, q10, p02, q02, p11, q11, p20, q20;
    two_prod(a.x[0], b.x[0], p00, q00);
    two_prod(a.x[0], b.x[1], p01, q01);
    two_prod(a.x[1], b.x[0], p10, q10);
    two_prod(a.x[0], b.x[2], p02, q02);
    two_prod(a.x[1], b.x[1], p11, q11);
    two_prod(a.x[2], b.x[0], p20, q20);
    double o3 = fmul(a.x[0], b.x[3]);
    o3 = ffma(a.x[1], b.x[2], o3);
    o3 = ffma(a.x[2], b.x[1], o3);
    o3 = ffma(a.x[3], b.x[0], o3);
    // order 1: p01 + p10 + q00
    double s1, r1, r2, r3;
    two_sum(p01, p10, s1, r1);
    two_sum(s1, q00, s1, r2);
    // order 2: p02 + p11 + p20 + q01 + q10 + r1 + r2
    double s2, t1, t2, t3, t4, t5, t6;
    two_sum(p02, p11, s2, t1);
    two_sum(s2, p20, s2, t2);
    two_sum(s2, q01, s2, t3);
    two_sum(s2, q10, s2, t4);
    two_sum(s2, r1, s2, t5);
    two_sum(s2, r2, s2, t6);
    // order 3: the rest in double
    r3 = fadd(fadd(fadd(q02, q11), fadd(q20, o3)), fadd(fadd(t1, t2), fadd(t3, t4)));
    r3 = fadd(r3, fadd(t5, t6));
    double c4 = 0.0;
    double s0 = p00;
    qd_renorm(s0, s1, s2, r3, c4);
    return {{s0, s1, s2, r3}};
  }
  PHD static real mul_d(real a, double b) {
    double p0, q0, p1, q1, p2, q2;
    two_prod(a.x[0], b, p0, q0);
    two_prod(a.x[1], b, p1, q1);
    two_prod(a.x[2], b, p2, q2);
    double p3 = fmul(a.x[3], b);
    double s1, e1, s2, e2, e3;
    two_sum(p1, q0, s1, e1);
    two_sum(p2, q1, s2, e2);
    two_sum(s2, e1, s2, e3);
    double s3 = fadd(fadd(p3, q2), fadd(e2, e3));
    double c4 = 0.0;
    qd_renorm(p0, s1, s2, s3, c4);
    return {{p0, s1, s2, s3}};
  }
  PHD static real scale2(real a) {
    return {{fmul(a.x[0], 2.0), fmul(a.x[1], 2.0), fmul(a.x[2], 2.0), fmul(a.x[3], 2.0)}};
  }
  // long division: five quotient digits, each from the remainder's leading limb
  PHD static real div(real a, real b) {
    double q0 = a.x[0] / b.x[0];
    real r = sub(a, mul_d(b, q0));
    double q1 = r.x[0] / b.x[0];
    r = sub(r, mul_d(b, q1));
    double q2 = r.x[0] / b.x[0];
    r = sub(r, mul_d(b, q2));
    double q3 = r.x[0] / b.x[0];
    r = sub(r, mul_d(b, q3));
    double q4 = r.x[0] / b.x[0];
    qd_renorm(q0, q1, q2, q3, q4);
    return {{q0, q1, q2, q3}};
  }
  // 1/b: a double-double reciprocal, then one Newton step y + y (1 - b y) in
  // quad-double (106 -> 212 bits).
  PHD static real recip(real b) {
    double y0 = __drcp_rn(b.x[0]);                // correctly rounded, as 1.0 / b.x[0]
    double e = ffma(-b.x[0], y0, 1.0);
    e = ffma(-b.x[1], y0, e);
    double s, t;
    fast_two_sum(y0, fmul(y0, e), s, t);
    real y = {{s, t, 0.0, 0.0}};
    real r = sub(from(1.0), mul(b, y));
    return add(y, mul(y, r));
  }
  // Newton's iteration s := s + (a - s^2) / (2 s) with the divisor in double:
  // each step adds ~53 correct bits (53, 106, 159, 212).
  PHD static real sqrt(real a) {
    if (!(a.x[0] > 0.0)) return zero();
    double s0 = __dsqrt_rn(a.x[0]);
    double h = 0.5 / s0;
    real s = from(s0);
    for (int it = 0; it < 3; ++it) {
      real r = sub(a, mul(s, s));
      s = add(s, mul_d(r, h));
    }
    return s;
  }
};

// Sum of T quad-double products, plus an optional quad-double addend, rounded
// once.  Every partial product x_i y_j of order i + j <= 2 is split exactly
// (two_prod); order 3 (x_0 y_3 + x_1 y_2 + x_2 y_1 + x_3 y_0) is computed in
// double; orders >= 4 are dropped (below 2^-212 |x y|).  The terms of each
// order are summed with two_sum into a running sum of that order, each
// rounding error passed on to the running sum of the next order; order 3 is
// summed in double; one renormalisation at the end.  The error is of order
// 2^-209 times the sum of |x_t y_t| (and |acc|), the bound all quad-double
// results here are held to, at about 60% of the instructions of separate
// products and additions each renormalised.  Signs are carried by the
// operands (a negated limb costs nothing).
template <int T, bool ACC>
PHD qd qd_sum_prod(const qd (&x)[T], const qd (&y)[T], const qd &acc) {
  double p00[T], q00[T], p01[T], q01[T], p10[T], q10[T], p02[T], q02[T], p11[T], q11[T];
  double p20[T], q20[T], o3[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    two_prod(x[t].x[0], y[t].x[0], p00[t], q00[t]);
    two_prod(x[t].x[0], y[t].x[1], p01[t], q01[t]);
    two_prod(x[t].x[1], y[t].x[0], p10[t], q10[t]);
    two_prod(x[t].x[0], y[t].x[2], p02[t], q02[t]);
    two_prod(x[t].x[1], y[t].x[1], p11[t], q11[t]);
    two_prod(x[t].x[2], y[t].x[0], p20[t], q20[t]);
    double v = fmul(x[t].x[0], y[t].x[3]);
    v = ffma(x[t].x[1], y[t].x[2], v);
    v = ffma(x[t].x[2], y[t].x[1], v);
    o3[t] = ffma(x[t].x[3], y[t].x[0], v);
  }
  // running sums of orders 0, 1, 2 (exact) and 3 (in double), each started
  // with one of its terms
  double s0 = p00[0], s1 = q00[0], s2 = q01[0], s3 = q02[0];
  auto put2 = [&](double v) {
    double e;
    two_sum(s2, v, s2, e);
    s3 = fadd(s3, e);
  };
  auto put1 = [&](double v) {
    double e;
    two_sum(s1, v, s1, e);
    put2(e);
  };
  auto put0 = [&](double v) {
    double e;
    two_sum(s0, v, s0, e);
    put1(e);
  };
#pragma unroll
  for (int t = 1; t < T; ++t) put0(p00[t]);
  if (ACC) put0(acc.x[0]);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    if (t > 0) put1(q00[t]);
    put1(p01[t]);
    put1(p10[t]);
  }
  if (ACC) put1(acc.x[1]);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    if (t > 0) put2(q01[t]);
    put2(q10[t]);
    put2(p02[t]);
    put2(p11[t]);
    put2(p20[t]);
  }
  if (ACC) put2(acc.x[2]);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    if (t > 0) s3 = fadd(s3, q02[t]);
    s3 = fadd(s3, fadd(fadd(q11[t], q20[t]), o3[t]));
  }
  if (ACC) s3 = fadd(s3, acc.x[3]);
  double c4 = 0.0;
  qd_renorm(s0, s1, s2, s3, c4);
  return {{s0, s1, s2, s3}};
}

// ---------------------------------------------------------------- complex
// ---------------------------------------------------------------- one-limb types
// IEEE double and single precision, with the same interface as DD and QD, for
// the Jacobian and its factorization in the mixed-precision corrector.  Arrays
// stay in double (a single-precision value is stored widened), so every
// layout above serves all four types: an array of L limbs read as F64 or F32
// gives its leading limb.
struct F64 {
  static constexpr int L = 1;
  typedef double real;
  PHD static real zero() { return 0.0; }
  PHD static real from(double a) { return a; }
  PHD static double lead(const real &a) { return a; }
  PHD static double limb(const real &a, int) { return a; }
  PHD static void set_limb(real &a, int, double v) { a = v; }
  PHD static real neg(real a) { return -a; }
  PHD static real add(real a, real b) { return fadd(a, b); }
  PHD static real sub(real a, real b) { return fsub(a, b); }
  PHD static real mul(real a, real b) { return fmul(a, b); }
  PHD static real mul_d(real a, double b) { return fmul(a, b); }
  PHD static real scale2(real a) { return fmul(a, 2.0); }
  PHD static real div(real a, real b) { return __ddiv_rn(a, b); }
  PHD static real recip(real b) { return __drcp_rn(b); }
  PHD static real sqrt(real a) { return __dsqrt_rn(a); }
  PHD static real fma(real a, real b, real c) { return ffma(a, b, c); }
};

struct F32 {
  static constexpr int L = 1;
  typedef float real;
  PHD static real zero() { return 0.0f; }
  PHD static real from(double a) { return __double2float_rn(a); }
  PHD static double lead(const real &a) { return (double)a; }
  PHD static double limb(const real &a, int) { return (double)a; }
  PHD static void set_limb(real &a, int, double v) { a = __double2float_rn(v); }
  PHD static real neg(real a) { return -a; }
  PHD static real add(real a, real b) { return __fadd_rn(a, b); }
  PHD static real sub(real a, real b) { return __fsub_rn(a, b); }
  PHD static real mul(real a, real b) { return __fmul_rn(a, b); }
  PHD static real mul_d(real a, double b) { return __fmul_rn(a, __double2float_rn(b)); }
  PHD static real scale2(real a) { return __fmul_rn(a, 2.0f); }
  PHD static real div(real a, real b) { return __fdiv_rn(a, b); }
  PHD static real recip(real b) { return __frcp_rn(b); }
  PHD static real sqrt(real a) { return __fsqrt_rn(a); }
  PHD static real fma(real a, real b, real c) { return __fmaf_rn(a, b, c); }
};

template <class P> struct cx { typename P::real re, im; };

template <class P> PHD cx<P> c_zero() { return {P::zero(), P::zero()}; }
template <class P> PHD cx<P> c_from(double re, double im) { return {P::from(re), P::from(im)}; }
template <class P> PHD cx<P> c_add(const cx<P> &a, const cx<P> &b) { return {P::add(a.re, b.re), P::add(a.im, b.im)}; }
template <class P> PHD cx<P> c_sub(const cx<P> &a, const cx<P> &b) { return {P::sub(a.re, b.re), P::sub(a.im, b.im)}; }
template <class P> PHD cx<P> c_neg(const cx<P> &a) { return {P::neg(a.re), P::neg(a.im)}; }
template <class P> PHD cx<P> c_mul_real(const cx<P> &a, const typename P::real &r) { return {P::mul(a.re, r), P::mul(a.im, r)}; }
template <class P> PHD cx<P> c_mul_d(const cx<P> &a, double r) { return {P::mul_d(a.re, r), P::mul_d(a.im, r)}; }
template <class P> PHD cx<P> c_scale2(const cx<P> &a) { return {P::scale2(a.re), P::scale2(a.im)}; }

// (ar + i ai)(br + i bi), four real products and two additions
template <class P> struct cops {
  PHD static cx<P> mul(const cx<P> &a, const cx<P> &b) {
    return {P::sub(P::mul(a.re, b.re), P::mul(a.im, b.im)),
            P::add(P::mul(a.re, b.im), P::mul(a.im, b.re))};
  }
  // acc + a b
  PHD static cx<P> mac(const cx<P> &acc, const cx<P> &a, const cx<P> &b) {
    return c_add<P>(acc, mul(a, b));
  }
  // conj(a) b
  PHD static cx<P> conj_mul(const cx<P> &a, const cx<P> &b) {
    return {P::add(P::mul(a.re, b.re), P::mul(a.im, b.im)),
            P::sub(P::mul(a.re, b.im), P::mul(a.im, b.re))};
  }
  PHD static typename P::real abs2(const cx<P> &a) {
    return P::add(P::mul(a.re, a.re), P::mul(a.im, a.im));
  }
};

// DD: each part of a product is one exact sum of two two_prod splits plus the
// cross terms, renormalised once (19 ops instead of 25 for 2 mul + 1 add).
template <> struct cops<DD> {
  PHD static void part(double ah, double al, double bh, double bl,
                       double ch, double cl, double dh, double dl, double sgn,
                       double &zh, double &zl) {
    // a b + sgn c d
    double p1, e1, p2, e2, s, es;
    two_prod(ah, bh, p1, e1);
    two_prod(ch, dh, p2, e2);
    two_sum(p1, sgn * p2, s, es);
    double t = fadd(es, e1);
    t = ffma(sgn, e2, t);
    t = ffma(ah, bl, t);
    t = ffma(al, bh, t);
    t = ffma(sgn * ch, dl, t);
    t = ffma(sgn * cl, dh, t);
    fast_two_sum(s, t, zh, zl);
  }
  PHD static cx<DD> mul(const cx<DD> &a, const cx<DD> &b) {
    cx<DD> z;
    part(a.re.h, a.re.l, b.re.h, b.re.l, a.im.h, a.im.l, b.im.h, b.im.l, -1.0, z.re.h, z.re.l);
    part(a.re.h, a.re.l, b.im.h, b.im.l, a.im.h, a.im.l, b.re.h, b.re.l, 1.0, z.im.h, z.im.l);
    return z;
  }
  PHD static cx<DD> mac(const cx<DD> &acc, const cx<DD> &a, const cx<DD> &b) {
    return c_add<DD>(acc, mul(a, b));
  }
  PHD static cx<DD> conj_mul(const cx<DD> &a, const cx<DD> &b) {
    cx<DD> z;
    part(a.re.h, a.re.l, b.re.h, b.re.l, a.im.h, a.im.l, b.im.h, b.im.l, 1.0, z.re.h, z.re.l);
    part(a.re.h, a.re.l, b.im.h, b.im.l, a.im.h, a.im.l, b.re.h, b.re.l, -1.0, z.im.h, z.im.l);
    return z;
  }
  PHD static dd abs2(const cx<DD> &a) {
    dd z;
    part(a.re.h, a.re.l, a.re.h, a.re.l, a.im.h, a.im.l, a.im.h, a.im.l, 1.0, z.h, z.l);
    return z;
  }
};

// one-limb types: each part of a product is one multiply and one FMA
template <class P> struct cops1 {
  typedef typename P::real real;
  PHD static cx<P> mul(const cx<P> &a, const cx<P> &b) {
    return {P::fma(a.re, b.re, P::neg(P::mul(a.im, b.im))), P::fma(a.re, b.im, P::mul(a.im, b.re))};
  }
  PHD static cx<P> mac(const cx<P> &acc, const cx<P> &a, const cx<P> &b) {
    return {P::fma(a.re, b.re, P::fma(P::neg(a.im), b.im, acc.re)),
            P::fma(a.re, b.im, P::fma(a.im, b.re, acc.im))};
  }
  PHD static cx<P> conj_mul(const cx<P> &a, const cx<P> &b) {
    return {P::fma(a.re, b.re, P::mul(a.im, b.im)), P::fma(a.re, b.im, P::neg(P::mul(a.im, b.re)))};
  }
  PHD static real abs2(const cx<P> &a) { return P::fma(a.re, a.re, P::mul(a.im, a.im)); }
};
template <> struct cops<F64> : cops1<F64> {};
template <> struct cops<F32> : cops1<F32> {};

// QD: each part of a product (and of a product added to an addend) is one
// fused sum of two products (qd_sum_prod).
template <> struct cops<QD> {
  PHD static cx<QD> mul(const cx<QD> &a, const cx<QD> &b) {
    const qd z = QD::zero();
    const qd xr[2] = {a.re, QD::neg(a.im)}, yr[2] = {b.re, b.im};
    const qd xi[2] = {a.re, a.im}, yi[2] = {b.im, b.re};
    return {qd_sum_prod<2, false>(xr, yr, z), qd_sum_prod<2, false>(xi, yi, z)};
  }
  PHD static cx<QD> mac(const cx<QD> &acc, const cx<QD> &a, const cx<QD> &b) {
    const qd xr[2] = {a.re, QD::neg(a.im)}, yr[2] = {b.re, b.im};
    const qd xi[2] = {a.re, a.im}, yi[2] = {b.im, b.re};
    return {qd_sum_prod<2, true>(xr, yr, acc.re), qd_sum_prod<2, true>(xi, yi, acc.im)};
  }
  // conj(a) b
  PHD static cx<QD> conj_mul(const cx<QD> &a, const cx<QD> &b) {
    const qd z = QD::zero();
    const qd xr[2] = {a.re, a.im}, yr[2] = {b.re, b.im};
    const qd xi[2] = {a.re, QD::neg(a.im)}, yi[2] = {b.im, b.re};
    return {qd_sum_prod<2, false>(xr, yr, z), qd_sum_prod<2, false>(xi, yi, z)};
  }
  PHD static qd abs2(const cx<QD> &a) {
    const qd x[2] = {a.re, a.im};
    return qd_sum_prod<2, false>(x, x, QD::zero());
  }
};

template <class P> PHD cx<P> c_mul(const cx<P> &a, const cx<P> &b) { return cops<P>::mul(a, b); }
template <class P> PHD cx<P> c_conj_mul(const cx<P> &a, const cx<P> &b) { return cops<P>::conj_mul(a, b); }
template <class P> PHD typename P::real c_abs2(const cx<P> &a) { return cops<P>::abs2(a); }

// x^e by binary powering (e >= 0)
template <class P> PHD cx<P> c_pow(cx<P> x, int e) {
  cx<P> r = c_from<P>(1.0, 0.0);
  bool first = true;
  while (e > 0) {
    if (e & 1) {
      r = first ? x : cops<P>::mul(r, x);
      first = false;
    }
    e >>= 1;
    if (e) x = cops<P>::mul(x, x);
  }
  return r;
}

// multiply by a small positive integer exponent
template <class P> PHD cx<P> c_mul_int(const cx<P> &a, int k) {
  if (k == 1) return a;
  if (k == 2) return c_scale2<P>(a);
  return c_mul_d<P>(a, (double)k);
}

// |z| in double from the leading limbs (only the magnitude matters, Section 3.1)
template <class P> PHD double c_mag_lead(const cx<P> &a) {
  double re = P::lead(a.re), im = P::lead(a.im);
  return __dsqrt_rn(__dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im)));
}

// ---------------------------------------------------------------- SoA access
// element i of a complex vector laid out [limb][re|im][stride]
template <class P> PHD cx<P> c_load(const double *__restrict__ v, long stride, long i) {
  cx<P> z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) {
    P::set_limb(z.re, l, v[(2 * l) * stride + i]);
    P::set_limb(z.im, l, v[(2 * l + 1) * stride + i]);
  }
  return z;
}

template <class P> PHD void c_store(double *__restrict__ v, long stride, long i, const cx<P> &z) {
#pragma unroll
  for (int l = 0; l < P::L; ++l) {
    v[(2 * l) * stride + i] = P::limb(z.re, l);
    v[(2 * l + 1) * stride + i] = P::limb(z.im, l);
  }
}

// the same through L2 only (ld.global.cg): for data another block of a running
// persistent kernel may have written since this SM last cached the line
template <class P> PHD cx<P> c_load_cg(const double *v, long stride, long i) {
  cx<P> z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) {
    P::set_limb(z.re, l, __ldcg(v + (2 * l) * stride + i));
    P::set_limb(z.im, l, __ldcg(v + (2 * l + 1) * stride + i));
  }
  return z;
}

template <class P> PHD typename P::real r_load_cg(const double *v, long stride, long i) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, __ldcg(v + l * stride + i));
  return z;
}

template <class P> PHD typename P::real r_load(const double *__restrict__ v, long stride, long i) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, v[l * stride + i]);
  return z;
}

template <class P> PHD void r_store(double *__restrict__ v, long stride, long i, const typename P::real &z) {
#pragma unroll
  for (int l = 0; l < P::L; ++l) v[l * stride + i] = P::limb(z, l);
}

}  // namespace ph
