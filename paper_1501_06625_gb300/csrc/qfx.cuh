// qfx.cuh -- quad-double values as 256-bit fixed-point integers with an
// exponent, for the steps of the solvers where a QD sum of products would
// take hundreds of FP64 instructions.
//
// A QD number (four doubles) holds about 212 significant bits, so it fits a
// 256-bit two's-complement integer m with a power-of-two scale: value = m 2^e.
// On this GPU an FP64 instruction occupies its SM sub-partition for ~64 cycles
// while integer instructions issue every cycle, and a QD product or sum of two
// products in FP64 form takes one to three hundred FP64 instructions (about
// 275 for one part of a complex update); in integers a product is ten
// 64 x 64-bit products of the top words and their carries.  Measured on one
// update a - x y + u v: 8,900 against 16,000 cycles along one warp's chain,
// 2.2x / 3.9x / 5.3x the throughput at 4 / 8 / 16 warps per SM.  Conversions place each limb's
// 53-bit significand at its offset; rounding back takes the nearest double
// four times from what remains (the correctly rounded four-limb value of the
// fixed-point result).  Truncation: a converted value keeps every bit down to
// 2^-252 of its leading limb's magnitude, a product drops partial products
// below 2^-246 of itself, and a sum is truncated below 2^-252 of its largest
// term: errors far below QD's 2^-209.
#pragma once
#include "exsum.cuh"

namespace ph {

typedef Fix<4> Q256;

// value m 2^e; |m| < 2^253
struct QF {
  Q256 m;
  int e;
};

constexpr int kQFZeroE = -1000000;       // the scale of zero: below any other value's

__device__ __forceinline__ Q256 q_zero() {
  Q256 r;
#pragma unroll
  for (int q = 0; q < 4; ++q) r.w[q] = 0ull;
  return r;
}

// arithmetic shift right by s >= 0 (s >= 256 leaves only the sign)
__device__ __forceinline__ Q256 q_sar(const Q256 &a, int s) {
  const unsigned long long fill = (long long)a.w[3] < 0 ? ~0ull : 0ull;
  if (s >= 256) {
    Q256 r;
#pragma unroll
    for (int q = 0; q < 4; ++q) r.w[q] = fill;
    return r;
  }
  const int ws = s >> 6, bs = s & 63;
  // src(k): word k of a, the sign fill above word 3 (selects, no indexed access)
  unsigned long long src[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    unsigned long long v = fill;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (k == q) v = a.w[q];
    src[k] = v;
  }
  Q256 r;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned long long lo = src[q + 3], hi = src[q + 4];
    if (ws == 0) { lo = src[q]; hi = src[q + 1]; }
    else if (ws == 1) { lo = src[q + 1]; hi = src[q + 2]; }
    else if (ws == 2) { lo = src[q + 2]; hi = src[q + 3]; }
    r.w[q] = bs ? (lo >> bs) | (hi << (64 - bs)) : lo;
  }
  return r;
}

// a 2^s for 0 <= s < 64 (no overflow by construction at the call sites)
__device__ __forceinline__ Q256 q_shl_small(const Q256 &a, int s) {
  if (s == 0) return a;
  Q256 r;
  r.w[0] = a.w[0] << s;
#pragma unroll
  for (int q = 1; q < 4; ++q) r.w[q] = (a.w[q] << s) | (a.w[q - 1] >> (64 - s));
  return r;
}

// the QD value x (limbs ordered by magnitude) in fixed point: the leading
// limb's top bit at bit 252.  *bad is set for a non-finite limb.
__device__ __forceinline__ QF qf_from(const qd &x, bool *bad) {
  QF r;
  r.m = q_zero();
  const unsigned ef0 = dbl_ef(x.x[0]);
  if (ef0 == 0u) {
    r.e = kQFZeroE;
    return r;
  }
  if (ef0 == 0x7ffu) *bad = true;
  r.e = (int)ef0 - 1023 - 252;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    int sg, e;
    unsigned long long m;
    dbl_fields(x.x[l], sg, m, e);
    if (dbl_ef(x.x[l]) == 0x7ffu) *bad = true;
    if (m == 0) continue;
    Q256 t = fix_place<4>(m, e - r.e);
    if (sg) t = fix_neg<4>(t);
    r.m = fix_add<4>(r.m, t);
  }
  return r;
}

// a b: the top 256 bits of the 512-bit product of the magnitudes (partial
// products below word 4 dropped), then shifted so that |m| < 2^253 again
__device__ __forceinline__ QF qf_mul(const QF &a, const QF &b) {
  const bool na = (long long)a.m.w[3] < 0, nb = (long long)b.m.w[3] < 0;
  const Q256 x = na ? fix_neg<4>(a.m) : a.m, y = nb ? fix_neg<4>(b.m) : b.m;
  typedef unsigned __int128 u128;
  auto hi = [](unsigned long long p, unsigned long long q) { return __umul64hi(p, q); };
  // column sums of words 4..7 of the product (u128: no carry is lost)
  u128 c4 = (u128)hi(x.w[0], y.w[3]) + hi(x.w[1], y.w[2]) + hi(x.w[2], y.w[1]) + hi(x.w[3], y.w[0]);
  c4 += (u128)(x.w[1] * y.w[3]) + (x.w[2] * y.w[2]) + (x.w[3] * y.w[1]);
  u128 c5 = (u128)hi(x.w[1], y.w[3]) + hi(x.w[2], y.w[2]) + hi(x.w[3], y.w[1]);
  c5 += (u128)(x.w[2] * y.w[3]) + (x.w[3] * y.w[2]);
  u128 c6 = (u128)hi(x.w[2], y.w[3]) + hi(x.w[3], y.w[2]);
  c6 += (u128)(x.w[3] * y.w[3]);
  u128 c7 = (u128)hi(x.w[3], y.w[3]);
  c5 += c4 >> 64;
  c6 += c5 >> 64;
  c7 += c6 >> 64;
  QF r;
  r.m.w[0] = (unsigned long long)c4;
  r.m.w[1] = (unsigned long long)c5;
  r.m.w[2] = (unsigned long long)c6;
  r.m.w[3] = (unsigned long long)c7;
  // |x|, |y| < 2^253: the product is below 2^250 here; three bits up
  r.m = q_shl_small(r.m, 3);
  r.e = (a.e == kQFZeroE || b.e == kQFZeroE) ? kQFZeroE : a.e + b.e + 256 - 3;
  if (na != nb) r.m = fix_neg<4>(r.m);
  return r;
}

__device__ __forceinline__ QF qf_neg(const QF &a) { return {fix_neg<4>(a.m), a.e}; }

// the sum of T fixed-point values (each |m| < 2^253), aligned to a common
// scale with 2 + log2(T) bits of headroom, rounded to QD
template <int T>
__device__ __forceinline__ qd qf_sum_to_qd(const QF (&v)[T]) {
  int emax = kQFZeroE;
#pragma unroll
  for (int i = 0; i < T; ++i) emax = max(emax, v[i].e);
  if (emax == kQFZeroE) return QD::zero();
  constexpr int head = T <= 2 ? 1 : T <= 4 ? 2 : T <= 8 ? 3 : 4;
  const int base = emax + head;                  // the largest term's top bit at 252 - head
  Q256 acc = q_zero();
#pragma unroll
  for (int i = 0; i < T; ++i) {
    if (v[i].e == kQFZeroE) continue;
    acc = fix_add<4>(acc, q_sar(v[i].m, base - v[i].e));
  }
  qd r;
  fix_round4(acc, base, r.x);
  return r;
}

// a - ar b + sg ai c (one part of a complex QD update), in fixed point
__device__ __forceinline__ qd qf_upd(const qd &a, const qd &ar, const qd &b, const qd &ai,
                                     const qd &c, double sg) {
  bool bad = false;
  const QF A = qf_from(a, &bad);
  const QF p1 = qf_mul(qf_from(ar, &bad), qf_from(b, &bad));
  QF p2 = qf_mul(qf_from(ai, &bad), qf_from(c, &bad));
  if (sg < 0) p2 = qf_neg(p2);
  if (bad) return {{a.x[0] - ar.x[0] * b.x[0] + sg * ai.x[0] * c.x[0], 0.0, 0.0, 0.0}};
  const QF t[3] = {A, qf_neg(p1), p2};
  return qf_sum_to_qd<3>(t);
}

// acc += x1 y1 + sg x2 y2 for QD values, the products in 256-bit fixed point
// aligned to the accumulator's last-bit weight 2^base (every product's
// magnitude is below 2^(base + 252 - lg) by the caller's bound)
__device__ __forceinline__ void qf_dot2(Q256 &acc, const qd &x1, const qd &y1, const qd &x2,
                                       const qd &y2, double sg, int base, bool *bad) {
  const QF p1 = qf_mul(qf_from(x1, bad), qf_from(y1, bad));
  QF p2 = qf_mul(qf_from(x2, bad), qf_from(y2, bad));
  if (sg < 0) p2 = qf_neg(p2);
  if (p1.e != kQFZeroE) acc = fix_add<4>(acc, q_sar(p1.m, base - p1.e));
  if (p2.e != kQFZeroE) acc = fix_add<4>(acc, q_sar(p2.m, base - p2.e));
}

__device__ __forceinline__ Q256 q_shfl_xor(const Q256 &a, int m) {
  Q256 r;
#pragma unroll
  for (int q = 0; q < 4; ++q) r.w[q] = __shfl_xor_sync(0xffffffffu, a.w[q], m);
  return r;
}

// a - ar b + sg ai c with ar, ai already in fixed point (abad: either was not
// finite); a non-finite input gives NaN
__device__ __forceinline__ qd qf_upd2(const qd &a, const QF &ar, const qd &b, const QF &ai,
                                      const qd &c, double sg, bool abad) {
  bool bad = abad;
  const QF A = qf_from(a, &bad);
  const QF p1 = qf_mul(ar, qf_from(b, &bad));
  QF p2 = qf_mul(ai, qf_from(c, &bad));
  if (sg < 0) p2 = qf_neg(p2);
  if (bad) return {{__longlong_as_double(0x7ff8000000000000ll), 0.0, 0.0, 0.0}};
  const QF t[3] = {A, qf_neg(p1), p2};
  return qf_sum_to_qd<3>(t);
}

// qf_dot2 with x1, x2 already in fixed point
__device__ __forceinline__ void qf_dot2c(Q256 &acc, const QF &x1, const qd &y1, const QF &x2,
                                        const qd &y2, double sg, int base, bool *bad) {
  const QF p1 = qf_mul(x1, qf_from(y1, bad));
  QF p2 = qf_mul(x2, qf_from(y2, bad));
  if (sg < 0) p2 = qf_neg(p2);
  if (p1.e != kQFZeroE) acc = fix_add<4>(acc, q_sar(p1.m, base - p1.e));
  if (p2.e != kQFZeroE) acc = fix_add<4>(acc, q_sar(p2.m, base - p2.e));
}

// qf_upd2 with b, c already in fixed point
__device__ __forceinline__ qd qf_upd3(const qd &a, const QF &ar, const QF &b, const QF &ai,
                                      const QF &c, double sg, bool abad) {
  bool bad = abad;
  const QF A = qf_from(a, &bad);
  const QF p1 = qf_mul(ar, b);
  QF p2 = qf_mul(ai, c);
  if (sg < 0) p2 = qf_neg(p2);
  if (bad) return {{__longlong_as_double(0x7ff8000000000000ll), 0.0, 0.0, 0.0}};
  const QF t[3] = {A, qf_neg(p1), p2};
  return qf_sum_to_qd<3>(t);
}

// The complex product a b of QD values in fixed point: the four real parts
// converted once, four products of their top words, each part's two products
// summed exactly and rounded to four limbs.  A non-finite part falls back to
// the FP64 form (which propagates it).
__device__ __forceinline__ cx<QD> qf_cmul(const cx<QD> &a, const cx<QD> &b) {
  bool bad = false;
  const QF ar = qf_from(a.re, &bad), ai = qf_from(a.im, &bad);
  const QF br = qf_from(b.re, &bad), bi = qf_from(b.im, &bad);
  if (bad) return cops<QD>::mul(a, b);
  const QF re[2] = {qf_mul(ar, br), qf_neg(qf_mul(ai, bi))};
  const QF im[2] = {qf_mul(ar, bi), qf_mul(ai, br)};
  return {qf_sum_to_qd<2>(re), qf_sum_to_qd<2>(im)};
}

}  // namespace ph
