// exsum.cuh -- exact sums of double-double / quad-double values across the 32
// lanes of a warp, in fixed-point integer arithmetic.
//
// On GB300 an FP64 instruction occupies its SM sub-partition for ~64 cycles,
// while 32-bit integer multiply-adds run at about 30x the rate with a latency
// of a few cycles (measured: 600 G DFMA/s against 18.9 T IMAD/s on this GPU).
// A five-level shuffle tree of DD additions (8 FP64 instructions a level) or
// QD additions (94) sits on the critical chain of every MGS pivot.  Here the
// lanes agree on the exponent e of the last bit of the largest leading limb
// (one integer max-reduction; that limb is below 2^(e + 53)), each lane writes
// its value as a two's-complement integer of W 64-bit words whose last bit
// weighs 2^(e + 59 - 64 W) (the top word keeps room for the sum of 32 values
// and the sign), the integers are added along a shuffle tree with carries
// (integer instructions only), and the total is rounded back to L limbs, each
// the nearest double to what remains: the correctly rounded multi-limb value
// of the exact sum of the truncated inputs.  W = 2 for DD (each input
// truncated below 2^(e - 69): with 32 inputs, an error under 2^-116 of the
// largest term, below double-double's 2^-104) and W = 4 for QD (2^-244
// against 2^-208).
//
// Zero inputs add nothing; a non-finite input makes every lane's result NaN;
// results below the normal range of a double are flushed to zero.  Every lane
// of the warp must call (full-mask shuffles) and every lane gets the total.
//
// The second half of the file holds the double-double forms of the
// throughput-bound kernels: a dot-product term or an update split into exact
// products and cross products (8 FP64 instructions) whose terms are summed as
// 128-bit integers and rounded back to two limbs.
#pragma once
#include "mp.cuh"

namespace ph {

template <int W> struct Fix { unsigned long long w[W]; };

// |m| * 2^s as W words (m < 2^53), truncated toward zero
template <int W>
__device__ __forceinline__ Fix<W> fix_place(unsigned long long m, int s) {
  Fix<W> r;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    const int sh = s - 64 * q;
    unsigned long long v = 0;
    if (sh >= 0) v = sh < 64 ? (m << sh) : 0ull;
    else v = -sh < 64 ? (m >> (-sh)) : 0ull;
    r.w[q] = v;
  }
  return r;
}

template <int W>
__device__ __forceinline__ Fix<W> fix_add(const Fix<W> &a, const Fix<W> &b) {
  Fix<W> r;
  asm("add.cc.u64 %0, %1, %2;" : "=l"(r.w[0]) : "l"(a.w[0]), "l"(b.w[0]));
#pragma unroll
  for (int q = 1; q < W - 1; ++q)
    asm("addc.cc.u64 %0, %1, %2;" : "=l"(r.w[q]) : "l"(a.w[q]), "l"(b.w[q]));
  asm("addc.u64 %0, %1, %2;" : "=l"(r.w[W - 1]) : "l"(a.w[W - 1]), "l"(b.w[W - 1]));
  return r;
}

template <int W>
__device__ __forceinline__ Fix<W> fix_neg(const Fix<W> &a) {
  Fix<W> z, n;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    z.w[q] = 0ull;
    n.w[q] = ~a.w[q];
  }
  z.w[0] = 1ull;
  return fix_add<W>(n, z);
}

template <int W>
__device__ __forceinline__ bool fix_negative(const Fix<W> &a) {
  return (long long)a.w[W - 1] < 0;
}

// the fields of a double: sign, 53-bit integer significand, unbiased exponent
// of its last bit (value = (-1)^sign m 2^e); zero and subnormals give m = 0
__device__ __forceinline__ void dbl_fields(double d, int &sign, unsigned long long &m, int &e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  sign = (int)(b >> 63);
  const int ef = (int)((b >> 52) & 0x7ff);
  m = ef == 0 ? 0ull : ((b & 0xfffffffffffffull) | (1ull << 52));
  e = ef - 1075;
}

// adds one double into the accumulator whose last bit weighs 2^base
template <int W>
__device__ __forceinline__ void fix_acc_double(Fix<W> &acc, double d, int base) {
  int sg, e;
  unsigned long long m;
  dbl_fields(d, sg, m, e);
  if (m == 0) return;
  Fix<W> t = fix_place<W>(m, e - base);
  if (sg) t = fix_neg<W>(t);
  acc = fix_add<W>(acc, t);
}

// position of the highest set bit of a non-negative accumulator, -1 if zero
template <int W>
__device__ __forceinline__ int fix_top(const Fix<W> &a) {
#pragma unroll
  for (int q = W - 1; q >= 0; --q)
    if (a.w[q]) return 64 * q + 63 - __clzll((long long)a.w[q]);
  return -1;
}

// bits [lo, lo + 64) of a non-negative accumulator (lo may be negative)
template <int W>
__device__ __forceinline__ unsigned long long fix_bits(const Fix<W> &a, int lo) {
  unsigned long long r = 0;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    const int sh = 64 * q - lo;                    // where word q's bit 0 lands
    if (sh >= 64 || sh <= -64) continue;
    r |= sh >= 0 ? (a.w[q] << sh) : (a.w[q] >> (-sh));
  }
  return r;
}

// the double nearest to the signed accumulator (last bit 2^base), and the
// accumulator minus that double (exact)
template <int W>
__device__ __forceinline__ double fix_round_off(Fix<W> &acc, int base) {
  const bool neg = fix_negative<W>(acc);
  Fix<W> a = neg ? fix_neg<W>(acc) : acc;
  const int p = fix_top<W>(a);
  if (p < 0) return 0.0;
  unsigned long long m;
  int lsb = p - 52;                                // weight of the significand's last bit
  if (lsb <= 0) {
    m = fix_bits<W>(a, 0);                         // the whole value fits in 53 bits
    lsb = 0;
  } else {
    m = fix_bits<W>(a, lsb) & ((1ull << 53) - 1);
    const unsigned long long half = fix_bits<W>(a, lsb - 1) & 1ull;
    bool sticky = false;
    if (half) {                                    // below-half bits decide ties
      const int rest = lsb - 1;
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const int lo = 64 * q, hi = lo + 64;
        if (lo >= rest) break;
        unsigned long long mask = hi <= rest ? ~0ull : ((1ull << (rest - lo)) - 1);
        if (a.w[q] & mask) sticky = true;
      }
    }
    if (half && (sticky || (m & 1ull))) {
      m += 1;
      if (m >> 53) {                               // carried into a new bit
        m >>= 1;
        lsb += 1;
      }
    }
  }
  const int e = lsb + base;                        // value = m 2^e
  // build the double (normal range only; below it, zero)
  double d = 0.0;
  int top = 63 - __clzll((long long)m);            // m may have fewer than 53 bits
  const int ex = e + top;                          // unbiased exponent
  if (m != 0 && ex >= -1022 && ex <= 1023) {
    const unsigned long long mant = (m << (52 - top)) & 0xfffffffffffffull;
    const unsigned long long bits = ((unsigned long long)(ex + 1023) << 52) | mant;
    d = __longlong_as_double((long long)bits);
  } else if (m != 0 && ex > 1023) {
    d = __longlong_as_double(0x7ff0000000000000ll);
  }
  // subtract the rounded value: acc -= sign * m 2^(lsb)
  Fix<W> t = fix_place<W>(m, lsb);
  if (!neg) t = fix_neg<W>(t);
  acc = fix_add<W>(acc, t);
  return neg ? -d : d;
}

// The double m 2^E for a significand with its top bit at bit 52 (or m = 2^53
// after rounding up, handled by the caller); zero below the normal range,
// infinity above it.
__device__ __forceinline__ double fix_make_double(unsigned long long m, int E) {
  const int ex = E + 52;                           // unbiased exponent
  if (ex > 1023) return __longlong_as_double(0x7ff0000000000000ll);
  if (ex < -1022) return 0.0;
  return __longlong_as_double(
      (long long)(((unsigned long long)(ex + 1023) << 52) | (m & 0xfffffffffffffull)));
}

// A non-zero 128-bit magnitude (h, l) shifted left by lz = its leading zeros
// (n1, n0), the 53 leading bits m, whether round-to-nearest-even rounds m up,
// and the 11 bits of n1 below m.
__device__ __forceinline__ void fix_norm128(unsigned long long h, unsigned long long l, int &lz,
                                            unsigned long long &m, bool &up,
                                            unsigned long long &r, unsigned long long &n0) {
  lz = h ? __clzll((long long)h) : 64 + __clzll((long long)l);
  unsigned long long n1;
  if (lz >= 64) {
    n1 = l << (lz - 64);
    n0 = 0ull;
  } else if (lz == 0) {
    n1 = h;
    n0 = l;
  } else {
    n1 = (h << lz) | (l >> (64 - lz));
    n0 = l << lz;
  }
  m = n1 >> 11;
  r = n1 & 0x7ffull;
  up = (r & 0x400ull) && ((r & 0x3ffull) || n0 || (m & 1ull));
}

// Two limbs from a two-word accumulator (last bit 2^base) in straight-line
// code: v0 the double nearest to it, v1 the double nearest to what remains
// (the same values as two fix_round_off<2> calls).
__device__ __forceinline__ void fix_round2(const Fix<2> &acc, int base, double &v0, double &v1) {
  unsigned long long h = acc.w[1], l = acc.w[0];
  const bool neg = (long long)h < 0;
  if (neg) {                                       // magnitude of the two's complement value
    l = ~l + 1ull;
    h = ~h + (l == 0ull ? 1ull : 0ull);
  }
  v0 = v1 = 0.0;
  if ((h | l) == 0ull) return;
  int lz;
  unsigned long long m, r, n0;
  bool up;
  fix_norm128(h, l, lz, m, up, r, n0);
  const int e = 127 - lz - 52 + base;              // weight of m's last bit
  const unsigned long long mu = m + (up ? 1ull : 0ull);
  v0 = (mu >> 53) ? fix_make_double(1ull << 52, e + 1) : fix_make_double(mu, e);
  // what remains, in the normalised frame: (r - 2^11 up) 2^64 + n0, signed
  long long R1 = (long long)r - (up ? 0x800ll : 0ll);
  unsigned long long R0 = n0;
  const bool rneg = R1 < 0;
  if (rneg) {
    R0 = ~R0 + 1ull;
    R1 = ~R1 + (R0 == 0ull ? 1ll : 0ll);
  }
  if ((R1 | (long long)R0) != 0) {
    int lz2;
    unsigned long long m2, r2, n02;
    bool up2;
    fix_norm128((unsigned long long)R1, R0, lz2, m2, up2, r2, n02);
    // bit 127 of the normalised frame weighs 2^(127 - lz + base); the
    // remainder's frame is that one shifted by 64 + lz bits
    const int e2 = 127 - lz2 - 52 + base - lz;
    const unsigned long long mu2 = m2 + (up2 ? 1ull : 0ull);
    v1 = (mu2 >> 53) ? fix_make_double(1ull << 52, e2 + 1) : fix_make_double(mu2, e2);
    if (rneg) v1 = -v1;
  }
  if (neg) {
    v0 = -v0;
    v1 = -v1;
  }
}

// leading zeros of a 256-bit magnitude (256 for zero)
__device__ __forceinline__ int fix_clz4(const Fix<4> &a) {
  return a.w[3] ? __clzll((long long)a.w[3])
       : a.w[2] ? 64 + __clzll((long long)a.w[2])
       : a.w[1] ? 128 + __clzll((long long)a.w[1])
       : a.w[0] ? 192 + __clzll((long long)a.w[0]) : 256;
}

// a 2^s for 0 <= s < 256 (bits above 255 dropped), by selects
__device__ __forceinline__ Fix<4> fix_shl4(const Fix<4> &a, int s) {
  const int ws = s >> 6, bs = s & 63;
  Fix<4> r;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    // words q - ws and q - ws - 1 of a (zero below word 0)
    unsigned long long hi = 0ull, lo = 0ull;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (q - k >= 0 && ws == k) hi = a.w[q - k];
      if (q - k - 1 >= 0 && ws == k) lo = a.w[q - k - 1];
    }
    r.w[q] = bs ? (hi << bs) | (lo >> (64 - bs)) : hi;
  }
  return r;
}

// Four limbs from a four-word accumulator (last bit 2^base) in straight-line
// code: each limb the double nearest to what the previous limbs leave (the
// same values as four fix_round_off<4> calls).  Each step normalises the
// remainder so that its top bit is bit 255, takes the 53 bits below it,
// rounds to nearest even on the 203 bits under them, and keeps the signed
// remainder in the same frame.
__device__ __forceinline__ void fix_round4(const Fix<4> &acc, int base, double (&v)[4]) {
  Fix<4> a = acc;
#pragma unroll
  for (int l = 0; l < 4; ++l) v[l] = 0.0;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const bool neg = (long long)a.w[3] < 0;
    const Fix<4> mag = neg ? fix_neg<4>(a) : a;
    const int lz = fix_clz4(mag);
    if (lz == 256) break;
    Fix<4> n = fix_shl4(mag, lz);
    const unsigned long long m = n.w[3] >> 11, r = n.w[3] & 0x7ffull;
    const bool sticky = (r & 0x3ffull) || n.w[2] || n.w[1] || n.w[0];
    const bool up = (r & 0x400ull) && (sticky || (m & 1ull));
    const int e = base - lz + 203;                 // weight of m's last bit
    const unsigned long long mu = m + (up ? 1ull : 0ull);
    const double d = (mu >> 53) ? fix_make_double(1ull << 52, e + 1) : fix_make_double(mu, e);
    v[l] = neg ? -d : d;
    // what remains: the 11 bits below m, less 2^11 if m was rounded up
    n.w[3] = (unsigned long long)((long long)r - (up ? 0x800ll : 0ll));
    a = neg ? fix_neg<4>(n) : n;
    base -= lz;
  }
}

template <int W, int L>
__device__ __forceinline__ void warp_exact_sum_limbs(double (&v)[L]) {
  // largest exponent of the leading limbs; any non-finite input poisons all
  int sg, e;
  unsigned long long m;
  const unsigned long long b0 = (unsigned long long)__double_as_longlong(v[0]);
  const bool bad = ((b0 >> 52) & 0x7ff) == 0x7ff;
  dbl_fields(v[0], sg, m, e);
  const int ekey = m ? e + 2048 : 0;               // non-negative for the max
  const int emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)ekey);
  const unsigned anybad = __reduce_or_sync(0xffffffffu, bad ? 1u : 0u);
  if (anybad) {
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  if (emax == 0) {                                 // every input is zero
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = 0.0;
    return;
  }
  // the largest leading limb is below 2^(E + 53); the sum of 32 values below
  // 2^(E + 58): the top word keeps 5 guard bits and the sign
  const int E = emax - 2048;
  const int base = E + 53 + 6 - 64 * W;
  Fix<W> acc;
#pragma unroll
  for (int q = 0; q < W; ++q) acc.w[q] = 0ull;
#pragma unroll
  for (int l = 0; l < L; ++l) fix_acc_double<W>(acc, v[l], base);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Fix<W> o;
#pragma unroll
    for (int q = 0; q < W; ++q) o.w[q] = __shfl_xor_sync(0xffffffffu, acc.w[q], off);
    acc = fix_add<W>(acc, o);
  }
  if constexpr (W == 2 && L == 2) {
    fix_round2(acc, base, v[0], v[1]);
  } else if constexpr (W == 4 && L == 4) {
    fix_round4(acc, base, v);
  } else {
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = fix_round_off<W>(acc, base);
  }
}

// The exact warp sum of a DD (W = 2) or QD (W = 4) value, rounded to L limbs.
__device__ __forceinline__ dd warp_exact_sum(const dd &a) {
  double v[2] = {a.h, a.l};
  warp_exact_sum_limbs<2, 2>(v);
  return {v[0], v[1]};
}

__device__ __forceinline__ qd warp_exact_sum(const qd &a) {
  double v[4] = {a.x[0], a.x[1], a.x[2], a.x[3]};
  warp_exact_sum_limbs<4, 4>(v);
  return {{v[0], v[1], v[2], v[3]}};
}

// ------------------------------------------------ double-double in fixed point
// Throughput forms of the DD dot-product and update steps, for kernels with
// enough warps to hide integer latency (measured on this GPU at 16 warps per
// SM: a DD update a - x y + u v costs 27 FP64 instructions in the FP64 form
// and 8 here, and runs 2.1x as fast; with one warp its latency is higher, so
// latency-bound kernels keep the FP64 form).  Each product of leading limbs is
// split exactly (two_prod), the cross products of a leading and a trailing
// limb are summed in double, and all terms are added exactly as 128-bit
// two's-complement integers with a common last-bit weight 2^base; the total is
// rounded back to two limbs (fix_round2).

typedef unsigned __int128 fx128;

// Biased exponent field of a double: 0 for zero and subnormals, 2047 for inf
// and NaN; a double with field f is below 2^(f - 1022) in magnitude.
__device__ __forceinline__ unsigned dbl_ef(double d) {
  return (unsigned)((unsigned long long)__double_as_longlong(d) >> 52) & 0x7ffu;
}

// Last-bit weight of a 128-bit accumulator for terms below 2^(key - 1022) in
// magnitude whose sum is below 2^lg times that bound (sign bit kept free).
__device__ __forceinline__ int fx_base(int key, int lg) { return key - 1022 + lg + 1 - 128; }

// d as a signed 128-bit integer in units of 2^base, truncated toward zero
// (subnormals count as zero)
__device__ __forceinline__ fx128 fx_place(double d, int base) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int ef = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = ef ? ((b & 0xfffffffffffffull) | (1ull << 52)) : 0ull;
  const int s = ef - 1075 - base;
  fx128 v;
  if (s >= 0) v = s < 128 ? ((fx128)m << s) : (fx128)0;
  else v = s > -64 ? (fx128)(m >> (-s)) : (fx128)0;
  return (b >> 63) ? (fx128)0 - v : v;
}

__device__ __forceinline__ dd fx_round_dd(fx128 acc, int base) {
  Fix<2> f;
  f.w[0] = (unsigned long long)acc;
  f.w[1] = (unsigned long long)(acc >> 64);
  dd r;
  fix_round2(f, base, r.h, r.l);
  return r;
}

__device__ __forceinline__ fx128 fx_shfl_xor(fx128 a, int m) {
  const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)a, m);
  const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(a >> 64), m);
  return ((fx128)hi << 64) | lo;
}

// sum over the warp (every lane gets it)
__device__ __forceinline__ fx128 fx_warp_sum(fx128 a) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) a += fx_shfl_xor(a, m);
  return a;
}

// acc += x1 y1 + sg x2 y2 (sg = +-1) in units of 2^base: the exact leading
// products and the four cross products (8 FP64 instructions)
__device__ __forceinline__ void fx_dot2(fx128 &acc, const dd &x1, const dd &y1, const dd &x2,
                                        const dd &y2, double sg, int base) {
  const double x2h = sg * x2.h, x2l = sg * x2.l;
  double p1, e1, p2, e2;
  two_prod(x1.h, y1.h, p1, e1);
  two_prod(x2h, y2.h, p2, e2);
  double c = ph::fmul(x1.h, y1.l);
  c = ph::ffma(x1.l, y1.h, c);
  c = ph::ffma(x2h, y2.l, c);
  c = ph::ffma(x2l, y2.h, c);
  acc += fx_place(p1, base) + fx_place(e1, base) + fx_place(p2, base) + fx_place(e2, base) +
         fx_place(c, base);
}

// a - ar b + sg ai c (one part of a complex update), exactly summed and
// rounded to two limbs: the same value as Part<DD>::upd up to its rounding
// (this one is the nearer to the exact result)
__device__ __forceinline__ dd fx_upd(const dd &a, const dd &ar, const dd &b, const dd &ai,
                                     const dd &c, double sg) {
  const double aih = sg * ai.h, ail = sg * ai.l;
  double p1, e1, p2, e2;
  two_prod(ar.h, b.h, p1, e1);
  two_prod(aih, c.h, p2, e2);
  double x = ph::fmul(ar.h, b.l);
  x = ph::ffma(ar.l, b.h, x);
  double y = ph::fmul(aih, c.l);
  y = ph::ffma(ail, c.h, y);
  // terms added: a.h, a.l, p2, e2, y; subtracted (in the integers): p1, e1, x
  const unsigned key = max(max(max(dbl_ef(a.h), dbl_ef(a.l)), max(dbl_ef(p1), dbl_ef(e1))),
                           max(max(dbl_ef(p2), dbl_ef(e2)), max(dbl_ef(x), dbl_ef(y))));
  if (key == 0u) return {0.0, 0.0};
  if (key == 0x7ffu) return {a.h - p1 + p2, 0.0};         // inf or NaN, as the FP64 form
  const int base = fx_base((int)key, 2);                   // a.h, p1, p2: the sum is below 4x
  const fx128 acc = fx_place(a.h, base) + fx_place(a.l, base) + fx_place(p2, base) +
                    fx_place(e2, base) + fx_place(y, base) -
                    (fx_place(p1, base) + fx_place(e1, base) + fx_place(x, base));
  return fx_round_dd(acc, base);
}

}  // namespace ph
