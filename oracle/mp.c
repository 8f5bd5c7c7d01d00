/*
 * mp.c -- the oracle's real and complex arithmetic in L = 2 (double-double)
 * or L = 4 (quad-double) limbs.  TEST INFRASTRUCTURE: see oracle.h.
 *
 * The paper computes in complex double double and quad double (Section 3.1,
 * "three modes"), taking the arithmetic from the QD library (Introduction).
 * This file does not follow any particular double-double or quad-double
 * algorithm.  It uses only two error-free transformations of IEEE doubles:
 *   two_sum  (Knuth):  a + b = s + e exactly, s = fl(a + b);
 *   two_prod (FMA):    a * b = p + e exactly, p = fl(a * b);
 * so every sum or product of multi-limb numbers becomes a short list of doubles
 * whose exact sum is the exact result.  orc_round_sum then rounds that exact
 * sum once to L limbs.  Division is long division with exact remainders and
 * square roots are Newton's iteration, both on top of those operations.
 *
 * Must be compiled with -ffp-contract=off: a fused a*b+c would break two_sum.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define MAXTERMS 96

void orc_two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  *s = x;
  *e = (a - av) + (b - bv);
}

void orc_two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *p = x;
  *e = fma(a, b, -x);
}

/* Sort by decreasing magnitude (insertion sort; lists are short). */
static void sort_mag(double *a, int k) {
  for (int i = 1; i < k; i++) {
    double v = a[i];
    int j = i - 1;
    while (j >= 0 && fabs(a[j]) < fabs(v)) { a[j + 1] = a[j]; j--; }
    a[j + 1] = v;
  }
}

static int drop_zeros(double *a, int k) {
  int m = 0;
  for (int i = 0; i < k; i++) if (a[i] != 0.0) a[m++] = a[i];
  return m;
}

/* Distillation: repeat { sort by magnitude; sweep two_sum from the smallest
   term upwards } until a sweep changes nothing.  Every two_sum is exact, so
   the sum of the list never changes.  At the fixed point fl(a[i] + a[i+1]) ==
   a[i] for all i, i.e. |a[i+1]| <= ulp(a[i])/2: a nonoverlapping expansion. */
static int distill(double *a, int k) {
  k = drop_zeros(a, k);
  for (int pass = 0; pass < 4 * k + 8; pass++) {
    sort_mag(a, k);
    int changed = 0;
    for (int i = k - 2; i >= 0; i--) {
      double s, e;
      orc_two_sum(a[i], a[i + 1], &s, &e);
      if (s != a[i] || e != a[i + 1]) changed = 1;
      a[i] = s;
      a[i + 1] = e;
    }
    k = drop_zeros(a, k);
    if (!changed) break;
  }
  return k;
}

/* Round the exact sum of m doubles to L limbs (leading limb first, each limb
   at most half an ulp of the one before it).  Relative error ~2^(-53 L). */
void orc_round_sum(const double *in, int m, int L, double *out) {
  double a[MAXTERMS];
  int k = 0;
  for (int i = 0; i < m && k < MAXTERMS; i++) a[k++] = in[i];
  k = distill(a, k);
  if (k <= L) {
    for (int i = 0; i < L; i++) out[i] = i < k ? a[i] : 0.0;
    return;
  }
  /* the tail below limb L-1 is smaller than half an ulp of a[L-1] */
  double tail = 0.0;
  for (int i = k - 1; i >= L; i--) tail += a[i];
  double o[ORC_MAXL + 1];
  for (int i = 0; i < L - 1; i++) o[i] = a[i];
  o[L - 1] = a[L - 1] + tail;
  int kk = distill(o, L);
  for (int i = 0; i < L; i++) out[i] = i < kk ? o[i] : 0.0;
}

/* ---- reals ---------------------------------------------------------------- */

orc_real orc_r_from(double d) {
  orc_real r;
  memset(&r, 0, sizeof r);
  r.v[0] = d;
  return r;
}

orc_real orc_r_neg(int L, orc_real a) {
  for (int i = 0; i < L; i++) a.v[i] = -a.v[i];
  return a;
}

orc_real orc_r_add(int L, orc_real a, orc_real b) {
  double t[2 * ORC_MAXL];
  orc_real z;
  memset(&z, 0, sizeof z);
  for (int i = 0; i < L; i++) { t[i] = a.v[i]; t[L + i] = b.v[i]; }
  orc_round_sum(t, 2 * L, L, z.v);
  return z;
}

orc_real orc_r_sub(int L, orc_real a, orc_real b) {
  return orc_r_add(L, a, orc_r_neg(L, b));
}

/* all L*L limb products, each split exactly into two doubles */
static int prod_terms(int L, const orc_real *a, const orc_real *b, double sign, double *t) {
  int m = 0;
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++) {
      double p, e;
      orc_two_prod(sign * a->v[i], b->v[j], &p, &e);
      t[m++] = p;
      t[m++] = e;
    }
  return m;
}

orc_real orc_r_mul(int L, orc_real a, orc_real b) {
  double t[2 * ORC_MAXL * ORC_MAXL];
  orc_real z;
  memset(&z, 0, sizeof z);
  int m = prod_terms(L, &a, &b, 1.0, t);
  orc_round_sum(t, m, L, z.v);
  return z;
}

/* Long division: quotient digits q_k = r_0 / b_0 with the exact remainder
   r := r - q_k b kept to L+2 limbs; L+1 digits, then rounded to L limbs. */
orc_real orc_r_div(int L, orc_real a, orc_real b) {
  double r[ORC_MAXL + 2], q[ORC_MAXL + 1];
  double t[3 * ORC_MAXL + 4];
  orc_real z;
  memset(&z, 0, sizeof z);
  for (int i = 0; i < L + 2; i++) r[i] = i < L ? a.v[i] : 0.0;
  for (int kq = 0; kq <= L; kq++) {
    q[kq] = r[0] / b.v[0];
    int m = 0;
    for (int i = 0; i < L + 2; i++) t[m++] = r[i];
    for (int j = 0; j < L; j++) {
      double p, e;
      orc_two_prod(-q[kq], b.v[j], &p, &e);
      t[m++] = p;
      t[m++] = e;
    }
    orc_round_sum(t, m, L + 2, r);
  }
  orc_round_sum(q, L + 1, L, z.v);
  return z;
}

/* Newton's iteration s := s + (a - s^2) / (2 s) from the double square root;
   each step doubles the number of correct bits (53, 106, 212, 424). */
orc_real orc_r_sqrt(int L, orc_real a) {
  if (a.v[0] <= 0.0) return orc_r_from(0.0);
  /* one limb: IEEE 754 requires sqrt correctly rounded, which is the exact
     root rounded once; Newton steps in rounded doubles could move it */
  if (L == 1) return orc_r_from(sqrt(a.v[0]));
  orc_real s = orc_r_from(sqrt(a.v[0]));
  for (int it = 0; it < 3; it++) {
    orc_real res = orc_r_sub(L, a, orc_r_mul(L, s, s));
    orc_real two_s = orc_r_add(L, s, s);
    s = orc_r_add(L, s, orc_r_div(L, res, two_s));
  }
  return s;
}

/* ---- complex --------------------------------------------------------------- */

orc_cplx orc_c_add(int L, orc_cplx a, orc_cplx b) {
  orc_cplx z;
  z.re = orc_r_add(L, a.re, b.re);
  z.im = orc_r_add(L, a.im, b.im);
  return z;
}

orc_cplx orc_c_sub(int L, orc_cplx a, orc_cplx b) {
  orc_cplx z;
  z.re = orc_r_sub(L, a.re, b.re);
  z.im = orc_r_sub(L, a.im, b.im);
  return z;
}

/* (ar + i ai)(br + i bi): both parts of the four-product form are summed
   exactly and rounded once. */
orc_cplx orc_c_mul(int L, orc_cplx a, orc_cplx b) {
  double t[4 * ORC_MAXL * ORC_MAXL];
  orc_cplx z;
  memset(&z, 0, sizeof z);
  int m = prod_terms(L, &a.re, &b.re, 1.0, t);
  m += prod_terms(L, &a.im, &b.im, -1.0, t + m);
  orc_round_sum(t, m, L, z.re.v);
  m = prod_terms(L, &a.re, &b.im, 1.0, t);
  m += prod_terms(L, &a.im, &b.re, 1.0, t + m);
  orc_round_sum(t, m, L, z.im.v);
  return z;
}

orc_cplx orc_c_conj_mul(int L, orc_cplx a, orc_cplx b) {
  orc_cplx ac = a;
  ac.im = orc_r_neg(L, a.im);
  return orc_c_mul(L, ac, b);
}

orc_cplx orc_c_mul_real(int L, orc_cplx a, orc_real r) {
  orc_cplx z;
  z.re = orc_r_mul(L, a.re, r);
  z.im = orc_r_mul(L, a.im, r);
  return z;
}

orc_cplx orc_c_div_real(int L, orc_cplx a, orc_real r) {
  orc_cplx z;
  z.re = orc_r_div(L, a.re, r);
  z.im = orc_r_div(L, a.im, r);
  return z;
}

orc_real orc_c_abs2(int L, orc_cplx a) {
  double t[4 * ORC_MAXL * ORC_MAXL];
  orc_real z;
  memset(&z, 0, sizeof z);
  int m = prod_terms(L, &a.re, &a.re, 1.0, t);
  m += prod_terms(L, &a.im, &a.im, 1.0, t + m);
  orc_round_sum(t, m, L, z.v);
  return z;
}

/* The norms that steer Newton's method are taken in plain double from the
   leading limbs (Section 3.1: only their magnitude matters). */
double orc_c_mag_d(orc_cplx a) {
  double re = a.re.v[0], im = a.im.v[0];
  return sqrt(re * re + im * im);
}

orc_cplx orc_c_load(int L, const double *v, long stride, long i) {
  orc_cplx z;
  memset(&z, 0, sizeof z);
  for (int l = 0; l < L; l++) {
    z.re.v[l] = v[(2 * l) * stride + i];
    z.im.v[l] = v[(2 * l + 1) * stride + i];
  }
  return z;
}

void orc_c_store(int L, double *v, long stride, long i, orc_cplx z) {
  for (int l = 0; l < L; l++) {
    v[(2 * l) * stride + i] = z.re.v[l];
    v[(2 * l + 1) * stride + i] = z.im.v[l];
  }
}

/* ---- vectorised pins -------------------------------------------------------
   real ops on arrays [L][count]:  0 add, 1 sub, 2 mul, 3 div, 4 sqrt(x),
   5 two_sum (L=2 out: s,e of x0,y0), 6 two_prod;
   complex ops on [L][2][count]:   0 add, 1 sub, 2 mul, 3 conj_mul, 4 abs2
   (abs2 writes a real [L][count]). */
int orc_vec_real(int op, int L, int count, const double *x, const double *y, double *z) {
  if (L != 1 && L != 2 && L != 4) return ORC_EINVAL;
  for (int i = 0; i < count; i++) {
    orc_real a, b, c;
    memset(&a, 0, sizeof a);
    memset(&b, 0, sizeof b);
    for (int l = 0; l < L; l++) {
      a.v[l] = x[(long)l * count + i];
      b.v[l] = y ? y[(long)l * count + i] : 0.0;
    }
    memset(&c, 0, sizeof c);
    switch (op) {
      case 0: c = orc_r_add(L, a, b); break;
      case 1: c = orc_r_sub(L, a, b); break;
      case 2: c = orc_r_mul(L, a, b); break;
      case 3: c = orc_r_div(L, a, b); break;
      case 4: c = orc_r_sqrt(L, a); break;
      case 5: orc_two_sum(a.v[0], b.v[0], &c.v[0], &c.v[1]); break;
      case 6: orc_two_prod(a.v[0], b.v[0], &c.v[0], &c.v[1]); break;
      default: return ORC_EINVAL;
    }
    for (int l = 0; l < L; l++) z[(long)l * count + i] = c.v[l];
  }
  return ORC_OK;
}

int orc_vec_cplx(int op, int L, int count, const double *x, const double *y, double *z) {
  if (L != 1 && L != 2 && L != 4) return ORC_EINVAL;
  for (int i = 0; i < count; i++) {
    orc_cplx a = orc_c_load(L, x, count, i), b, c;
    if (y) b = orc_c_load(L, y, count, i); else memset(&b, 0, sizeof b);
    switch (op) {
      case 0: c = orc_c_add(L, a, b); break;
      case 1: c = orc_c_sub(L, a, b); break;
      case 2: c = orc_c_mul(L, a, b); break;
      case 3: c = orc_c_conj_mul(L, a, b); break;
      case 4: {
        orc_real r = orc_c_abs2(L, a);
        for (int l = 0; l < L; l++) z[(long)l * count + i] = r.v[l];
        continue;
      }
      default: return ORC_EINVAL;
    }
    orc_c_store(L, z, count, i, c);
  }
  return ORC_OK;
}
