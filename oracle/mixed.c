/*
 * mixed.c -- the oracle's mixed-precision corrector: the precision form of the
 * path tracker.  The paper's corrector works in double-double or quad-double
 * throughout (Section 3.1, Fig. 2); the
 * precision form keeps only the residual and the accumulated update in that
 * working precision and solves the Newton system in IEEE double or single.
 * TEST INFRASTRUCTURE: see oracle.h.
 *
 * One corrector iteration at (x, t), in this order:
 *   1. h = h(x, t) and its Jacobian J in working precision (orc_eval), and the
 *      paper's residual tests on max |h_i| (the same as orc_newton);
 *   2. J and -h rounded to the low precision (lin = 1: double, the leading
 *      limb; lin = 2: single, the leading limb rounded to float), -h first
 *      scaled by 2^-e with 2^e <= max |h_i| < 2^(e+1): the scaling is exact,
 *      and without it a residual below single precision's range (near 1e-38,
 *      which quad-double reaches) would round to zero;
 *   3. textbook modified Gram-Schmidt on [J | -h] in that precision (the same
 *      column order as mgs.c: r_kk = ||a_k||, q_k = a_k / r_kk, r_kj = q_k^H a_j,
 *      a_j -= r_kj q_k), then back substitution R d = Q^H(-h);
 *   4. x := x + 2^e d in working precision, and the paper's test on max |d_i|.
 * Step 3 also gives the condition estimate max_k r_kk / min_k r_kk, a lower
 * bound of the 2-norm condition number of the rounded J.
 *
 * Each low-precision operation below is one IEEE operation of that type (the
 * file is compiled without contraction, so no FMA appears).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* MGS least squares in type T on an N x (n+1) column-major complex matrix
   (separate real and imaginary arrays); on return d holds the solution and
   *cond the estimate.  Returns ORC_OK or ORC_NONFINITE. */
#define ORC_LP_MGS(T, NAME, SQRT)                                                          \
  static int NAME(int N, int n, T *ar, T *ai, double *dre, double *dim, double *cond) {   \
    int nc = n + 1;                                                                        \
    T *rr = calloc((size_t)nc * nc, sizeof(T)), *ri = calloc((size_t)nc * nc, sizeof(T)); \
    T *yr = malloc(sizeof(T) * n), *yi = malloc(sizeof(T) * n);                            \
    if (!rr || !ri || !yr || !yi) { free(rr); free(ri); free(yr); free(yi); return ORC_ENOMEM; } \
    int status = ORC_OK;                                                                   \
    T rmax = 0, rmin = 0;                                                                  \
    for (int k = 0; k < n; k++) {                                                          \
      T *kr = ar + (long)k * N, *ki = ai + (long)k * N;                                    \
      T s = 0;                                                                             \
      for (int i = 0; i < N; i++) s = s + (kr[i] * kr[i] + ki[i] * ki[i]);                 \
      T rkk = SQRT(s);                                                                     \
      if (!(rkk > 0) || !isfinite((double)rkk)) { status = ORC_NONFINITE; break; }         \
      if (k == 0 || rkk > rmax) rmax = rkk;                                                \
      if (k == 0 || rkk < rmin) rmin = rkk;                                                \
      rr[(long)k * nc + k] = rkk;                                                          \
      for (int i = 0; i < N; i++) { kr[i] = kr[i] / rkk; ki[i] = ki[i] / rkk; }            \
      for (int j = k + 1; j <= n; j++) {                                                   \
        T *jr = ar + (long)j * N, *ji = ai + (long)j * N;                                  \
        T pr = 0, pi = 0;                                                                  \
        for (int i = 0; i < N; i++) {                                                      \
          pr = pr + (kr[i] * jr[i] + ki[i] * ji[i]);                                       \
          pi = pi + (kr[i] * ji[i] - ki[i] * jr[i]);                                       \
        }                                                                                  \
        rr[(long)k * nc + j] = pr;                                                         \
        ri[(long)k * nc + j] = pi;                                                         \
        for (int i = 0; i < N; i++) {                                                      \
          T ur = pr * kr[i] - pi * ki[i], ui = pr * ki[i] + pi * kr[i];                    \
          jr[i] = jr[i] - ur;                                                              \
          ji[i] = ji[i] - ui;                                                              \
        }                                                                                  \
      }                                                                                    \
    }                                                                                      \
    if (status == ORC_OK) {                                                                \
      for (int k = n - 1; k >= 0; k--) {                                                   \
        T sr = rr[(long)k * nc + n], si = ri[(long)k * nc + n];                            \
        for (int j = k + 1; j < n; j++) {                                                  \
          T wr = rr[(long)k * nc + j], wi = ri[(long)k * nc + j];                          \
          sr = sr - (wr * yr[j] - wi * yi[j]);                                             \
          si = si - (wr * yi[j] + wi * yr[j]);                                             \
        }                                                                                  \
        yr[k] = sr / rr[(long)k * nc + k];                                                 \
        yi[k] = si / rr[(long)k * nc + k];                                                 \
      }                                                                                    \
      for (int k = 0; k < n; k++) { dre[k] = (double)yr[k]; dim[k] = (double)yi[k]; }      \
      *cond = (double)rmax / (double)rmin;                                                 \
    }                                                                                      \
    free(rr); free(ri); free(yr); free(yi);                                                \
    return status;                                                                         \
  }

ORC_LP_MGS(double, lp_mgs_d, sqrt)
ORC_LP_MGS(float, lp_mgs_f, sqrtf)

int orc_lowprec_solve(int lin, int N, int n, const double *J, const double *rhs, double *dx,
                      double *cond) {
  if ((lin != 1 && lin != 2) || n < 1 || N < n) return ORC_EINVAL;
  long NN = (long)N * n, cols = (long)N * (n + 1);
  int st;
  double c = NAN;
  if (lin == 1) {
    double *ar = malloc(sizeof(double) * cols), *ai = malloc(sizeof(double) * cols);
    if (!ar || !ai) { free(ar); free(ai); return ORC_ENOMEM; }
    for (long e = 0; e < NN; e++) { ar[e] = J[e]; ai[e] = J[NN + e]; }
    for (int i = 0; i < N; i++) { ar[NN + i] = rhs[i]; ai[NN + i] = rhs[N + i]; }
    st = lp_mgs_d(N, n, ar, ai, dx, dx + n, &c);
    free(ar); free(ai);
  } else {
    float *ar = malloc(sizeof(float) * cols), *ai = malloc(sizeof(float) * cols);
    if (!ar || !ai) { free(ar); free(ai); return ORC_ENOMEM; }
    for (long e = 0; e < NN; e++) { ar[e] = (float)J[e]; ai[e] = (float)J[NN + e]; }
    for (int i = 0; i < N; i++) { ar[NN + i] = (float)rhs[i]; ai[NN + i] = (float)rhs[N + i]; }
    st = lp_mgs_f(N, n, ar, ai, dx, dx + n, &c);
    free(ar); free(ai);
  }
  if (cond) *cond = c;
  return st;
}

/* max_i |v_i| from the leading limbs (limb 0's real plane, then its imaginary
   plane), in double, as in the paper's Max_Array (Section 3.1) */
static double max_mag_lead(const double *v, int m) {
  double r = 0.0;
  for (int i = 0; i < m; i++) {
    double a = sqrt(v[i] * v[i] + v[m + i] * v[m + i]);
    if (!(a <= r)) r = a;
  }
  return r;
}

int orc_newton_mixed(const orc_system *f, const orc_system *g, const double *gamma, int k,
                     double t, double *x, const orc_params *p, int fixed, int lin,
                     int *iters, int *updates, double *res, double *dxn, double *cond) {
  int L = f->L, N = f->N, n = f->n;
  if (lin != 1 && lin != 2) return -ORC_EINVAL;
  double *h = malloc(sizeof(double) * 2 * L * N);
  double *J = malloc(sizeof(double) * 2 * L * (size_t)N * n);
  double *jl = malloc(sizeof(double) * 2 * (size_t)N * n);
  double *rl = malloc(sizeof(double) * 2 * N);
  double *d = malloc(sizeof(double) * 2 * n);
  if (!h || !J || !jl || !rl || !d) {
    free(h); free(J); free(jl); free(rl); free(d);
    return -ORC_ENOMEM;
  }
  double tl[ORC_MAXL] = {t, 0.0, 0.0, 0.0};
  double last = p->max_res;
  int success = fixed ? 1 : 0;
  long NN = (long)N * n;
  *iters = 0;
  *updates = 0;
  for (int it = 0; it < p->max_newton; it++) {
    orc_eval(f, g, gamma, k, tl, x, h, J, p->fixed_rows);
    (*iters)++;
    /* the residual norm from the leading limbs (limb 0 re at [0][0], im at [0][1]) */
    double r = max_mag_lead(h, N);
    *res = r;
    if (!fixed) {
      if (!isfinite(r) || r > last) break;
      if (r < orc_tol_res(p, t)) { success = 1; break; }
    }
    /* leading limbs: J is [limb][re|im][NN], h is [limb][re|im][N] */
    memcpy(jl, J, sizeof(double) * 2 * NN);
    int e = (r > 0.0 && isfinite(r)) ? ilogb(r) : 0;
    for (int i = 0; i < N; i++) { rl[i] = -ldexp(h[i], -e); rl[N + i] = -ldexp(h[N + i], -e); }
    double c = NAN;
    int st = orc_lowprec_solve(lin, N, n, jl, rl, d, &c);
    if (cond) *cond = c;
    if (st != ORC_OK) {
      if (!fixed) break;
      for (int e = 0; e < 2 * n; e++) d[e] = NAN;
    }
    for (int q = 0; q < 2 * n; q++) d[q] = ldexp(d[q], e);
    double dm = max_mag_lead(d, n);
    *dxn = dm;
    for (int i = 0; i < n; i++) {
      orc_cplx di;
      memset(&di, 0, sizeof di);
      di.re.v[0] = d[i];
      di.im.v[0] = d[n + i];
      orc_c_store(L, x, n, i, orc_c_add(L, orc_c_load(L, x, n, i), di));
    }
    (*updates)++;
    if (!fixed) {
      if (!isfinite(dm)) break;
      if (dm < orc_tol_dx(p, t)) { success = 1; break; }
    }
    last = r;
  }
  free(h); free(J); free(jl); free(rl); free(d);
  return success;
}

/* Whether three successive update norms d2, d1, d0 contract (both ratios
   below 1) more slowly than quadratically (d0/d1 > (d1/d2)^1.5). */
static int contracts_linearly(double d2, double d1, double d0) {
  if (!(d2 > 0.0) || !(d1 > 0.0) || !(d0 >= 0.0) || !isfinite(d0)) return 0;
  double r1 = d1 / d2, r0 = d0 / d1;
  return r1 < 1.0 && r0 < 1.0 && r0 > r1 * sqrt(r1);
}

/* One step's corrector of the precision form with the signals the step
   control needs (the rules stated in oracle.h at orc_track_mixed). */
int orc_corrector_mixed(const orc_system *f, const orc_system *g, const double *gamma, int k,
                        double t, double *x, const orc_params *p, int fixed, int lin,
                        orc_mixed_out *o) {
  int L = f->L, N = f->N, n = f->n;
  memset(o, 0, sizeof *o);
  o->res = o->dxn = NAN;
  o->cond = INFINITY;
  if (lin != 1) return -ORC_EINVAL;
  double *h = malloc(sizeof(double) * 2 * L * N);
  double *J = malloc(sizeof(double) * 2 * L * (size_t)N * n);
  double *jl = malloc(sizeof(double) * 2 * (size_t)N * n);
  double *rl = malloc(sizeof(double) * 2 * N);
  double *d = malloc(sizeof(double) * 2 * n);
  if (!h || !J || !jl || !rl || !d) {
    free(h); free(J); free(jl); free(rl); free(d);
    return -ORC_ENOMEM;
  }
  const double u_lin = ldexp(1.0, -53);
  double tl[ORC_MAXL] = {t, 0.0, 0.0, 0.0};
  double last = p->max_res, d1 = NAN, d2 = NAN;
  int success = fixed ? 1 : 0;
  int max_it = fixed ? p->max_newton : p->max_newton + 1;
  long NN = (long)N * n;
  for (int it = 0; it < max_it; it++) {
    orc_eval(f, g, gamma, k, tl, x, h, J, p->fixed_rows);
    o->iters++;
    double r = max_mag_lead(h, N);
    o->res = r;
    if (!fixed) {
      if (!isfinite(r) || r > last) { success = 0; break; }
      if (r < orc_tol_res(p, t)) { success = 1; break; }
    }
    memcpy(jl, J, sizeof(double) * 2 * NN);
    int e = (r > 0.0 && isfinite(r)) ? ilogb(r) : 0;
    for (int i = 0; i < N; i++) { rl[i] = -ldexp(h[i], -e); rl[N + i] = -ldexp(h[N + i], -e); }
    double c = NAN;
    int st = orc_lowprec_solve(lin, N, n, jl, rl, d, &c);
    o->solves++;
    o->cond = st == ORC_OK ? c : INFINITY;
    if (!(o->cond * u_lin <= 1e-6)) o->escalate = 2;   /* kappa u_low above the threshold */
    if (st != ORC_OK) {
      if (!fixed) { success = 0; break; }
      for (int q = 0; q < 2 * n; q++) d[q] = NAN;
    }
    for (int q = 0; q < 2 * n; q++) d[q] = ldexp(d[q], e);
    double dm = max_mag_lead(d, n);
    /* the previous update was below sqrt(tol_dx): the working-precision
       corrector would square it below tol_dx by now */
    int prev_small = o->updates >= 1 && d1 <= sqrt(orc_tol_dx(p, t));
    if (prev_small) o->onpath = 1;
    if (o->updates >= 2 && contracts_linearly(d2, d1, dm)) o->linear = 1;
    d2 = d1;
    d1 = dm;
    o->dxn = dm;
    for (int i = 0; i < n; i++) {
      orc_cplx di;
      memset(&di, 0, sizeof di);
      di.re.v[0] = d[i];
      di.im.v[0] = d[n + i];
      orc_c_store(L, x, n, i, orc_c_add(L, orc_c_load(L, x, n, i), di));
    }
    o->updates++;
    if (!fixed) {
      if (!isfinite(dm)) { success = 0; break; }
      if (dm < orc_tol_dx(p, t)) { success = 1; break; }
      last = r;
    }
    if (o->iters >= p->max_newton && !(prev_small && o->iters < max_it)) {
      success = fixed ? 1 : 0;
      break;
    }
  }
  free(h); free(J); free(jl); free(rl); free(d);
  return success;
}
