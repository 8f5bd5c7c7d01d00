/*
 * poly.c -- the oracle's polynomial systems and the homotopy
 *   h(x,t) = gamma (1-t)^k g(x) + t^k f(x)            (Section 2, Eq. (1))
 * with its Jacobian.  TEST INFRASTRUCTURE: see oracle.h.
 *
 * A system is given fully expanded, as a list of terms c * prod_j x_j^{a_j}
 * per polynomial (Section 3.1: every polynomial as its list of monomials with
 * their coefficients).  Values and partial derivatives are computed by symbolic
 * differentiation,
 *   d/dx_j [c prod_l x_l^{a_l}] = (c a_j) x_j^{a_j - 1} prod_{l != j} x_l^{a_l},
 * each product evaluated by plain repeated multiplication, coefficient first,
 * then the variables in the order the term lists them.  This is deliberately
 * not the reverse mode of algorithmic differentiation that the paper (and the
 * GPU library) use, so the two share no rounding pattern.  Sums run over the
 * terms left to right.
 *
 * The start system, when none is given, is the total-degree system
 * g_i = x_i^{d_i} - 1 with d_i the total degree of f_i.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

void orc_system_free(orc_system *s) {
  if (!s) return;
  free(s->term_ptr); free(s->var_ptr); free(s->var_idx); free(s->var_exp);
  free(s->coeff); free(s->deg);
  free(s);
}

int orc_system_degree(const orc_system *s, int i) { return s->deg[i]; }

int orc_system_new(int L, int N, int n, const int32_t *term_ptr, const int32_t *var_ptr,
                   const int32_t *var_idx, const int32_t *var_exp, const double *coeff,
                   orc_system **out) {
  *out = NULL;
  if ((L != 1 && L != 2 && L != 4) || N < 1 || n < 1 || N < n) return ORC_EINVAL;
  if (term_ptr[0] != 0) return ORC_EINVAL;
  for (int i = 0; i < N; i++) if (term_ptr[i + 1] < term_ptr[i]) return ORC_EINVAL;
  int M = term_ptr[N];
  if (var_ptr[0] != 0) return ORC_EINVAL;
  for (int k = 0; k < M; k++) if (var_ptr[k + 1] < var_ptr[k]) return ORC_EINVAL;
  int nnz = var_ptr[M];
  for (int p = 0; p < nnz; p++)
    if (var_idx[p] < 0 || var_idx[p] >= n || var_exp[p] < 1) return ORC_EINVAL;
  /* the variables of one term must be distinct */
  for (int k = 0; k < M; k++)
    for (int p = var_ptr[k]; p < var_ptr[k + 1]; p++)
      for (int q = p + 1; q < var_ptr[k + 1]; q++)
        if (var_idx[p] == var_idx[q]) return ORC_EINVAL;

  orc_system *s = calloc(1, sizeof *s);
  if (!s) return ORC_ENOMEM;
  s->L = L; s->N = N; s->n = n; s->M = M;
  s->term_ptr = malloc(sizeof(int32_t) * (N + 1));
  s->var_ptr = malloc(sizeof(int32_t) * (M + 1));
  s->var_idx = malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  s->var_exp = malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  s->coeff = malloc(sizeof(orc_cplx) * (M > 0 ? M : 1));
  s->deg = malloc(sizeof(int) * N);
  if (!s->term_ptr || !s->var_ptr || !s->var_idx || !s->var_exp || !s->coeff || !s->deg) {
    orc_system_free(s);
    return ORC_ENOMEM;
  }
  memcpy(s->term_ptr, term_ptr, sizeof(int32_t) * (N + 1));
  memcpy(s->var_ptr, var_ptr, sizeof(int32_t) * (M + 1));
  memcpy(s->var_idx, var_idx, sizeof(int32_t) * nnz);
  memcpy(s->var_exp, var_exp, sizeof(int32_t) * nnz);
  for (int k = 0; k < M; k++) s->coeff[k] = orc_c_load(L, coeff, M, k);
  for (int i = 0; i < N; i++) {
    int d = 0;
    for (int k = term_ptr[i]; k < term_ptr[i + 1]; k++) {
      int dk = 0;
      for (int p = var_ptr[k]; p < var_ptr[k + 1]; p++) dk += var_exp[p];
      if (dk > d) d = dk;
    }
    s->deg[i] = d;
  }
  *out = s;
  return ORC_OK;
}

static orc_cplx czero(void) {
  orc_cplx z;
  memset(&z, 0, sizeof z);
  return z;
}

/* f(x) and its Jacobian, J column-major N x n (entries not touched by a term
   stay zero). */
static void eval_system(const orc_system *s, const orc_cplx *x, orc_cplx *f, orc_cplx *J) {
  int L = s->L, N = s->N, n = s->n;
  for (int i = 0; i < N; i++) f[i] = czero();
  for (long e = 0; e < (long)N * n; e++) J[e] = czero();
  for (int i = 0; i < N; i++) {
    for (int k = s->term_ptr[i]; k < s->term_ptr[i + 1]; k++) {
      int p0 = s->var_ptr[k], p1 = s->var_ptr[k + 1];
      /* value: c, then each variable as often as its exponent */
      orc_cplx v = s->coeff[k];
      for (int p = p0; p < p1; p++)
        for (int e = 0; e < s->var_exp[p]; e++) v = orc_c_mul(L, v, x[s->var_idx[p]]);
      f[i] = orc_c_add(L, f[i], v);
      /* partial derivative with respect to the variable at position q */
      for (int q = p0; q < p1; q++) {
        orc_cplx d = orc_c_mul_real(L, s->coeff[k], orc_r_from((double)s->var_exp[q]));
        for (int p = p0; p < p1; p++) {
          int cnt = s->var_exp[p] - (p == q ? 1 : 0);
          for (int e = 0; e < cnt; e++) d = orc_c_mul(L, d, x[s->var_idx[p]]);
        }
        long at = (long)s->var_idx[q] * N + i;
        J[at] = orc_c_add(L, J[at], d);
      }
    }
  }
}

/* g_i = x_i^{d_i} - 1 and dg_i/dx_i = d_i x_i^{d_i - 1} */
static void eval_total_degree(const orc_system *f, const orc_cplx *x, orc_cplx *g, orc_cplx *J) {
  int L = f->L, n = f->n;
  for (long e = 0; e < (long)n * n; e++) J[e] = czero();
  for (int i = 0; i < n; i++) {
    int d = f->deg[i];
    orc_cplx p = x[i];
    for (int e = 1; e < d; e++) p = orc_c_mul(L, p, x[i]);
    orc_cplx one = czero();
    one.re.v[0] = 1.0;
    g[i] = orc_c_sub(L, p, one);
    orc_cplx dp = czero();
    dp.re.v[0] = (double)d;
    for (int e = 1; e < d; e++) dp = orc_c_mul(L, dp, x[i]);
    J[(long)i * n + i] = dp;
  }
}

int orc_eval(const orc_system *f, const orc_system *g, const double *gamma, int k,
             const double *t, const double *x, double *h, double *J, int fixed) {
  int L = f->L, N = f->N, n = f->n;
  if (k < 0) return ORC_EINVAL;
  if (g && (g->L != L || g->N != N || g->n != n)) return ORC_EINVAL;
  if (gamma && !g) {
    if (N != n) return ORC_EINVAL;
    for (int i = 0; i < N; i++) if (f->deg[i] < 1) return ORC_EINVAL;
  }
  orc_cplx *xv = malloc(sizeof(orc_cplx) * n);
  orc_cplx *fv = malloc(sizeof(orc_cplx) * N);
  orc_cplx *Jf = malloc(sizeof(orc_cplx) * (size_t)N * n);
  orc_cplx *gv = malloc(sizeof(orc_cplx) * N);
  orc_cplx *Jg = malloc(sizeof(orc_cplx) * (size_t)N * n);
  if (!xv || !fv || !Jf || !gv || !Jg) {
    free(xv); free(fv); free(Jf); free(gv); free(Jg);
    return ORC_ENOMEM;
  }
  for (int j = 0; j < n; j++) xv[j] = orc_c_load(L, x, n, j);
  eval_system(f, xv, fv, Jf);
  long NN = (long)N * n;
  if (!gamma) {
    for (int i = 0; i < N; i++) orc_c_store(L, h, N, i, fv[i]);
    for (long e = 0; e < NN; e++) orc_c_store(L, J, NN, e, Jf[e]);
  } else {
    if (g) eval_system(g, xv, gv, Jg);
    else eval_total_degree(f, xv, gv, Jg);
    orc_real tt, omt, tk, omtk;
    memset(&tt, 0, sizeof tt);
    for (int l = 0; l < L; l++) tt.v[l] = t[l];
    omt = orc_r_sub(L, orc_r_from(1.0), tt);
    tk = orc_r_from(1.0);
    omtk = orc_r_from(1.0);
    for (int e = 0; e < k; e++) {
      tk = orc_r_mul(L, tk, tt);
      omtk = orc_r_mul(L, omtk, omt);
    }
    orc_cplx gam = orc_c_load(L, gamma, 1, 0);
    orc_cplx sg = orc_c_mul_real(L, gam, omtk);
    /* a row held fixed (g has no terms there): f's row as it is */
    for (int i = 0; i < N; i++) {
      int hold = fixed && g && g->term_ptr[i + 1] == g->term_ptr[i];
      orc_cplx v = hold ? fv[i]
                        : orc_c_add(L, orc_c_mul(L, sg, gv[i]), orc_c_mul_real(L, fv[i], tk));
      orc_c_store(L, h, N, i, v);
    }
    for (long e = 0; e < NN; e++) {
      int i = (int)(e % N);                     /* J is [column j][row i] */
      int hold = fixed && g && g->term_ptr[i + 1] == g->term_ptr[i];
      orc_cplx v = hold ? Jf[e]
                        : orc_c_add(L, orc_c_mul(L, sg, Jg[e]), orc_c_mul_real(L, Jf[e], tk));
      orc_c_store(L, J, NN, e, v);
    }
  }
  free(xv); free(fv); free(Jf); free(gv); free(Jg);
  return ORC_OK;
}
