/*
 * mgs.c -- the oracle's least-squares solver: textbook modified Gram-Schmidt
 * QR of the augmented matrix [J | rhs], then back substitution.
 * TEST INFRASTRUCTURE: see oracle.h.
 *
 * The paper solves the Newton system J dz = -f(z) (Section 2, Eq. (2)) with
 * the modified Gram-Schmidt method instead of LU with partial pivoting
 * (Introduction); N >= n (Section 2, input specification) makes it a least
 * squares problem.  This is the untiled, right-looking column version:
 *   for k = 0..n-1:  r_kk = ||a_k||_2,  q_k = a_k / r_kk,
 *                    for j > k:  r_kj = q_k^H a_j,  a_j := a_j - r_kj q_k
 * run over the n+1 columns of [J | rhs], so column n ends as Q^H rhs in R and
 * its remaining norm is the least-squares residual.  Then R dx = Q^H rhs is
 * solved from the bottom row up.  Sums run left to right over the rows.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

int orc_mgs_solve(int L, int N, int n, const double *J, const double *rhs, double *dx,
                  double *Q, double *R, double *resid_norm) {
  if ((L != 1 && L != 2 && L != 4) || n < 1 || N < n) return ORC_EINVAL;
  int nc = n + 1;
  orc_cplx *A = malloc(sizeof(orc_cplx) * (size_t)N * nc);
  orc_cplx *Rm = calloc((size_t)nc * nc, sizeof(orc_cplx));
  orc_cplx *y = malloc(sizeof(orc_cplx) * n);
  if (!A || !Rm || !y) { free(A); free(Rm); free(y); return ORC_ENOMEM; }
  long NN = (long)N * n;
  for (int j = 0; j < n; j++)
    for (int i = 0; i < N; i++) A[(long)j * N + i] = orc_c_load(L, J, NN, (long)j * N + i);
  for (int i = 0; i < N; i++) A[(long)n * N + i] = orc_c_load(L, rhs, N, i);

  int status = ORC_OK;
  for (int k = 0; k < n; k++) {
    orc_cplx *ak = A + (long)k * N;
    orc_real s = orc_r_from(0.0);
    for (int i = 0; i < N; i++) s = orc_r_add(L, s, orc_c_abs2(L, ak[i]));
    orc_real rkk = orc_r_sqrt(L, s);
    if (!(rkk.v[0] > 0.0) || !isfinite(rkk.v[0])) { status = ORC_NONFINITE; break; }
    Rm[(long)k * nc + k].re = rkk;
    for (int i = 0; i < N; i++) ak[i] = orc_c_div_real(L, ak[i], rkk);
    for (int j = k + 1; j < nc; j++) {
      orc_cplx *aj = A + (long)j * N;
      orc_cplx r;
      memset(&r, 0, sizeof r);
      for (int i = 0; i < N; i++) r = orc_c_add(L, r, orc_c_conj_mul(L, ak[i], aj[i]));
      Rm[(long)j * nc + k] = r;
      for (int i = 0; i < N; i++) aj[i] = orc_c_sub(L, aj[i], orc_c_mul(L, r, ak[i]));
    }
  }
  if (status == ORC_OK) {
    orc_cplx *an = A + (long)n * N;
    orc_real s = orc_r_from(0.0);
    for (int i = 0; i < N; i++) s = orc_r_add(L, s, orc_c_abs2(L, an[i]));
    Rm[(long)n * nc + n].re = orc_r_sqrt(L, s);
    if (resid_norm) *resid_norm = Rm[(long)n * nc + n].re.v[0];
    /* back substitution R dx = y, y = column n of R */
    for (int k = n - 1; k >= 0; k--) {
      orc_cplx v = Rm[(long)n * nc + k];
      for (int j = k + 1; j < n; j++) v = orc_c_sub(L, v, orc_c_mul(L, Rm[(long)j * nc + k], y[j]));
      y[k] = orc_c_div_real(L, v, Rm[(long)k * nc + k].re);
    }
    for (int k = 0; k < n; k++) orc_c_store(L, dx, n, k, y[k]);
  }
  if (Q)
    for (long e = 0; e < NN; e++) orc_c_store(L, Q, NN, e, A[e]);
  if (R)
    for (long e = 0; e < (long)nc * nc; e++) orc_c_store(L, R, (long)nc * nc, e, Rm[e]);
  free(A); free(Rm); free(y);
  return status;
}
