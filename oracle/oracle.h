/*
 * oracle.h -- plain, slow CPU reference for one predictor-corrector step of
 * polynomial homotopy continuation in complex double-double (L = 2 limbs) and
 * quad-double (L = 4 limbs) arithmetic (Verschelde & Yu, "Accelerating
 * Polynomial Homotopy Continuation on a Graphics Processing Unit with Double
 * Double and Quad Double Arithmetic", 2015).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, calls or
 * executes this code: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or table with the CUDA
 * library; the two only agree on the memory layout of their arguments.
 *
 * Layout shared with the library's C ABI (an interface, not code):
 *   a vector of m complex numbers in L limbs is m*2*L doubles, ordered
 *   [limb][re|im][index]  (limb 0 = leading double);
 *   an N x n complex matrix is column-major: [limb][re|im][col][row].
 *
 * Every arithmetic result is the exact result rounded once to L limbs: the
 * inputs are split into a list of doubles whose sum is exact (error-free
 * transformations), and that exact sum is rounded by orc_round_sum.
 */
#ifndef PH_ORACLE_H
#define PH_ORACLE_H
#include <stdint.h>

#define ORC_MAXL 4

/* status codes: the same numeric values as the library's ph_status */
enum {
  ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ECUDA = 3, ORC_DIVERGED = 4,
  ORC_MAXSTEPS = 5, ORC_STEPMIN = 6, ORC_NONFINITE = 7, ORC_TIMEOUT = 8
};

/* ---- scalars ------------------------------------------------------------ */
typedef struct { double v[ORC_MAXL]; } orc_real;           /* L limbs used */
typedef struct { orc_real re, im; } orc_cplx;

void orc_two_sum(double a, double b, double *s, double *e);
void orc_two_prod(double a, double b, double *p, double *e);
void orc_round_sum(const double *in, int m, int L, double *out);

orc_real orc_r_from(double d);
orc_real orc_r_add(int L, orc_real a, orc_real b);
orc_real orc_r_sub(int L, orc_real a, orc_real b);
orc_real orc_r_mul(int L, orc_real a, orc_real b);
orc_real orc_r_div(int L, orc_real a, orc_real b);
orc_real orc_r_sqrt(int L, orc_real a);
orc_real orc_r_neg(int L, orc_real a);

orc_cplx orc_c_add(int L, orc_cplx a, orc_cplx b);
orc_cplx orc_c_sub(int L, orc_cplx a, orc_cplx b);
orc_cplx orc_c_mul(int L, orc_cplx a, orc_cplx b);
orc_cplx orc_c_conj_mul(int L, orc_cplx a, orc_cplx b);    /* conj(a) * b */
orc_cplx orc_c_mul_real(int L, orc_cplx a, orc_real r);
orc_cplx orc_c_div_real(int L, orc_cplx a, orc_real r);
orc_real orc_c_abs2(int L, orc_cplx a);                     /* |a|^2 */
double   orc_c_mag_d(orc_cplx a);                          /* |a| from leading limbs, in double */

/* SoA load/store of element i of a vector with `stride` complex entries */
orc_cplx orc_c_load(int L, const double *v, long stride, long i);
void     orc_c_store(int L, double *v, long stride, long i, orc_cplx z);

/* vectorised entry points for the arithmetic pins (op codes in mp.c) */
int orc_vec_real(int op, int L, int count, const double *x, const double *y, double *z);
int orc_vec_cplx(int op, int L, int count, const double *x, const double *y, double *z);

/* ---- polynomial systems -------------------------------------------------- */
typedef struct orc_system {
  int L, N, n, M;
  int32_t *term_ptr, *var_ptr, *var_idx, *var_exp;
  orc_cplx *coeff;
  int *deg;                      /* total degree of each polynomial */
} orc_system;
int  orc_system_new(int L, int N, int n, const int32_t *term_ptr, const int32_t *var_ptr,
                    const int32_t *var_idx, const int32_t *var_exp, const double *coeff,
                    orc_system **out);
void orc_system_free(orc_system *s);
int  orc_system_degree(const orc_system *s, int i);

/* h(x,t) = gamma (1-t)^k g(x) + t^k f(x) and its Jacobian.  g == NULL means the
   total-degree start system g_i = x_i^{d_i} - 1.  gamma == NULL evaluates f alone.
   fixed != 0 (with g): a row where g has no terms is f's row unchanged (the
   monodromy homotopy of Section 4.2 holds the cyclic equations fixed). */
int orc_eval(const orc_system *f, const orc_system *g, const double *gamma, int k,
             const double *t, const double *x, double *h, double *J, int fixed);

/* ---- modified Gram-Schmidt least squares --------------------------------- */
/* Textbook MGS on the augmented N x (n+1) matrix [J | rhs]; Q (N x n) and the
   (n+1) x (n+1) upper-triangular R are optional outputs (R[n][n] is the
   residual norm); dx solves R dx = Q^H rhs by back substitution. */
int orc_mgs_solve(int L, int N, int n, const double *J, const double *rhs, double *dx,
                  double *Q, double *R, double *resid_norm);

/* ---- predictor, corrector, path tracker ----------------------------------- */
typedef struct {
  double max_dt, min_dt, tol_res, tol_dx, max_res, max_x;
  int32_t max_steps, max_newton, pred_order, relax_k, fixed_steps;
  int32_t fixed_rows;   /* rows where g has no terms are held fixed: h_i = f_i */
  double tol_path;      /* > 0: the corrector's tolerance (both tests) on steps
                           to t < 1; the step to t = 1 keeps tol_res, tol_dx */
} orc_params;

/* The corrector's tolerances for a step to t. */
double orc_tol_res(const orc_params *p, double t);
double orc_tol_dx(const orc_params *p, double t);

typedef struct {
  int32_t status, steps, accepted, rejected, newton_iters, updates;
  double t_final, res, dx;
} orc_stats;

typedef struct {
  double t, res, dx;
  int32_t accepted, updates;
} orc_record;

/* step-size controller state (Fig. 3) */
typedef struct {
  double t, dt;
  int32_t nsucc, nsteps, done, status;
} orc_ctrl;

void orc_ctrl_init(orc_ctrl *c, const orc_params *p);
/* next t to try, or -1 when the controller has stopped */
double orc_ctrl_next_t(orc_ctrl *c, const orc_params *p);
void orc_ctrl_report(orc_ctrl *c, const orc_params *p, double t_new, int success);

int orc_predict(int L, int n, int npts, const double *ts, const double *xs, double t,
                double *x_out);
int orc_newton(const orc_system *f, const orc_system *g, const double *gamma, int k,
               double t, double *x, const orc_params *p, int fixed,
               int *iters, int *updates, double *res, double *dxn);
int orc_track(const orc_system *f, const orc_system *g, const double *gamma,
              const double *x0, const orc_params *p, double *x_out, orc_stats *st,
              orc_record *log, int log_cap, int *log_len);
int orc_replay(const orc_system *f, const orc_system *g, const double *gamma,
               const double *x0, const orc_params *p, const orc_record *log, int nrec,
               double *x_out);

/* ---- the precision form's path tracker (lin = 1: Newton systems in double) ----
   A step below t = endgame runs the mixed corrector (orc_newton_mixed's
   iteration) with these rules, restated from the library's precision form:
   * one iteration beyond max_newton when the previous update was below
     sqrt(tol_dx) (the working-precision corrector would have squared it below
     tol_dx by then);
   * a failed step is corrected once more from the predicted point in working
     precision when a double solve had kappa_hat u_double above 1e-6 (kappa_hat
     = max r_kk / min r_kk), when an update below sqrt(tol_dx) was followed by
     another, or when the last three updates contracted more slowly than
     quadratically (d0/d1 > (d1/d2)^1.5, both ratios below 1); in the last case
     the rest of the path runs in working precision;
   * steps at or beyond endgame, and every step once the path runs in working
     precision, use the working-precision corrector (orc_newton).
   Logs record the last pass of each step; statistics count both passes. */
typedef struct {
  int32_t iters, updates, escalate, onpath, linear, solves;
  double res, dxn, cond;
} orc_mixed_out;

int orc_corrector_mixed(const orc_system *f, const orc_system *g, const double *gamma, int k,
                        double t, double *x, const orc_params *p, int fixed, int lin,
                        orc_mixed_out *o);

typedef struct {
  int32_t solves_f64, escalated, wp_rest, reserved;
  double cond;                      /* condition estimate of the last double solve */
} orc_mixed_stats;

int orc_track_mixed(const orc_system *f, const orc_system *g, const double *gamma,
                    const double *x0, const orc_params *p, double endgame, double *x_out,
                    orc_stats *st, orc_mixed_stats *ms, orc_record *log, int log_cap,
                    int *log_len);

/* ---- mixed-precision corrector (mixed.c) ---------------------------------- */
/* Least squares in low precision (lin = 1: double, 2: single) by textbook MGS
   on [J | rhs]; J is [re|im][col][row] and rhs [re|im][N] in double (rounded to
   float first when lin = 2); dx is [re|im][n]; *cond = max r_kk / min r_kk. */
int orc_lowprec_solve(int lin, int N, int n, const double *J, const double *rhs, double *dx,
                      double *cond);
/* orc_newton with the Newton system solved by orc_lowprec_solve on the rounded
   J and -h, the update accumulated in working precision */
int orc_newton_mixed(const orc_system *f, const orc_system *g, const double *gamma, int k,
                     double t, double *x, const orc_params *p, int fixed, int lin,
                     int *iters, int *updates, double *res, double *dxn, double *cond);

#endif
