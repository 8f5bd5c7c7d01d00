// ctrl.h -- step-size control of the path tracker (Fig. 3), compiled for both
// the host (exported as ph_ctrl_* so it can be checked without a GPU) and the
// device controller kernel.
//
// t := min(1, t + dt) is tried; on success t advances, the success count grows
// and, once more than two successes are in a row, dt doubles up to max_dt; on
// failure the count resets and dt halves.  Readings where the figure is silent:
// a failure keeps t at the last accepted point; dt < min_dt stops the path
// (PH_STEPMIN; h_min of Section 2, Eq. (4)); the path ends once the step to t = 1
// is accepted; #steps > max_steps (checked before a step) stops it
// (PH_MAXSTEPS).  A fixed schedule (fixed_steps > 0) tries t_j = j / fixed_steps
// and accepts every step.
#pragma once
#include <math.h>

#include "ph.h"

#ifdef __CUDACC__
#define PH_HD __host__ __device__ __forceinline__
#else
#define PH_HD inline
#endif

PH_HD void ctrl_init(ph_ctrl_state *c, const ph_track_params *p) {
  c->t = 0.0;
  c->dt = p->max_dt;
  c->nsucc = 0;
  c->nsteps = 0;
  c->done = 0;
  c->status = PH_OK;
}

PH_HD double ctrl_next_t(ph_ctrl_state *c, const ph_track_params *p) {
  if (c->done) return -1.0;
  if (p->fixed_steps > 0) return (double)(c->nsteps + 1) / (double)p->fixed_steps;
  if (c->nsteps > p->max_steps) {
    c->done = 1;
    c->status = PH_MAXSTEPS;
    return -1.0;
  }
  double tn = c->t + c->dt;
  return tn < 1.0 ? tn : 1.0;
}

PH_HD void ctrl_report(ph_ctrl_state *c, const ph_track_params *p, double t_new, int success) {
  if (p->fixed_steps > 0) {
    c->t = t_new;
    c->nsteps += 1;
    if (c->nsteps >= p->fixed_steps) c->done = 1;
    return;
  }
  if (success) {
    c->t = t_new;
    c->nsucc += 1;
    if (c->nsucc > 2) c->dt = (2.0 * c->dt < p->max_dt) ? 2.0 * c->dt : p->max_dt;
    if (c->t >= 1.0) c->done = 1;
  } else {
    c->nsucc = 0;
    c->dt = c->dt / 2.0;
    if (c->dt < p->min_dt) {
      c->done = 1;
      c->status = PH_STEPMIN;
    }
  }
  c->nsteps += 1;
}

// The corrector's tolerances for a step to t_new: tol_path (when positive) on
// the way, tol_res / tol_dx for the step that lands on t = 1.
PH_HD double ctrl_tol_res(const ph_track_params *p, double t_new) {
  return (p->tol_path > 0.0 && t_new < 1.0) ? p->tol_path : p->tol_res;
}
PH_HD double ctrl_tol_dx(const ph_track_params *p, double t_new) {
  return (p->tol_path > 0.0 && t_new < 1.0) ? p->tol_path : p->tol_dx;
}

// The precision form (lin_prec != 0): a failed step is corrected again in
// working precision only if one of its double-precision solves had kappa
// u_double above this: below it the double corrector contracts like the
// working-precision one.
constexpr double kEscalateRho = 1e-6;

// Whether three successive updates d2, d1, d0 of a low-precision corrector
// contract, but more slowly than Newton's quadratic convergence.  With
// r1 = d1 / d2 and r0 = d0 / d1, quadratic convergence gives r0 ~ r1^2; a
// corrector limited by its solves (relative error kappa u_low per iteration)
// gives r0 ~ r1.  The test: both ratios below 1 and r0 > r1^1.5.
PH_HD bool linear_contraction(double d2, double d1, double d0) {
  if (!(d2 > 0.0) || !(d1 > 0.0) || !(d0 >= 0.0) || !(d0 < INFINITY)) return false;
  const double r1 = d1 / d2, r0 = d0 / d1;
  return r1 < 1.0 && r0 < 1.0 && r0 > r1 * sqrt(r1);
}
