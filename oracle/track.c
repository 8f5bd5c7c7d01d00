/*
 * track.c -- the oracle's predictor, Newton corrector and path tracker.
 * TEST INFRASTRUCTURE: see oracle.h.
 *
 * Predictor (Section 3.1): each coordinate x_i(t) is extrapolated to the new t
 *   by the polynomial of degree p through the last p+1 accepted points
 *   (t_j, x_i(t_j)); here in Newton's divided-difference form, evaluated by
 *   Horner's rule, in working precision.  p = min(pred_order, #accepted - 1).
 * Corrector (Fig. 2): at most max_newton
 *   iterations of: evaluate h and J; fail if ||h|| grew past the previous
 *   residual (the first bound is max_res); succeed if ||h|| < tol_res; solve
 *   J dx = -h; x := x + dx; succeed if ||dx|| < tol_dx (with tol_path > 0, both
 *   tests use tol_path on the steps to t < 1).  Norms are max norms
 *   of |z| taken in double from the leading limbs (Section 3.1).
 * Step control (Fig. 3): t := min(1,
 *   t + dt); predict; correct; on success keep the point, count it, and after
 *   more than two successes in a row double dt (capped at max_dt); on failure
 *   reset the count and halve dt.  Readings where the figure is silent: a
 *   failed step restores t and x to the last accepted point; dt < min_dt ends
 *   the path (h_min of Section 2, Eq. (4)); the path ends after the step to
 *   t = 1 is accepted; #steps > max_steps ends it (checked before each step).
 * Fixed schedule: t_j = j / fixed_steps and exactly max_newton updates per
 *   step, no test and no rejection.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* ---- predictor ---------------------------------------------------------------- */

int orc_predict(int L, int n, int npts, const double *ts, const double *xs, double t,
                double *x_out) {
  if (npts < 1 || npts > 16) return ORC_EINVAL;
  long pt = (long)2 * L * n;               /* doubles per point */
  for (int i = 0; i < n; i++) {
    orc_cplx c[16];
    for (int j = 0; j < npts; j++) c[j] = orc_c_load(L, xs + j * pt, n, i);
    for (int lvl = 1; lvl < npts; lvl++)
      for (int j = npts - 1; j >= lvl; j--) {
        orc_real dt = orc_r_sub(L, orc_r_from(ts[j]), orc_r_from(ts[j - lvl]));
        c[j] = orc_c_div_real(L, orc_c_sub(L, c[j], c[j - 1]), dt);
      }
    orc_cplx v = c[npts - 1];
    for (int j = npts - 2; j >= 0; j--) {
      orc_real w = orc_r_sub(L, orc_r_from(t), orc_r_from(ts[j]));
      v = orc_c_add(L, orc_c_mul_real(L, v, w), c[j]);
    }
    orc_c_store(L, x_out, n, i, v);
  }
  return ORC_OK;
}

/* ---- corrector ----------------------------------------------------------------- */

static double max_mag(int L, const double *v, int m) {
  double r = 0.0;
  for (int i = 0; i < m; i++) {
    double a = orc_c_mag_d(orc_c_load(L, v, m, i));
    if (!(a <= r)) r = a;                  /* NaN propagates */
  }
  return r;
}

double orc_tol_res(const orc_params *p, double t) {
  return (p->tol_path > 0.0 && t < 1.0) ? p->tol_path : p->tol_res;
}

double orc_tol_dx(const orc_params *p, double t) {
  return (p->tol_path > 0.0 && t < 1.0) ? p->tol_path : p->tol_dx;
}

int orc_newton(const orc_system *f, const orc_system *g, const double *gamma, int k,
               double t, double *x, const orc_params *p, int fixed,
               int *iters, int *updates, double *res, double *dxn) {
  int L = f->L, N = f->N, n = f->n;
  double *h = malloc(sizeof(double) * 2 * L * N);
  double *J = malloc(sizeof(double) * 2 * L * (size_t)N * n);
  double *rhs = malloc(sizeof(double) * 2 * L * N);
  double *dx = malloc(sizeof(double) * 2 * L * n);
  if (!h || !J || !rhs || !dx) { free(h); free(J); free(rhs); free(dx); return -ORC_ENOMEM; }
  double tl[ORC_MAXL] = {t, 0.0, 0.0, 0.0};
  double last = p->max_res;
  int success = fixed ? 1 : 0;
  *iters = 0;
  *updates = 0;
  for (int it = 0; it < p->max_newton; it++) {
    orc_eval(f, g, gamma, k, tl, x, h, J, p->fixed_rows);
    (*iters)++;
    double r = max_mag(L, h, N);
    *res = r;
    if (!fixed) {
      if (!isfinite(r) || r > last) break;
      if (r < orc_tol_res(p, t)) { success = 1; break; }
    }
    for (int e = 0; e < 2 * L * N; e++) rhs[e] = -h[e];
    int st = orc_mgs_solve(L, N, n, J, rhs, dx, NULL, NULL, NULL);
    if (st != ORC_OK) {
      if (!fixed) break;
      for (int e = 0; e < 2 * L * n; e++) dx[e] = NAN;
    }
    double d = max_mag(L, dx, n);
    *dxn = d;
    for (int i = 0; i < n; i++) {
      orc_cplx xi = orc_c_add(L, orc_c_load(L, x, n, i), orc_c_load(L, dx, n, i));
      orc_c_store(L, x, n, i, xi);
    }
    (*updates)++;
    if (!fixed) {
      if (!isfinite(d)) break;
      if (d < orc_tol_dx(p, t)) { success = 1; break; }
    }
    last = r;
  }
  free(h); free(J); free(rhs); free(dx);
  return success;
}

/* ---- step-size control ------------------------------------------------------------- */

void orc_ctrl_init(orc_ctrl *c, const orc_params *p) {
  c->t = 0.0;
  c->dt = p->max_dt;
  c->nsucc = 0;
  c->nsteps = 0;
  c->done = 0;
  c->status = ORC_OK;
}

double orc_ctrl_next_t(orc_ctrl *c, const orc_params *p) {
  if (c->done) return -1.0;
  if (p->fixed_steps > 0) return (double)(c->nsteps + 1) / (double)p->fixed_steps;
  if (c->nsteps > p->max_steps) {
    c->done = 1;
    c->status = ORC_MAXSTEPS;
    return -1.0;
  }
  double tn = c->t + c->dt;
  return tn < 1.0 ? tn : 1.0;
}

void orc_ctrl_report(orc_ctrl *c, const orc_params *p, double t_new, int success) {
  if (p->fixed_steps > 0) {
    c->t = t_new;
    c->nsteps++;
    if (c->nsteps >= p->fixed_steps) c->done = 1;
    return;
  }
  if (success) {
    c->t = t_new;
    c->nsucc++;
    if (c->nsucc > 2) c->dt = 2.0 * c->dt < p->max_dt ? 2.0 * c->dt : p->max_dt;
    if (c->t >= 1.0) c->done = 1;
  } else {
    c->nsucc = 0;
    c->dt = c->dt / 2.0;
    if (c->dt < p->min_dt) {
      c->done = 1;
      c->status = ORC_STEPMIN;
    }
  }
  c->nsteps++;
}

/* ---- path tracker -------------------------------------------------------------------- */

typedef struct {
  int L, n, cap, count, head;        /* ring of accepted points, newest at head */
  double *ts, *xs;
} history;

static int hist_init(history *H, int L, int n, int cap) {
  H->L = L; H->n = n; H->cap = cap; H->count = 0; H->head = -1;
  H->ts = malloc(sizeof(double) * cap);
  H->xs = malloc(sizeof(double) * 2 * L * (size_t)n * cap);
  return H->ts && H->xs;
}

static void hist_free(history *H) { free(H->ts); free(H->xs); }

static void hist_push(history *H, double t, const double *x) {
  long pt = (long)2 * H->L * H->n;
  H->head = (H->head + 1) % H->cap;
  H->ts[H->head] = t;
  memcpy(H->xs + H->head * pt, x, sizeof(double) * pt);
  if (H->count < H->cap) H->count++;
}

/* the newest m points, oldest first, gathered into ts/xs */
static void hist_last(const history *H, int m, double *ts, double *xs) {
  long pt = (long)2 * H->L * H->n;
  for (int j = 0; j < m; j++) {
    int slot = (H->head - (m - 1 - j) + 2 * H->cap) % H->cap;
    ts[j] = H->ts[slot];
    memcpy(xs + j * pt, H->xs + slot * pt, sizeof(double) * pt);
  }
}

static int check_params(const orc_params *p) {
  if (p->max_newton < 1 || p->pred_order < 0 || p->pred_order > 8 || p->relax_k < 1) return 0;
  if (p->fixed_steps <= 0 && !(p->max_dt > 0.0 && p->min_dt > 0.0)) return 0;
  return 1;
}

int orc_track(const orc_system *f, const orc_system *g, const double *gamma,
              const double *x0, const orc_params *p, double *x_out, orc_stats *st,
              orc_record *log, int log_cap, int *log_len) {
  int L = f->L, n = f->n;
  long pt = (long)2 * L * n;
  memset(st, 0, sizeof *st);
  if (log_len) *log_len = 0;
  if (!check_params(p) || !gamma) return st->status = ORC_EINVAL;
  for (long e = 0; e < pt; e++)
    if (!isfinite(x0[e])) {
      memcpy(x_out, x0, sizeof(double) * pt);
      return st->status = ORC_NONFINITE;
    }
  history H;
  int npmax = p->pred_order + 1;
  double *ts = malloc(sizeof(double) * npmax);
  double *xs = malloc(sizeof(double) * pt * npmax);
  double *x = malloc(sizeof(double) * pt);
  if (!hist_init(&H, L, n, npmax) || !ts || !xs || !x) {
    hist_free(&H); free(ts); free(xs); free(x);
    return st->status = ORC_ENOMEM;
  }
  hist_push(&H, 0.0, x0);
  orc_ctrl c;
  orc_ctrl_init(&c, p);
  int fixed = p->fixed_steps > 0;
  for (;;) {
    double tn = orc_ctrl_next_t(&c, p);
    if (tn < 0.0) break;
    int m = H.count < npmax ? H.count : npmax;
    hist_last(&H, m, ts, xs);
    orc_predict(L, n, m, ts, xs, tn, x);
    int iters = 0, upd = 0;
    double res = NAN, dxn = NAN;
    int ok = orc_newton(f, g, gamma, p->relax_k, tn, x, p, fixed, &iters, &upd, &res, &dxn);
    if (ok < 0) { c.status = -ok; break; }
    st->steps++;
    st->newton_iters += iters;
    st->updates += upd;
    st->res = res;
    st->dx = dxn;
    if (ok) st->accepted++; else st->rejected++;
    if (log && log_len && *log_len < log_cap) {
      orc_record *r = &log[(*log_len)++];
      r->t = tn; r->res = res; r->dx = dxn; r->accepted = ok; r->updates = upd;
    }
    orc_ctrl_report(&c, p, tn, ok);
    if (ok) {
      hist_push(&H, tn, x);
      if (!fixed && max_mag(L, x, n) > p->max_x) {
        c.status = ORC_DIVERGED;
        break;
      }
    }
  }
  int m = 1;
  hist_last(&H, m, ts, xs);
  memcpy(x_out, xs, sizeof(double) * pt);
  st->t_final = ts[0];
  st->status = c.status;
  hist_free(&H); free(ts); free(xs); free(x);
  return st->status;
}

/* Replays a recorded schedule without deciding anything: for each accepted
   record, predict at its t from the accepted points so far and apply exactly
   its number of Newton updates. */
int orc_replay(const orc_system *f, const orc_system *g, const double *gamma,
               const double *x0, const orc_params *p, const orc_record *log, int nrec,
               double *x_out) {
  int L = f->L, n = f->n;
  long pt = (long)2 * L * n;
  if (!check_params(p) || !gamma) return ORC_EINVAL;
  history H;
  int npmax = p->pred_order + 1;
  double *ts = malloc(sizeof(double) * npmax);
  double *xs = malloc(sizeof(double) * pt * npmax);
  double *x = malloc(sizeof(double) * pt);
  if (!hist_init(&H, L, n, npmax) || !ts || !xs || !x) {
    hist_free(&H); free(ts); free(xs); free(x);
    return ORC_ENOMEM;
  }
  hist_push(&H, 0.0, x0);
  orc_params q = *p;
  q.max_newton = 1;
  for (int s = 0; s < nrec; s++) {
    if (!log[s].accepted) continue;
    int m = H.count < npmax ? H.count : npmax;
    hist_last(&H, m, ts, xs);
    orc_predict(L, n, m, ts, xs, log[s].t, x);
    for (int u = 0; u < log[s].updates; u++) {
      int iters, upd;
      double res, dxn;
      orc_newton(f, g, gamma, p->relax_k, log[s].t, x, &q, 1, &iters, &upd, &res, &dxn);
    }
    hist_push(&H, log[s].t, x);
  }
  hist_last(&H, 1, ts, xs);
  memcpy(x_out, xs, sizeof(double) * pt);
  hist_free(&H); free(ts); free(xs); free(x);
  return ORC_OK;
}

/* The precision form's tracker: Fig. 3 with the mixed corrector and the rules
   stated in oracle.h. */
int orc_track_mixed(const orc_system *f, const orc_system *g, const double *gamma,
                    const double *x0, const orc_params *p, double endgame, double *x_out,
                    orc_stats *st, orc_mixed_stats *ms, orc_record *log, int log_cap,
                    int *log_len) {
  int L = f->L, n = f->n;
  long pt = (long)2 * L * n;
  memset(st, 0, sizeof *st);
  memset(ms, 0, sizeof *ms);
  if (log_len) *log_len = 0;
  if (!check_params(p) || !gamma) return st->status = ORC_EINVAL;
  if (!(endgame > 0.0)) endgame = 1.0;
  for (long e = 0; e < pt; e++)
    if (!isfinite(x0[e])) {
      memcpy(x_out, x0, sizeof(double) * pt);
      return st->status = ORC_NONFINITE;
    }
  history H;
  int npmax = p->pred_order + 1;
  double *ts = malloc(sizeof(double) * npmax);
  double *xs = malloc(sizeof(double) * pt * npmax);
  double *x = malloc(sizeof(double) * pt);
  if (!hist_init(&H, L, n, npmax) || !ts || !xs || !x) {
    hist_free(&H); free(ts); free(xs); free(x);
    return st->status = ORC_ENOMEM;
  }
  hist_push(&H, 0.0, x0);
  orc_ctrl c;
  orc_ctrl_init(&c, p);
  int fixed = p->fixed_steps > 0, wp_rest = 0;
  for (;;) {
    double tn = orc_ctrl_next_t(&c, p);
    if (tn < 0.0) break;
    int m = H.count < npmax ? H.count : npmax;
    hist_last(&H, m, ts, xs);
    orc_predict(L, n, m, ts, xs, tn, x);
    int iters = 0, upd = 0, ok;
    double res = NAN, dxn = NAN;
    if (tn < endgame && !wp_rest) {
      orc_mixed_out o;
      ok = orc_corrector_mixed(f, g, gamma, p->relax_k, tn, x, p, fixed, 1, &o);
      if (ok < 0) { c.status = -ok; break; }
      st->newton_iters += o.iters;
      st->updates += o.updates;
      ms->solves_f64 += o.solves;
      if (o.solves) ms->cond = o.cond;
      iters = o.iters; upd = o.updates; res = o.res; dxn = o.dxn;
      int esc = o.escalate;
      if (!ok && o.onpath) esc = 2;
      if (!ok && o.linear && !fixed) {
        esc = 2;
        wp_rest = 1;
      }
      if (!ok && esc && !fixed) {                /* once more, in working precision */
        ms->escalated++;
        orc_predict(L, n, m, ts, xs, tn, x);
        ok = orc_newton(f, g, gamma, p->relax_k, tn, x, p, fixed, &iters, &upd, &res, &dxn);
        if (ok < 0) { c.status = -ok; break; }
        st->newton_iters += iters;
        st->updates += upd;
      }
    } else {
      ok = orc_newton(f, g, gamma, p->relax_k, tn, x, p, fixed, &iters, &upd, &res, &dxn);
      if (ok < 0) { c.status = -ok; break; }
      st->newton_iters += iters;
      st->updates += upd;
    }
    st->steps++;
    st->res = res;
    st->dx = dxn;
    if (ok) st->accepted++; else st->rejected++;
    if (log && log_len && *log_len < log_cap) {
      orc_record *r = &log[(*log_len)++];
      r->t = tn; r->res = res; r->dx = dxn; r->accepted = ok; r->updates = upd;
    }
    orc_ctrl_report(&c, p, tn, ok);
    if (ok) {
      hist_push(&H, tn, x);
      if (!fixed && max_mag(L, x, n) > p->max_x) {
        c.status = ORC_DIVERGED;
        break;
      }
    }
  }
  ms->wp_rest = wp_rest;
  hist_last(&H, 1, ts, xs);
  memcpy(x_out, xs, sizeof(double) * pt);
  st->t_final = ts[0];
  st->status = c.status;
  hist_free(&H); free(ts); free(xs); free(x);
  return st->status;
}
