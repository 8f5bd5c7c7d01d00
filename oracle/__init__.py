"""CPU oracle for the DD/QD path tracker -- TEST INFRASTRUCTURE ONLY.

A plain, slow C implementation (files in this directory) of what the hot path
computes: multi-limb arithmetic, evaluation of h(x,t) and its Jacobian by
symbolic differentiation, textbook modified Gram-Schmidt least squares, the
extrapolation predictor, Newton's method and the step-size control of the
paper.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
use it; it shares no code with the CUDA library and does not import it.

Arrays follow the library's layout: complex vectors are float64 [L][2][m]
(limb, re/im, index); matrices are column-major [L][2][cols][rows].
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["mp.c", "poly.c", "mgs.c", "track.c", "mixed.c"]
_LIB = None
_LOCK = threading.Lock()

OK, EINVAL, ENOMEM, ECUDA, DIVERGED, MAXSTEPS, STEPMIN, NONFINITE, TIMEOUT = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "DIVERGED", "MAXSTEPS", "STEPMIN",
                "NONFINITE", "TIMEOUT"]


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C11, no FMA contraction)."""
    out = lib_path()
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(out) and \
            os.path.getmtime(out) >= max(os.path.getmtime(d) for d in deps):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Params(C.Structure):
    _fields_ = [("max_dt", C.c_double), ("min_dt", C.c_double), ("tol_res", C.c_double),
                ("tol_dx", C.c_double), ("max_res", C.c_double), ("max_x", C.c_double),
                ("max_steps", C.c_int32), ("max_newton", C.c_int32), ("pred_order", C.c_int32),
                ("relax_k", C.c_int32), ("fixed_steps", C.c_int32), ("fixed_rows", C.c_int32),
                ("tol_path", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps", C.c_int32), ("accepted", C.c_int32),
                ("rejected", C.c_int32), ("newton_iters", C.c_int32), ("updates", C.c_int32),
                ("t_final", C.c_double), ("res", C.c_double), ("dx", C.c_double)]


class MixedStats(C.Structure):
    _fields_ = [("solves_f64", C.c_int32), ("escalated", C.c_int32), ("wp_rest", C.c_int32),
                ("reserved", C.c_int32), ("cond", C.c_double)]


class Record(C.Structure):
    _fields_ = [("t", C.c_double), ("res", C.c_double), ("dx", C.c_double),
                ("accepted", C.c_int32), ("updates", C.c_int32)]


class Ctrl(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("nsucc", C.c_int32),
                ("nsteps", C.c_int32), ("done", C.c_int32), ("status", C.c_int32)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = C.CDLL(build())
            L.orc_round_sum.argtypes = [_dp, C.c_int, C.c_int, _dp]
            L.orc_vec_real.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
            L.orc_vec_cplx.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
            L.orc_system_new.argtypes = [C.c_int, C.c_int, C.c_int, _ip, _ip, _ip, _ip, _dp,
                                         C.POINTER(C.c_void_p)]
            L.orc_system_free.argtypes = [C.c_void_p]
            L.orc_system_degree.argtypes = [C.c_void_p, C.c_int]
            L.orc_eval.argtypes = [C.c_void_p, C.c_void_p, _dp, C.c_int, _dp, _dp, _dp, _dp,
                                   C.c_int]
            L.orc_mgs_solve.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_predict.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_double, _dp]
            L.orc_newton.argtypes = [C.c_void_p, C.c_void_p, _dp, C.c_int, C.c_double, _dp,
                                     C.POINTER(Params), C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), _dp, _dp]
            L.orc_track.argtypes = [C.c_void_p, C.c_void_p, _dp, _dp, C.POINTER(Params), _dp,
                                    C.POINTER(Stats), C.POINTER(Record), C.c_int,
                                    C.POINTER(C.c_int)]
            L.orc_replay.argtypes = [C.c_void_p, C.c_void_p, _dp, _dp, C.POINTER(Params),
                                     C.POINTER(Record), C.c_int, _dp]
            L.orc_track_mixed.argtypes = [C.c_void_p, C.c_void_p, _dp, _dp, C.POINTER(Params),
                                          C.c_double, _dp, C.POINTER(Stats),
                                          C.POINTER(MixedStats), C.POINTER(Record), C.c_int,
                                          C.POINTER(C.c_int)]
            L.orc_lowprec_solve.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
            L.orc_newton_mixed.argtypes = [C.c_void_p, C.c_void_p, _dp, C.c_int, C.c_double,
                                           _dp, C.POINTER(Params), C.c_int, C.c_int,
                                           C.POINTER(C.c_int), C.POINTER(C.c_int), _dp, _dp,
                                           _dp]
            L.orc_ctrl_init.argtypes = [C.POINTER(Ctrl), C.POINTER(Params)]
            L.orc_ctrl_next_t.argtypes = [C.POINTER(Ctrl), C.POINTER(Params)]
            L.orc_ctrl_next_t.restype = C.c_double
            L.orc_ctrl_report.argtypes = [C.POINTER(Ctrl), C.POINTER(Params), C.c_double, C.c_int]
            _LIB = L
    return _LIB


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    return a.ctypes.data_as(_ip)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- arithmetic pins ----------------------------------------------------------------

REAL_OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4, "two_sum": 5, "two_prod": 6}
CPLX_OPS = {"add": 0, "sub": 1, "mul": 2, "conj_mul": 3, "abs2": 4}


def round_sum(terms, L: int) -> np.ndarray:
    t = _f64(terms)
    out = np.zeros(L)
    lib().orc_round_sum(_d(t), len(t), L, _d(out))
    return out


def vec_real(op: str, L: int, x, y=None) -> np.ndarray:
    """x, y: [L][count] limbs; returns [L][count]."""
    x = _f64(x)
    count = x.shape[1]
    y = _f64(y) if y is not None else None
    z = np.zeros((L, count))
    st = lib().orc_vec_real(REAL_OPS[op], L, count, _d(x), _d(y) if y is not None else None, _d(z))
    assert st == OK
    return z


def vec_cplx(op: str, L: int, x, y=None) -> np.ndarray:
    """x, y: [L][2][count]; returns [L][2][count] ([L][count] for abs2)."""
    x = _f64(x)
    count = x.shape[2]
    y = _f64(y) if y is not None else None
    z = np.zeros((L, count)) if op == "abs2" else np.zeros((L, 2, count))
    st = lib().orc_vec_cplx(CPLX_OPS[op], L, count, _d(x), _d(y) if y is not None else None, _d(z))
    assert st == OK
    return z


# ---- systems and evaluation --------------------------------------------------------------


class System:
    """A polynomial system held by the oracle, built from any object with the
    fields N, n, term_ptr, var_ptr, var_idx, var_exp and coeff_soa(L)."""

    def __init__(self, spec, L: int):
        self.L, self.N, self.n = L, spec.N, spec.n
        self._keep = [np.ascontiguousarray(spec.term_ptr, dtype=np.int32),
                      np.ascontiguousarray(spec.var_ptr, dtype=np.int32),
                      np.ascontiguousarray(spec.var_idx, dtype=np.int32),
                      np.ascontiguousarray(spec.var_exp, dtype=np.int32),
                      _f64(spec.coeff_soa(L))]
        h = C.c_void_p()
        tp, vp, vi, ve, co = self._keep
        st = lib().orc_system_new(L, spec.N, spec.n, _i(tp), _i(vp), _i(vi), _i(ve), _d(co),
                                  C.byref(h))
        if st != OK:
            raise ValueError(f"oracle rejected the system: {STATUS_NAMES[st]}")
        self.h = h

    def degree(self, i: int) -> int:
        return lib().orc_system_degree(self.h, i)

    def __del__(self):
        if getattr(self, "h", None) and _LIB is not None:
            _LIB.orc_system_free(self.h)
            self.h = None


def _gamma(gamma, L):
    if gamma is None:
        return None
    g = _f64(gamma)
    if g.shape != (L, 2):
        raise ValueError("gamma must be [L][2]")
    return g


def _real_limbs(t, L):
    t = np.atleast_1d(_f64(t))
    out = np.zeros(L)
    out[:len(t)] = t
    return out


def eval_h(f: System, x, t=1.0, gamma=None, k: int = 1, g: System | None = None,
           fixed_rows: int = 0):
    """Values h [L][2][N] and Jacobian J [L][2][n][N] of gamma (1-t)^k g + t^k f
    (f alone when gamma is None); with fixed_rows, rows where g has no terms
    are f's rows unchanged."""
    L = f.L
    x = _f64(x)
    gm = _gamma(gamma, L)
    tl = _real_limbs(t, L)
    h = np.zeros((L, 2, f.N))
    J = np.zeros((L, 2, f.n, f.N))
    st = lib().orc_eval(f.h, g.h if g else None, _d(gm) if gm is not None else None, k,
                        _d(tl), _d(x), _d(h), _d(J), int(fixed_rows))
    if st != OK:
        raise ValueError(f"oracle eval failed: {STATUS_NAMES[st]}")
    return h, J


def mgs_solve(J, rhs, want_qr: bool = False):
    """Least-squares solution of J dx = rhs by MGS on [J | rhs].
    Returns (status, dx, residual_norm[, Q, R])."""
    J = _f64(J)
    rhs = _f64(rhs)
    L, _, n, N = J.shape
    dx = np.zeros((L, 2, n))
    Q = np.zeros((L, 2, n, N)) if want_qr else None
    R = np.zeros((L, 2, n + 1, n + 1)) if want_qr else None
    rn = C.c_double(0.0)
    st = lib().orc_mgs_solve(L, N, n, _d(J), _d(rhs), _d(dx), _d(Q) if want_qr else None,
                             _d(R) if want_qr else None, C.cast(C.pointer(rn), _dp))
    if want_qr:
        return st, dx, rn.value, Q, R
    return st, dx, rn.value


def predict(ts, xs, t):
    """xs: [npts][L][2][n] accepted points (oldest first) at times ts."""
    xs = _f64(xs)
    npts, L, _, n = xs.shape
    ts = _f64(ts)
    out = np.zeros((L, 2, n))
    st = lib().orc_predict(L, n, npts, _d(ts), _d(xs), float(t), _d(out))
    assert st == OK
    return out


def make_params(p: dict) -> Params:
    q = Params()
    for name, _ in Params._fields_:
        if name in p:
            setattr(q, name, p[name])
    return q


def newton(f: System, x, t, gamma, params: dict, g: System | None = None, fixed=False):
    """One corrector run; returns (success, x, iters, updates, res, dx)."""
    L = f.L
    x = _f64(x).copy()
    gm = _gamma(gamma, L)
    p = make_params(params)
    it, up = C.c_int(0), C.c_int(0)
    res, dxn = C.c_double(0), C.c_double(0)
    ok = lib().orc_newton(f.h, g.h if g else None, _d(gm), int(params.get("relax_k", 1)),
                          float(t), _d(x), C.byref(p), int(fixed), C.byref(it), C.byref(up),
                          C.cast(C.pointer(res), _dp), C.cast(C.pointer(dxn), _dp))
    return bool(ok), x, it.value, up.value, res.value, dxn.value


LIN = {"f64": 1, "f32": 2}


def lowprec_solve(J, rhs, lin: str):
    """Least squares J dx = rhs in IEEE double ("f64") or single ("f32") by
    textbook MGS.  J: complex [N][n] (numpy), rhs: complex [N].  Returns
    (status, dx complex [n], condition estimate)."""
    J = np.asarray(J, dtype=np.complex128)
    N, n = J.shape
    jp = np.ascontiguousarray(np.stack([J.real.T, J.imag.T]))     # [re|im][col][row]
    rhs = np.asarray(rhs, dtype=np.complex128)
    rp = np.ascontiguousarray(np.stack([rhs.real, rhs.imag]))
    dx = np.zeros((2, n))
    cond = C.c_double(0.0)
    st = lib().orc_lowprec_solve(LIN[lin], N, n, _d(jp), _d(rp), _d(dx),
                                 C.cast(C.pointer(cond), _dp))
    return st, dx[0] + 1j * dx[1], cond.value


def newton_mixed(f: System, x, t, gamma, params: dict, lin: str, g: System | None = None,
                 fixed=False):
    """One mixed-precision corrector run (residual and update in working
    precision, the Newton system in `lin`); returns (success, x, iters, updates,
    res, dx, condition estimate of the last solve)."""
    L = f.L
    x = _f64(x).copy()
    gm = _gamma(gamma, L)
    p = make_params(params)
    it, up = C.c_int(0), C.c_int(0)
    res, dxn, cond = C.c_double(0), C.c_double(0), C.c_double(math.nan)
    ok = lib().orc_newton_mixed(f.h, g.h if g else None, _d(gm), int(params.get("relax_k", 1)),
                                float(t), _d(x), C.byref(p), int(fixed), LIN[lin],
                                C.byref(it), C.byref(up), C.cast(C.pointer(res), _dp),
                                C.cast(C.pointer(dxn), _dp), C.cast(C.pointer(cond), _dp))
    if ok < 0:
        raise ValueError(f"oracle mixed newton failed: {STATUS_NAMES[-ok]}")
    return bool(ok), x, it.value, up.value, res.value, dxn.value, cond.value


def track(f: System, x0, gamma, params: dict, g: System | None = None, log_cap: int = 20000):
    """Track one path; returns (status, x_end, stats dict, log list)."""
    L = f.L
    x0 = _f64(x0)
    gm = _gamma(gamma, L)
    p = make_params(params)
    xo = np.zeros_like(x0)
    st = Stats()
    log = (Record * log_cap)()
    nlog = C.c_int(0)
    status = lib().orc_track(f.h, g.h if g else None, _d(gm), _d(x0), C.byref(p), _d(xo),
                             C.byref(st), log, log_cap, C.byref(nlog))
    stats = {name: getattr(st, name) for name, _ in Stats._fields_}
    recs = [dict(t=log[i].t, res=log[i].res, dx=log[i].dx, accepted=log[i].accepted,
                 updates=log[i].updates) for i in range(nlog.value)]
    return status, xo, stats, recs


def track_mixed(f: System, x0, gamma, params: dict, g: System | None = None,
                log_cap: int = 20000):
    """Track one path in the precision form (Newton systems in double; the
    rules at orc_track_mixed); params' endgame_t as in the library.  Returns
    (status, x_end, stats dict (with solves_f64, escalated, wp_rest, cond),
    log list)."""
    L = f.L
    x0 = _f64(x0)
    gm = _gamma(gamma, L)
    p = make_params(params)
    xo = np.zeros_like(x0)
    st = Stats()
    ms = MixedStats()
    log = (Record * log_cap)()
    nlog = C.c_int(0)
    status = lib().orc_track_mixed(f.h, g.h if g else None, _d(gm), _d(x0), C.byref(p),
                                   float(params.get("endgame_t", 0.0)), _d(xo), C.byref(st),
                                   C.byref(ms), log, log_cap, C.byref(nlog))
    stats = {name: getattr(st, name) for name, _ in Stats._fields_}
    stats.update({name: getattr(ms, name) for name, _ in MixedStats._fields_ if name != "reserved"})
    recs = [dict(t=log[i].t, res=log[i].res, dx=log[i].dx, accepted=log[i].accepted,
                 updates=log[i].updates) for i in range(nlog.value)]
    return status, xo, stats, recs


def replay(f: System, x0, gamma, params: dict, records, g: System | None = None):
    """Replay a schedule: records with keys t, accepted, updates."""
    L = f.L
    x0 = _f64(x0)
    gm = _gamma(gamma, L)
    p = make_params(params)
    arr = (Record * max(1, len(records)))()
    for i, r in enumerate(records):
        arr[i].t = r["t"]
        arr[i].accepted = int(r["accepted"])
        arr[i].updates = int(r["updates"])
    xo = np.zeros_like(x0)
    st = lib().orc_replay(f.h, g.h if g else None, _d(gm), _d(x0), C.byref(p), arr,
                          len(records), _d(xo))
    if st != OK:
        raise ValueError(f"oracle replay failed: {STATUS_NAMES[st]}")
    return xo


class Controller:
    """The step-size controller alone, for scripted tests."""

    def __init__(self, params: dict):
        self.p = make_params(params)
        self.c = Ctrl()
        lib().orc_ctrl_init(C.byref(self.c), C.byref(self.p))

    def next_t(self) -> float:
        return lib().orc_ctrl_next_t(C.byref(self.c), C.byref(self.p))

    def report(self, t_new: float, success: bool):
        lib().orc_ctrl_report(C.byref(self.c), C.byref(self.p), float(t_new), int(success))

    @property
    def state(self) -> dict:
        return {name: getattr(self.c, name) for name, _ in Ctrl._fields_}
