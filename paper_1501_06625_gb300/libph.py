"""Python binding of libph (include/ph.h) -- argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: arrays (numpy arrays in host memory, or torch tensors in
device or pinned host memory) are checked for dtype and contiguity and passed
as raw pointers.  The shared library must have been built for sm_103a
(paper_1501_06625_gb300.build.build()); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_LIB = None
_LOCK = threading.Lock()

PH_D, PH_DD, PH_QD = 1, 2, 4
(PH_OK, PH_EINVAL, PH_ENOMEM, PH_ECUDA, PH_DIVERGED, PH_MAXSTEPS, PH_STEPMIN, PH_NONFINITE,
 PH_TIMEOUT) = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "DIVERGED", "MAXSTEPS", "STEPMIN",
                "NONFINITE", "TIMEOUT"]


class TrackParams(C.Structure):
    _fields_ = [("max_dt", C.c_double), ("min_dt", C.c_double), ("tol_res", C.c_double),
                ("tol_dx", C.c_double), ("max_res", C.c_double), ("max_x", C.c_double),
                ("max_steps", C.c_int32), ("max_newton", C.c_int32), ("pred_order", C.c_int32),
                ("relax_k", C.c_int32), ("fixed_steps", C.c_int32), ("control", C.c_int32),
                ("lin_prec", C.c_int32), ("fixed_rows", C.c_int32), ("endgame_t", C.c_double),
                ("cond_f32", C.c_double), ("tol_path", C.c_double)]


class PathStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps", C.c_int32), ("accepted", C.c_int32),
                ("rejected", C.c_int32), ("newton_iters", C.c_int32), ("updates", C.c_int32),
                ("t_final", C.c_double), ("res", C.c_double), ("dx", C.c_double),
                ("launches", C.c_int64), ("solves_f64", C.c_int32), ("solves_f32", C.c_int32),
                ("escalated", C.c_int32), ("wp_rest", C.c_int32), ("cond", C.c_double)]


class StepRecord(C.Structure):
    _fields_ = [("t", C.c_double), ("res", C.c_double), ("dx", C.c_double),
                ("accepted", C.c_int32), ("updates", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("max_n", C.c_int32), ("max_blocks", C.c_int32), ("pool_bytes", C.c_int64),
                ("queue_cap", C.c_int32), ("big_n", C.c_int32)]


class CtrlState(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("nsucc", C.c_int32),
                ("nsteps", C.c_int32), ("done", C.c_int32), ("status", C.c_int32)]


EXPORTS = ["ph_init", "ph_destroy", "ph_last_error", "ph_system_load", "ph_system_free",
           "ph_eval_jac", "ph_mgs_solve", "ph_track_path", "ph_ctrl_init", "ph_ctrl_next_t",
           "ph_ctrl_report", "ph_version", "ph_profile_newton", "ph_fp64_peak",
           "ph_mgs_solve_static", "ph_track_paths", "ph_server_create", "ph_server_submit",
           "ph_server_poll", "ph_server_wait", "ph_server_info", "ph_server_destroy",
           "ph_server_job_bytes", "ph_mgs_variant", "ph_sum_lanes", "ph_ctrl_linear_contraction",
           "ph_mgs_set_variant", "ph_set_wait_limit", "ph_set_memory_limit",
           "ph_debug_withhold_pivot", "ph_block_lanes", "ph_set_block_lanes",
           "ph_debug_warp_sum", "ph_unit_rates", "ph_debug_update"]


class PhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")


def lib():
    """The loaded libph.so; raises if it has not been built."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libph.so is not built ({path}); call "
                                   "paper_1501_06625_gb300.build.build() first")
            L = C.CDLL(path)
            vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
            L.ph_init.argtypes = [C.POINTER(vp), C.c_int, vp]
            L.ph_destroy.argtypes = [vp]
            L.ph_last_error.argtypes = [vp]
            L.ph_last_error.restype = C.c_char_p
            L.ph_system_load.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp,
                                         C.POINTER(vp)]
            L.ph_system_free.argtypes = [vp]
            L.ph_eval_jac.argtypes = [vp, vp, vp, vp, C.c_int, vp, vp, vp, vp]
            L.ph_mgs_solve.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp, dp]
            L.ph_track_path.argtypes = [vp, vp, vp, vp, vp, C.POINTER(TrackParams), vp,
                                        C.POINTER(PathStats), C.POINTER(StepRecord), C.c_int]
            L.ph_ctrl_init.argtypes = [C.POINTER(CtrlState), C.POINTER(TrackParams)]
            L.ph_ctrl_init.restype = None
            L.ph_ctrl_next_t.argtypes = [C.POINTER(CtrlState), C.POINTER(TrackParams)]
            L.ph_ctrl_next_t.restype = C.c_double
            L.ph_ctrl_report.argtypes = [C.POINTER(CtrlState), C.POINTER(TrackParams), C.c_double,
                                         C.c_int]
            L.ph_ctrl_report.restype = None
            L.ph_ctrl_linear_contraction.argtypes = [C.c_double, C.c_double, C.c_double]
            L.ph_ctrl_linear_contraction.restype = C.c_int
            L.ph_version.restype = C.c_char_p
            L.ph_profile_newton.argtypes = [vp, vp, vp, vp, C.c_int, vp, vp, C.c_int, dp]
            L.ph_set_wait_limit.argtypes = [vp, C.c_double]
            L.ph_debug_warp_sum.argtypes = [C.c_int, C.c_int, dp, dp]
            L.ph_debug_update.argtypes = [C.c_int, C.c_int, C.c_int, vp, vp]
            L.ph_unit_rates.argtypes = [vp, dp]
            L.ph_block_lanes.argtypes = [vp, vp, C.POINTER(C.c_int), dp]
            L.ph_set_block_lanes.argtypes = [vp, vp, C.c_int]
            L.ph_set_memory_limit.argtypes = [C.c_int64, C.POINTER(C.c_int64)]
            L.ph_debug_withhold_pivot.argtypes = [vp, C.c_int]
            L.ph_mgs_set_variant.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
            L.ph_mgs_variant.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                         C.POINTER(C.c_int), dp]
            L.ph_sum_lanes.argtypes = [vp, vp, vp, C.POINTER(C.c_int), dp]
            L.ph_fp64_peak.argtypes = [vp, C.c_double, dp]
            L.ph_server_create.argtypes = [vp, C.POINTER(ServerConfig), C.POINTER(vp)]
            L.ph_server_submit.argtypes = [vp, vp, vp, vp, vp, C.POINTER(TrackParams),
                                           C.POINTER(C.c_int64)]
            L.ph_server_poll.argtypes = [vp, C.c_int64, C.POINTER(C.c_int), vp,
                                         C.POINTER(PathStats), dp]
            L.ph_server_wait.argtypes = [vp, C.c_int64, C.c_int, vp, C.POINTER(PathStats), dp]
            L.ph_server_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.ph_server_destroy.argtypes = [vp]
            L.ph_server_job_bytes.argtypes = [vp, vp, vp, C.POINTER(C.c_int64)]
            L.ph_track_paths.argtypes = [vp, vp, vp, vp, C.c_int, vp, C.POINTER(TrackParams), vp,
                                         C.POINTER(PathStats), C.POINTER(StepRecord), C.c_int]
            L.ph_mgs_solve_static.argtypes = [C.c_int, vp, C.c_int, C.c_int, C.c_int, vp, vp, vp,
                                              dp]
            _LIB = L
    return _LIB


def _ptr(a, dtype=np.float64):
    """Raw pointer of a contiguous numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a contiguous {np.dtype(dtype).name} array")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):                       # torch.Tensor
        import torch
        want = torch.float64 if dtype == np.float64 else torch.int32
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, st: int):
    if st != PH_OK:
        raise PhError(st, ph_last_error(ctx))
    return st


def ph_version() -> str:
    return lib().ph_version().decode()


def ph_init(device: int = 0, stream=None):
    """Returns a context handle; stream is a torch.cuda.Stream, a raw handle or None."""
    h = C.c_void_p()
    raw = None
    if stream is not None:
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = lib().ph_init(C.byref(h), device, raw)
    if st != PH_OK:
        raise PhError(st, "ph_init failed")
    return h


def ph_destroy(ctx):
    return lib().ph_destroy(ctx)


def ph_last_error(ctx) -> str:
    return lib().ph_last_error(ctx).decode()


def ph_system_load(ctx, prec: int, N: int, n: int, term_ptr, var_ptr, var_idx, var_exp, coeff):
    h = C.c_void_p()
    st = lib().ph_system_load(ctx, prec, N, n, _ptr(term_ptr, np.int32), _ptr(var_ptr, np.int32),
                              _ptr(var_idx, np.int32), _ptr(var_exp, np.int32), _ptr(coeff),
                              C.byref(h))
    _check(ctx, st)
    return h


def ph_system_free(sys):
    return lib().ph_system_free(sys)


def ph_eval_jac(ctx, f, g, gamma, k, t, x, h, J):
    return _check(ctx, lib().ph_eval_jac(ctx, f, g, _ptr(gamma), k, _ptr(t), _ptr(x), _ptr(h),
                                         _ptr(J)))


def ph_mgs_solve(ctx, prec, N, n, J, rhs, dx) -> float:
    r = C.c_double(0.0)
    _check(ctx, lib().ph_mgs_solve(ctx, prec, N, n, _ptr(J), _ptr(rhs), _ptr(dx), C.byref(r)))
    return r.value


def ph_mgs_solve_static(device: int, stream, prec, N, n, J, rhs, dx) -> float:
    """ph_mgs_solve without a context and without allocating (static scratch)."""
    r = C.c_double(0.0)
    raw = None
    if stream is not None:
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = lib().ph_mgs_solve_static(device, raw, prec, N, n, _ptr(J), _ptr(rhs), _ptr(dx),
                                   C.byref(r))
    if st != PH_OK:
        raise PhError(st, "ph_mgs_solve_static failed")
    return r.value


def make_params(p: dict) -> TrackParams:
    q = TrackParams()
    for name, _ in TrackParams._fields_:
        if name in p:
            setattr(q, name, p[name])
    return q


def ph_track_path(ctx, f, g, gamma, x0, params: dict, x_out, log_cap: int = 0):
    """Returns (status, stats dict, list of step records)."""
    p = make_params(params)
    stats = PathStats()
    log = (StepRecord * max(1, log_cap))()
    st = lib().ph_track_path(ctx, f, g, _ptr(gamma), _ptr(x0), C.byref(p), _ptr(x_out),
                             C.byref(stats), log if log_cap > 0 else None, log_cap)
    if st in (PH_EINVAL, PH_ENOMEM, PH_ECUDA, PH_TIMEOUT):
        raise PhError(st, ph_last_error(ctx))
    sd = {name: getattr(stats, name) for name, _ in PathStats._fields_}
    n = min(sd["steps"], log_cap)
    recs = [dict(t=log[i].t, res=log[i].res, dx=log[i].dx, accepted=log[i].accepted,
                 updates=log[i].updates) for i in range(n)]
    return st, sd, recs


def ph_track_paths(ctx, f, g, gamma, x0, params: dict, x_out, log_cap: int = 0):
    """x0, x_out: [npaths][L][2][n].  Returns (list of stats dicts, list of logs)."""
    npaths = int(x0.shape[0])
    p = make_params(params)
    stats = (PathStats * max(1, npaths))()
    log = (StepRecord * max(1, npaths * log_cap))()
    _check(ctx, lib().ph_track_paths(ctx, f, g, _ptr(gamma), npaths, _ptr(x0), C.byref(p),
                                     _ptr(x_out), stats, log if log_cap > 0 else None, log_cap))
    sds = [{name: getattr(stats[i], name) for name, _ in PathStats._fields_} for i in range(npaths)]
    logs = []
    for i in range(npaths):
        nrec = min(sds[i]["steps"], log_cap)
        logs.append([dict(t=log[i * log_cap + r].t, res=log[i * log_cap + r].res,
                          dx=log[i * log_cap + r].dx, accepted=log[i * log_cap + r].accepted,
                          updates=log[i * log_cap + r].updates) for r in range(nrec)])
    return sds, logs


def ph_server_create(ctx, max_n: int, pool_bytes: int, queue_cap: int = 1024,
                     max_blocks: int = 0, big_n: int = 0):
    cfg = ServerConfig(max_n, max_blocks, pool_bytes, queue_cap, big_n)
    h = C.c_void_p()
    _check(ctx, lib().ph_server_create(ctx, C.byref(cfg), C.byref(h)))
    return h


def ph_server_submit(ctx, srv, f, g, gamma, x0, params: dict) -> int:
    jid = C.c_int64(0)
    p = make_params(params)
    _check(ctx, lib().ph_server_submit(srv, f, g, _ptr(gamma), _ptr(x0), C.byref(p),
                                       C.byref(jid)))
    return jid.value


def ph_server_poll(ctx, srv, job_id: int, x_out=None):
    """(done, stats dict or None, latency_ms or None)."""
    done = C.c_int(0)
    st = PathStats()
    lat = C.c_double(0.0)
    _check(ctx, lib().ph_server_poll(srv, job_id, C.byref(done), _ptr(x_out), C.byref(st),
                                     C.byref(lat)))
    if not done.value:
        return False, None, None
    return True, {k: getattr(st, k) for k, _ in PathStats._fields_}, lat.value


def ph_server_wait(ctx, srv, job_id: int, timeout_ms: int, x_out=None):
    st = PathStats()
    lat = C.c_double(0.0)
    _check(ctx, lib().ph_server_wait(srv, job_id, timeout_ms, _ptr(x_out), C.byref(st),
                                     C.byref(lat)))
    return {k: getattr(st, k) for k, _ in PathStats._fields_}, lat.value


def ph_server_info(srv) -> dict:
    v = [C.c_int64(0) for _ in range(4)]
    lib().ph_server_info(srv, *[C.byref(x) for x in v])
    return dict(waiting=v[0].value, on_device=v[1].value, kernel_launches=v[2].value,
                pool_free_bytes=v[3].value)


def ph_server_job_bytes(srv, f, g=None) -> int:
    b = C.c_int64(0)
    lib().ph_server_job_bytes(srv, f, g, C.byref(b))
    return b.value


def ph_server_destroy(srv):
    return lib().ph_server_destroy(srv)


def ph_ctrl_init(state: CtrlState, params: dict):
    p = make_params(params)
    lib().ph_ctrl_init(C.byref(state), C.byref(p))
    return p


def ph_ctrl_next_t(state: CtrlState, p: TrackParams) -> float:
    return lib().ph_ctrl_next_t(C.byref(state), C.byref(p))


def ph_ctrl_report(state: CtrlState, p: TrackParams, t_new: float, success: bool):
    lib().ph_ctrl_report(C.byref(state), C.byref(p), float(t_new), int(success))


def ph_ctrl_linear_contraction(d2: float, d1: float, d0: float) -> bool:
    return bool(lib().ph_ctrl_linear_contraction(float(d2), float(d1), float(d0)))


def ph_profile_newton(ctx, f, g, gamma, k, t, x, reps: int = 10):
    """Average ms per launch of [power table, monomial AD, summation, MGS]."""
    out = (C.c_double * 4)()
    _check(ctx, lib().ph_profile_newton(ctx, f, g, _ptr(gamma), k, _ptr(t), _ptr(x), reps, out))
    return list(out)


MGS_GRID, MGS_CLUSTER, MGS_TILED = 0, 1, 2
MGS_KINDS = ["grid", "cluster", "tiled"]


def ph_mgs_variant(ctx, prec: int, N: int, n: int):
    """(kind, size, [ms grid, ms cluster, ms tiled]) of the MGS solve of a shape
    (-1 where a variant was not measured)."""
    kind, size = C.c_int(0), C.c_int(0)
    ms = (C.c_double * 3)()
    _check(ctx, lib().ph_mgs_variant(ctx, prec, N, n, C.byref(kind), C.byref(size), ms))
    return kind.value, size.value, list(ms)


def ph_mgs_set_variant(ctx, prec: int, N: int, n: int, kind: int, size: int = 0):
    """Pins the solve variant of a shape (kind -1: back to the timed choice)."""
    return _check(ctx, lib().ph_mgs_set_variant(ctx, prec, N, n, kind, size))


def ph_block_lanes(ctx, f):
    """(lanes per output of the per-block summation, ms of 1..32 lanes or -1)."""
    lanes = C.c_int(0)
    ms = (C.c_double * 6)()
    _check(ctx, lib().ph_block_lanes(ctx, f, C.byref(lanes), ms))
    return lanes.value, list(ms)


def ph_set_block_lanes(ctx, f, lanes: int):
    return _check(ctx, lib().ph_set_block_lanes(ctx, f, lanes))


def ph_unit_rates(ctx):
    """G ops/s of FP64 FMA (pipe), FP64 FMA (tensor cores), 32-bit integer multiply-add."""
    r = (C.c_double * 3)()
    _check(ctx, lib().ph_unit_rates(ctx, r))
    return list(r)


def ph_debug_update(device: int, cases):
    """a - ar b + sg ai c in the MGS kernels' fixed-point forms for cases
    [count][6][limbs] (a, ar, b, ai, c, sg); returns [count][limbs] (test
    support)."""
    v = np.ascontiguousarray(cases, dtype=np.float64)
    count, six, limbs = v.shape
    assert six == 6
    out = np.zeros((count, limbs))
    st = lib().ph_debug_update(device, limbs, count, _ptr(v), _ptr(out))
    if st != PH_OK:
        raise PhError(st, "ph_debug_update failed")
    return out


def ph_debug_warp_sum(device: int, values):
    """The exact warp sum of 32 multi-limb values [32][limbs] (test support)."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    limbs = v.shape[1]
    out = np.zeros(limbs)
    st = lib().ph_debug_warp_sum(device, limbs, v.ctypes.data_as(C.POINTER(C.c_double)),
                                 out.ctypes.data_as(C.POINTER(C.c_double)))
    if st != PH_OK:
        raise PhError(st, "ph_debug_warp_sum failed")
    return out


def ph_set_wait_limit(ctx, ms: float):
    return _check(ctx, lib().ph_set_wait_limit(ctx, ms))


def ph_set_memory_limit(nbytes: int) -> int:
    """Caps the library's device memory (0: no cap); returns the bytes held now."""
    used = C.c_int64(0)
    st = lib().ph_set_memory_limit(nbytes, C.byref(used))
    if st != PH_OK:
        raise PhError(st, "ph_set_memory_limit failed")
    return used.value


def ph_debug_withhold_pivot(ctx, k: int):
    return _check(ctx, lib().ph_debug_withhold_pivot(ctx, k))


def ph_sum_lanes(ctx, f, g=None):
    """(lanes per output the summation uses, [ms for 1, 2, 4, 8, 16, 32 lanes])."""
    lanes = C.c_int(0)
    ms = (C.c_double * 6)()
    _check(ctx, lib().ph_sum_lanes(ctx, f, g, C.byref(lanes), ms))
    return lanes.value, list(ms)


def ph_fp64_peak(ctx, ms_target: float = 50.0) -> float:
    """Measured FP64 FMA rate, G lane-ops/s."""
    r = C.c_double(0.0)
    _check(ctx, lib().ph_fp64_peak(ctx, ms_target, C.byref(r)))
    return r.value


# ---- small conveniences (marshalling of the synthetic workloads) ---------------------

class Context:
    """Owns a ph_ctx; systems loaded through it are freed with it."""

    def __init__(self, device: int = 0, stream=None):
        self.h = ph_init(device, stream)
        self.systems = []

    def load(self, spec, L: int):
        s = ph_system_load(self.h, L, spec.N, spec.n,
                           np.ascontiguousarray(spec.term_ptr, dtype=np.int32),
                           np.ascontiguousarray(spec.var_ptr, dtype=np.int32),
                           np.ascontiguousarray(spec.var_idx, dtype=np.int32),
                           np.ascontiguousarray(spec.var_exp, dtype=np.int32),
                           np.ascontiguousarray(spec.coeff_soa(L), dtype=np.float64))
        self.systems.append(s)
        return s

    def free(self, s):
        """Frees one loaded system before the context closes."""
        self.systems.remove(s)
        ph_system_free(s)

    def close(self):
        if self.h:
            for s in self.systems:
                ph_system_free(s)
            self.systems = []
            ph_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
