#!/usr/bin/env python3
"""Benchmark of the DD/QD path tracker on GB300.

A step is one tracked path segment: the first 50 predictor-corrector steps of
the solution path of the dense n = 64 system (64 polynomials of 64 monomials
over 16 distinct variables, exponents in {1,2,3}, unit-modulus coefficients;
total-degree homotopy from the all-ones root, adaptive step control) in
complex double-double, by one ph_track_path call (max_steps = 49): every row
of the hot path (predictor, power table, monomial AD, summation, residual
norm, MGS, back substitution, update, step control) runs in every step.  A
whole path is not bounded in time: with degrees up to 48 the path is stiff at
the start and needs thousands of steps.  The first 20 steps of the same path
in complex quad-double are timed beside it.

value   corrector steps (Newton iterations: evaluation + MGS + update) per
        second, inputs resident on the device, CUDA events on the library's
        stream, L2 flushed (a 256 MiB write) between steps outside the events;
e2e     the same through the same call with pinned host buffers, the
        host<->device copies inside the timed region (wall clock);
roofline the dominant kernel's FP64 pipe rate (algorithmic FP64 operations
        per launch / its event-timed launch duration) against the FP64 rate
        measured on the device in the same run;
cpu_baseline the CPU oracle on a bounded sample of the same path.

--impl reference times the oracle itself (the deliberately slow reference)
on the same workload.  Multi-GPU: one process per GPU, each tracks its own
path (seed + rank), no collective on the data path ("replicas"; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "corrector steps/s and paths/s (DD/QD) vs plain all-QD form; p50/p99 path latency"
UNIT = "corrector steps/s"


# ---- algorithmic FP64 work per unit (instruction tallies of the library's
#      primitives; every FP64 add, mul or fma is one operation)
#   cmul: complex product (D: a product and an FMA per part; DD: fused parts,
#         19 each; QD: one fused sum of two products per part, 235 each);
#         cadd: complex sum (2 real additions);
#   cmul_int: product by the integer exponent 1, 2 (exact doubling), 3;
#   mgs_unit: one (row, pivot, later column) of MGS, both parts of the dot-product
#         term and of the update (DD: 2 x (24 + 27); QD: 2 x (275 + 275));
#   mgs_sq: one row of a column norm (both parts); mgs_back: one back-substitution
#         term (both parts of an update)
OPS = {
    1: dict(cmul=4, cadd=2, cmul_int=(0, 0, 2, 2), c_abs2=2, mgs_unit=8, mgs_sq=2, mgs_back=4),
    2: dict(cmul=38, cadd=22, cmul_int=(0, 0, 4, 12), c_abs2=19,
            mgs_unit=102, mgs_sq=24, mgs_back=54),
    4: dict(cmul=470, cadd=2 * 94, cmul_int=(0, 0, 8, 154), c_abs2=235,
            mgs_unit=1100, mgs_sq=324, mgs_back=550),
}


# The many-path kernel's DD MGS runs its dot products and updates in fixed
# point (exact products and cross terms in FP64, the sums in integer units):
# 8 FP64 instructions per part of a dot-product term and 8 per part of an
# update, 2 x (8 + 8) per (row, pivot, later column).
MGS_UNIT_FIXED_DD = 32


def ad_ops(spec, L: int) -> int:
    """FP64 operations of the monomial AD kernel for one evaluation."""
    o = OPS[L]
    total = 0
    vp = spec.var_ptr
    for k in range(spec.M):
        es = spec.var_exp[vp[k]:vp[k + 1]]
        v = len(es)
        cf = int(np.sum(es >= 2))
        if v == 0:
            continue
        muls = cf + v + (v - 1) + max(v - 2, 0)
        total += muls * o["cmul"] + sum(o["cmul_int"][min(int(e), 3)] for e in es)
    return total


def sum_ops(spec, L: int) -> int:
    o = OPS[L]
    contrib = int(spec.M + spec.var_ptr[-1])          # values + partials
    return contrib * o["cadd"]


def mgs_ops(N: int, n: int, L: int, unit=None) -> int:
    """Per solve: the dot-product term and the update of every (row, pivot,
    later column) of [J | rhs], the column norms, the back substitution.
    `unit` overrides the FP64 operations per (row, pivot, later column)."""
    o = OPS[L]
    pairs = n * (n + 1) // 2                          # (k, j) with k < j <= n
    u = o["mgs_unit"] if unit is None else unit
    return pairs * N * u + (n + 1) * N * o["mgs_sq"] + (n * (n - 1) // 2) * o["mgs_back"]


# ---- clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- the CPU oracle on a bounded sample

def oracle_sample(wl, seconds: float = 15.0, max_pc_steps: int = 50):
    """Tracks the first predictor-corrector steps of the workload's path with
    the oracle (one thread) until about `seconds` have passed; returns
    (corrector steps, wall seconds, pc steps)."""
    import oracle
    oracle.build()
    f = oracle.System(wl.f, wl.L)
    x0, gam = wl.x0_soa(), wl.gamma_soa()
    steps = 1
    iters, wall, pcs = 0, 0.0, 0
    while True:
        p = dict(wl.params, max_steps=steps - 1)
        t0 = time.perf_counter()
        st, x, stats, _ = oracle.track(f, x0, gam, p)
        dt = time.perf_counter() - t0
        iters, wall, pcs = stats["newton_iters"], dt, stats["steps"]
        if dt >= seconds or steps >= max_pc_steps or st != oracle.MAXSTEPS:
            break
        # grow the sample geometrically toward the time budget
        per = dt / max(1, stats["steps"])
        steps = min(max_pc_steps, max(steps + 1, int(seconds / max(per, 1e-6))))
    return iters, wall, pcs


def _oracle_path_worker(job):
    """One independent dense64 path (its own seed) for the all-cores oracle
    figure: (corrector steps, wall seconds) of its bounded sample."""
    seed, prec, seconds = job
    sys.path.insert(0, ROOT)
    from paper_1501_06625_gb300 import synth
    it, wall, _ = oracle_sample(synth.dense64(seed, prec), seconds=seconds)
    return it, wall


def oracle_all_cores(seed: int, prec: str, seconds: float, cores: int | None = None) -> dict:
    """The oracle with one independent path per host core (the dense64 system
    of seeds seed .. seed + cores - 1), each a bounded sample of about
    `seconds`; the figure is all corrector steps over the slowest worker's
    wall time.  Worker processes are started with spawn: a process forked
    after the first GPU call can hang."""
    import multiprocessing as mp
    if not cores:
        try:
            cores = len(os.sched_getaffinity(0))        # the cores this process may use
        except AttributeError:
            cores = os.cpu_count() or 1
    jobs = [(seed + i, prec, seconds) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_path_worker, jobs)
    its = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": its / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one dense64 {prec} path per core (seeds {seed}..{seed + cores - 1}), "
                      f"each its first predictor-corrector steps for about {seconds:g} s"}


def run_reference(args):
    from paper_1501_06625_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = synth.dense64(args.seed, args.prec)
    per_step = []
    total_iters = 0
    budget = max(5.0, 150.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        iters, wall, pcs = oracle_sample(wl, seconds=budget, max_pc_steps=12)
        if i >= args.warmup:
            per_step.append(wall)
            total_iters += iters
    value = total_iters / sum(per_step)
    sample = f"first {pcs} predictor-corrector steps of the {wl.name} path per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(per_step) / len(per_step), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "dd", "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.n, "terms_per_poly": 64, "vars_per_term": 16,
                       "exponents": [1, 2, 3], "homotopy": "total-degree, k=1", "seed": args.seed},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- the library

SEGMENT = {2: 50, 4: 20}       # predictor-corrector steps per bench step
CONTROL = {"control": 0}       # 1: host-side step control (for profiling runs)


# DRAM bytes (read + write) of one k_mgs<DD> launch on the dense64 DD system,
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the
# current kernel: the 64 x 65 matrix and the projection coefficients, read once.
MGS_DENSE64_DD_TRAFFIC = 279040


def seg_params(wl):
    return dict(wl.params, max_steps=SEGMENT[wl.L] - 1, control=CONTROL["control"])


def track_leg(libph, ctx, f, wl, dev, steps, warmup, torch, flush, events=True):
    """Tracks the path `warmup + steps` times with device-resident buffers;
    returns per-step ms and stats of the timed steps."""
    L, n = wl.L, wl.n
    x0 = torch.tensor(wl.x0_soa(), dtype=torch.float64, device=dev)
    gam = torch.tensor(wl.gamma_soa(), dtype=torch.float64, device=dev)
    xo = torch.empty_like(x0)
    stream = torch.cuda.current_stream(dev)
    ms, stats = [], []
    for i in range(warmup + steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, sd, _ = libph.ph_track_path(ctx.h, f, None, gam, x0, seg_params(wl), xo)
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
            stats.append(sd)
    return ms, stats, xo


def e2e_leg(libph, ctx, f, wl, steps, torch):
    """The same call with pinned host buffers (copies inside the call)."""
    x0 = torch.tensor(wl.x0_soa(), dtype=torch.float64).pin_memory()
    gam = torch.tensor(wl.gamma_soa(), dtype=torch.float64).pin_memory()
    xo = torch.empty_like(x0).pin_memory()
    walls, iters = [], 0
    for _ in range(steps):
        t0 = time.perf_counter()
        st, sd, _ = libph.ph_track_path(ctx.h, f, None, gam, x0, seg_params(wl), xo)
        walls.append(time.perf_counter() - t0)
        iters += sd["newton_iters"]
    h2d = x0.numel() * 8 + gam.numel() * 8
    d2h = xo.numel() * 8
    return iters / sum(walls), h2d, d2h


def batch_starts(wl, count, seed=7):
    """Total-degree start solutions exp(2 pi i m_i / d_i) (rounded to double):
    the all-ones root first, then random choices of the m_i."""
    d = wl.f.degrees()
    rng = np.random.default_rng(seed)
    out = np.zeros((count, wl.L, 2, wl.n))
    for p in range(count):
        ms = np.zeros(wl.n, dtype=int) if p == 0 else rng.integers(0, d)
        z = np.exp(2j * np.pi * ms / d)
        out[p, 0, 0], out[p, 0, 1] = z.real, z.imag
    return out


def batched_run(libph, ctx, f, wl, x0, params, torch, dev, flush):
    """One ph_track_paths call over device-resident start points, timed with
    CUDA events on the library's stream; returns (ms, stats)."""
    stream = torch.cuda.current_stream(dev)
    bx0 = torch.tensor(x0, dtype=torch.float64, device=dev)
    bxo = torch.empty_like(bx0)
    bgam = torch.tensor(wl.gamma_soa(), dtype=torch.float64, device=dev)
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats, _ = libph.ph_track_paths(ctx.h, f, None, bgam, bx0, params, bxo)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), stats


def precision_leg(libph, synth, ctx, torch, dev, flush, seed, paths):
    """The precision form against the plain form on the same batch of paths
    (distinct total-degree start roots, the same segment of adaptive steps,
    the same tolerances on every corrector): lin_prec 0 (all DD/QD), 1 (Newton
    systems in double) and 3 (single where it costs no convergence, else
    double); in QD also lin_prec 1 with one Newton iteration more, which the
    double corrector's linear tail near 1e-52 needs.  Workload: precision128
    (n = 128, coefficient moduli over 12 decades per equation, planted root),
    first step size 1e-3 and 5 (DD) / 6 (QD) Newton iterations, where the
    plain form accepts every step of its segment."""
    out = {}
    cases = [("dd", 6, 5, ((0, 0), (1, 0), (3, 0))),
             ("qd", 3, 6, ((0, 0), (1, 0), (3, 0), (1, 1)))]
    for prec, seg, mn, runs in cases:
        wl = synth.precision128(seed, prec)[0]
        f = ctx.load(wl.f, wl.L)
        x0 = batch_starts(wl, paths)
        row = {"paths": paths, "segment_steps": seg, "max_dt": 1e-3, "max_newton": mn}
        base = None
        for lin, extra in runs:
            params = dict(wl.params, max_steps=seg - 1, max_dt=1e-3, max_newton=mn + extra,
                          lin_prec=lin)
            ms, st = batched_run(libph, ctx, f, wl, x0, params, torch, dev, flush)
            it = sum(x["newton_iters"] for x in st)
            acc = sum(x["accepted"] for x in st)
            r = {"ms": ms, "corrector_steps_per_s": it / (ms * 1e-3),
                 "accepted_steps_per_s": acc / (ms * 1e-3), "accepted_steps": acc,
                 "segments_per_s": paths / (ms * 1e-3),
                 "solves_f64": sum(x["solves_f64"] for x in st),
                 "solves_f32": sum(x["solves_f32"] for x in st),
                 "escalated": sum(x["escalated"] for x in st)}
            conds = [x["cond"] for x in st if lin and np.isfinite(x["cond"]) and x["cond"] > 0]
            if conds:
                r["cond_estimate_median"] = float(np.median(conds))
                r["cond_estimate_max"] = float(np.max(conds))
            if base is None:
                base = r
            else:
                r["accepted_steps_vs_plain"] = r["accepted_steps_per_s"] / base["accepted_steps_per_s"]
            row[f"lin{lin}" + (f"_newton+{extra}" if extra else "")] = r
        out[f"precision128_{prec}"] = row
    return out


def precision_path_leg(libph, synth, ctx, torch, dev, flush, seed):
    """The precision form in the single-path tracker: one precision128 path
    (n = 128, coefficient moduli over 12 decades per equation) over the same
    segment of adaptive steps as the many-path comparison, plain (lin_prec 0,
    every Newton system in DD/QD) against lin_prec 1 (Newton systems in
    double, residual and update in DD/QD; in QD also with one Newton iteration
    more).  Each run is timed with CUDA events around one ph_track_path call
    after an untimed call that builds its step graph; the end points of the
    two forms are compared (their corrector tolerances are the same)."""
    out = {}
    cases = [("dd", 6, 5, ((0, 0), (1, 0))), ("qd", 3, 6, ((0, 0), (1, 0), (1, 1)))]
    stream = torch.cuda.current_stream(dev)
    for prec, seg, mn, runs in cases:
        wl = synth.precision128(seed, prec)[0]
        f = ctx.load(wl.f, wl.L)
        x0 = torch.tensor(batch_starts(wl, 1)[0], dtype=torch.float64, device=dev)
        gam = torch.tensor(wl.gamma_soa(), dtype=torch.float64, device=dev)
        row = {"segment_steps": seg, "max_dt": 1e-3, "max_newton": mn}
        base = None
        for lin, extra in runs:
            params = dict(wl.params, max_steps=seg - 1, max_dt=1e-3, max_newton=mn + extra,
                          lin_prec=lin)
            xo = torch.empty_like(x0)
            libph.ph_track_path(ctx.h, f, None, gam, x0, params, xo)      # builds the graph
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, sd, _ = libph.ph_track_path(ctx.h, f, None, gam, x0, params, xo)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            r = {"status": int(st), "ms": ms, "accepted_steps": sd["accepted"],
                 "newton_iters": sd["newton_iters"], "solves_f64": sd["solves_f64"],
                 "escalated": sd["escalated"],
                 "ms_per_accepted_step": ms / max(1, sd["accepted"])}
            if lin:
                r["cond_estimate"] = sd["cond"]
            x = xo.cpu().numpy()
            if base is None:
                base, xb = r, x
            else:
                r["accepted_steps_vs_plain"] = (base["ms_per_accepted_step"]
                                                / r["ms_per_accepted_step"])
                # limb by limb (the leading limbs agree), summed from the last
                dd = (x - xb)[::-1].sum(axis=0)
                r["end_point_diff_vs_plain"] = float(np.abs(dd[0] + 1j * dd[1]).max())
            row[f"lin{lin}" + (f"_newton+{extra}" if extra else "")] = r
        out[f"precision128_{prec}_single_path"] = row
    return out


# The paper's summation-kernel times on its K20C (Section 3.3, the tables for
# cyclic 128- and 352-roots, ms per evaluation at the best number of threads
# per sum): context, not targets.
PAPER_CYCLIC_SUM_MS = {(128, 1): 0.34, (128, 2): 0.53, (128, 4): 1.35,
                       (352, 1): 6.32, (352, 2): 9.69, (352, 4): 24.61}


def cyclic_leg(libph, synth, ctx, torch, dev, peak):
    """Cyclic n-roots (Section 4.2, Eq. (10)), n = 128 and 352, in D, DD and QD:
    one corrector iteration's kernels at a random point of the unit torus
    (t = 0.5, total-degree homotopy), event-timed on the library's stream: ms per
    evaluation of h and its Jacobian (power table + monomial AD + summation), of
    the summation alone (the paper's own timing of this system; also with each
    number of lanes per output, 1 to 32, as the paper's tables vary its threads
    per sum) and per MGS solve, and the AD kernel's fraction of the measured
    FP64 rate."""
    out = {}
    for n in (128, 352):
        spec = synth.cyclic_system(n)
        rng = np.random.default_rng(n)
        z = np.exp(2j * np.pi * rng.random(n))
        for L in (1, 2, 4):
            f = ctx.load(spec, L)
            xs = np.zeros((L, 2, n))
            xs[0, 0], xs[0, 1] = z.real, z.imag
            x = torch.tensor(xs, dtype=torch.float64, device=dev)
            gam = torch.zeros((L, 2), dtype=torch.float64, device=dev)
            gam[0, 0], gam[0, 1] = 0.6, 0.8
            tl = torch.zeros(L, dtype=torch.float64, device=dev)
            tl[0] = 0.5
            kms = libph.ph_profile_newton(ctx.h, f, None, gam, 1, tl, x, 3 if n > 200 else 10)
            lanes, by_lanes = libph.ph_sum_lanes(ctx.h, f)
            ev = kms[0] + kms[1] + kms[2]
            ad = ad_ops(spec, L)
            r = {"eval_ms": ev, "mgs_ms": kms[3], "kernel_ms": dict(zip(
                     ["prep", "monomial_ad", "summation", "mgs"], kms)),
                 "monomials": int(spec.M),
                 "ad_frac_of_fp64_peak": ad / (kms[1] * 1e-3) / 1e9 / peak,
                 "summation_ms": kms[2],
                 "summation_lanes": lanes,
                 "summation_ms_by_lanes": dict(zip(["1", "2", "4", "8", "16", "32"], by_lanes)),
                 "paper_k20c_summation_ms": PAPER_CYCLIC_SUM_MS[(n, L)],
                 "summation_vs_paper_k20c": PAPER_CYCLIC_SUM_MS[(n, L)] / kms[2]}
            out[f"cyclic{n}_{ {1: 'd', 2: 'dd', 4: 'qd'}[L] }"] = r
            ctx.free(f)
    return out


# The paper's Table 8: one monodromy path of cyclic n-roots on its Tesla K20C,
# per (n, limbs): success (1) or failure (0), predictor-corrector steps m, CPU
# and GPU seconds.  Context, not targets.
PAPER_CYCLIC_PATH = {(16, 1): (1, 32, 0.00, 0.03), (16, 2): (1, 20, 0.04, 0.06),
                     (16, 4): (1, 32, 0.48, 0.52), (64, 1): (0, 987, 4.48, 4.15),
                     (64, 2): (1, 225, 22.94, 2.57), (64, 4): (1, 987, 229.99, 17.93),
                     (144, 1): (0, 214, 12.58, 2.67), (144, 2): (0, 1500, 1487.86, 61.59),
                     (144, 4): (1, 214, 15898.67, 479.18)}


def monodromy_leg(libph, synth, ctx, torch, dev, seed, segment):
    """One monodromy path on cyclic n-roots, n = m^2 = 16, 64, 144 (Section
    4.2; the paper's runs of Table 8): the (m-1)-dimensional solution set cut
    by m - 1 random hyperplanes that move to m - 1 others, N = n + m - 1
    equations corrected by least squares, from a start point of Backelin's
    family (synth.cyclic_monodromy).  D, DD and QD with 3 / 5 / 6 Newton
    iterations per step and the library's default tolerances.  Whole paths
    for n <= 64; at n = 144 the first `segment` steps.  Each run is timed with
    CUDA events around one ph_track_path call, after an untimed call that
    builds its step graph (except the n = 64 QD path, timed in one call).
    Compared with the paper per predictor-corrector step and, for whole paths,
    per path: the paper's tolerances and Newton budget are not stated, so the
    step counts differ.  The paper's homotopy {f = 0, alpha (1-t) L + t K = 0}:
    F = [f; K], G = [0; L] with the cyclic rows held fixed (fixed_rows), so f
    is evaluated once per iteration."""
    out = {}
    newton = {1: 3, 2: 5, 4: 6}
    stream = torch.cuda.current_stream(dev)
    for n in (16, 64, 144):
        F, G, gam, x0 = synth.cyclic_monodromy(seed, n)
        for L, name in ((1, "d"), (2, "dd"), (4, "qd")):
            whole = n <= 64
            # a warm-up call (same parameters: it builds the step graph) where
            # it is cheap; the QD path at n = 64 is timed in one call, the
            # graph's construction (tens of ms) inside its seconds
            warm = not (n == 64 and L == 4)
            params = synth.default_params(L, max_newton=newton[L], fixed_rows=1,
                                          max_steps=5000 if whole else segment - 1)
            f, g = ctx.load(F, L), ctx.load(G, L)
            xs = np.zeros((L, 2, n))
            xs[0, 0], xs[0, 1] = x0.real, x0.imag
            gs = np.zeros((L, 2))
            gs[0] = [gam.real, gam.imag]
            dx0 = torch.tensor(xs, dtype=torch.float64, device=dev)
            dg = torch.tensor(gs, dtype=torch.float64, device=dev)
            xo = torch.empty_like(dx0)
            if warm:
                libph.ph_track_path(ctx.h, f, g, dg, dx0, params, xo)    # builds the graph
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, sd, _ = libph.ph_track_path(ctx.h, f, g, dg, dx0, params, xo)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            # one corrector iteration's kernels at the path's end point
            tl = torch.zeros(L, dtype=torch.float64, device=dev)
            tl[0] = sd["t_final"]
            kms = libph.ph_profile_newton(ctx.h, f, g, dg, 1, tl, xo, 3)
            ps, pm, pcpu, pgpu = PAPER_CYCLIC_PATH[(n, L)]
            per_step = ms / max(1, sd["steps"])
            out[f"cyclic{n}_{name}"] = {
                "N": F.N, "n": n, "whole_path": whole, "graph_built_in_timing": not warm,
                "status": int(st),
                "t_final": sd["t_final"], "steps": sd["steps"], "accepted": sd["accepted"],
                "newton_iters": sd["newton_iters"], "ms": ms, "ms_per_step": per_step,
                "ms_per_newton_iter": ms / max(1, sd["newton_iters"]),
                "kernel_ms": dict(zip(["prep", "monomial_ad", "summation", "mgs"], kms)),
                "paper_k20c": {"success": ps, "steps": pm, "gpu_s": pgpu, "cpu_s": pcpu,
                               "ms_per_step": 1e3 * pgpu / pm},
                "per_step_vs_paper": (1e3 * pgpu / pm) / per_step}
            if whole and st == libph.PH_OK:
                out[f"cyclic{n}_{name}"]["per_path_vs_paper"] = 1e3 * pgpu / ms
            if L == 4 and n >= 64:
                # the precision form on the same path (Newton systems in double,
                # residual and update in QD); it leaves the rest of the path to QD
                # once a failed double corrector contracted only linearly
                xm = torch.empty_like(dx0)
                e0.record(stream)
                st2, sd2, _ = libph.ph_track_path(ctx.h, f, g, dg, dx0, dict(params, lin_prec=1), xm)
                e1.record(stream)
                e1.synchronize()
                ms2 = e0.elapsed_time(e1)
                r2 = {"status": int(st2), "t_final": sd2["t_final"], "steps": sd2["steps"],
                      "accepted": sd2["accepted"], "newton_iters": sd2["newton_iters"],
                      "solves_f64": sd2["solves_f64"], "escalated": sd2["escalated"],
                      "wp_rest": sd2["wp_rest"], "ms": ms2,
                      "ms_per_step": ms2 / max(1, sd2["steps"]), "graph_built_in_timing": True}
                if whole and st2 == libph.PH_OK:
                    dd = (xm.cpu().numpy() - xo.cpu().numpy())[::-1].sum(axis=0)
                    r2["end_point_diff_vs_plain"] = float(np.abs(dd[0] + 1j * dd[1]).max())
                    r2["vs_plain"] = ms / ms2
                out[f"cyclic{n}_{name}"]["precision_form"] = r2
            ctx.free(f)
            ctx.free(g)
    return out


def monodromy_loops_leg(libph, synth, ctx, seed, loops, single):
    """Many monodromy loops at once, the form the paper's degree computation
    needs (each loop a path with its own random slices and constant): `loops`
    independent cyclic n-roots monodromy paths (synth.cyclic_monodromy with
    seeds seed*1000 + i, each its own pair of loaded systems), submitted at once
    to the serving loop (one persistent block per path, ph_server_*), whole
    paths, the same Newton budget and tolerances as the single-path leg.
    Against `single`, the single-path form's ms per path of the first loop."""
    out = {}
    newton = {2: 5, 4: 6}
    for n, L, name in ((16, 4, "qd"), (16, 2, "dd")):
        key = f"cyclic{n}_{name}"
        if single is None or key not in single:
            continue
        params = synth.default_params(L, max_newton=newton[L], max_steps=5000, fixed_rows=1)
        jobs = []
        for i in range(loops):
            F, G, gam, x0 = synth.cyclic_monodromy(seed * 1000 + i, n)
            f, g = ctx.load(F, L), ctx.load(G, L)
            xs = np.zeros((L, 2, n))
            xs[0, 0], xs[0, 1] = x0.real, x0.imag
            gs = np.zeros((L, 2))
            gs[0] = [gam.real, gam.imag]
            jobs.append((f, g, gs, xs))
        srv = libph.ph_server_create(ctx.h, max_n=n, pool_bytes=8 << 30, queue_cap=2 * loops)
        try:
            t0 = time.perf_counter()
            ids = [libph.ph_server_submit(ctx.h, srv, f, g, gs, xs, params)
                   for f, g, gs, xs in jobs]
            stats = [libph.ph_server_wait(ctx.h, srv, j, 600000)[0] for j in ids]
            wall = time.perf_counter() - t0
        finally:
            libph.ph_server_destroy(srv)
        for f, g, _, _ in jobs:
            ctx.free(f)
            ctx.free(g)
        ok = sum(1 for x in stats if x["status"] == libph.PH_OK)
        rate = loops / wall
        one = 1e3 / single[key]["ms"]
        out[key] = {"loops": loops, "wall_s": wall, "paths_per_s": rate, "succeeded": ok,
                    "steps": sum(x["steps"] for x in stats),
                    "longest_path_steps": max(x["steps"] for x in stats),
                    "newton_iters": sum(x["newton_iters"] for x in stats),
                    "single_path_per_s": one, "vs_single_path": rate / one}
    return out


# The paper's Table 5: degrees of the cyclic n-roots solution sets (n = m^2)
PAPER_CYCLIC_DEGREE = {16: 4, 64: 8, 144: 12}


def monodromy_degree_leg(synth, ctx, seed, sizes):
    """The degree of the cyclic n-roots solution set through its start point,
    computed as the paper does (Section 4.2, Table 5): rounds of monodromy
    loops (out to the slices K and back to L, each loop with its own alpha and
    beta) through the serving loop, from the points found so far, until a
    round adds no point.  Double-double, 5 Newton iterations per step; wall
    clock around the whole computation.  The points found are checked against
    the family's points on the slices computed from its linear
    parametrization (monodromy.family_points_on_slices)."""
    from paper_1501_06625_gb300 import monodromy
    out = {}
    for n, per_round in sizes:
        m = int(round(np.sqrt(n)))
        loop = synth.cyclic_monodromy_loop(seed, n)
        params = synth.default_params(2, max_newton=5, max_steps=5000)
        t0 = time.perf_counter()
        res = monodromy.loops(ctx, loop, 2, params, rounds=12, per_round=per_round,
                              seed=seed + 7, patience=2)
        wall = time.perf_counter() - t0
        G = loop["out"][1]
        c = G.coeff.reshape(m - 1, n + 1)
        ref = monodromy.family_points_on_slices(
            m, c[:, :n], c[:, n] + G.coeff_lo.reshape(m - 1, n + 1)[:, n])
        match = [float(np.abs(ref - (q[0, 0] + 1j * q[0, 1])[None, :]).max(axis=1).min())
                 for q in res["points"]]
        out[f"cyclic{n}_dd"] = {
            "degree_found": len(res["points"]), "paper_degree": PAPER_CYCLIC_DEGREE[n],
            "found_after_each_round": res["found"], "loops": res["loops"],
            "failed_paths": res["failed"], "paths": res["paths"],
            "newton_iters": res["newton_iters"], "wall_s": wall,
            "max_distance_to_parametrized_points": max(match)}
    return out


def serve_leg(libph, synth, ctx, nreq, seed, lin=0, seq_rate=None, sweep_requests=48):
    """A stream of path-tracking requests through the continuous-batching loop
    (ph_server_*).  A pool of 16 systems per (recipe, precision): n =
    round(exp(U[ln 16, ln 64])); the dense recipe (n terms per polynomial over
    min(16, n) variables, exponents {1,2,3}) or the sparse one (a linear term
    plus 3 two-variable terms, exponents {1,2}) with probability 1/2 each.  A
    request: double-double with probability 0.7, else quad-double; a system of
    the pool; a random total-degree start root; the first 20 predictor-corrector
    steps (adaptive).  Closed loop first (all submitted at once: the capacity),
    then Poisson arrivals at 0.8 x that capacity (latency under load), then
    Poisson arrivals of the first `sweep_requests` requests at 0.5, 1 and 2 x
    the sequential capacity.  The sequential figure tracks a sample of the
    same requests one by one with ph_track_path (measured first when not
    given)."""
    rng = np.random.default_rng(seed + 1000)
    systems = {}
    reqs = []
    for _ in range(nreq):
        dense = bool(rng.random() < 0.5)
        L = 2 if rng.random() < 0.7 else 4
        idx = int(rng.integers(0, 16))
        key = (dense, L, idx)
        if key not in systems:
            srng = synth.Rng(seed * 7919 + 131 * idx + 17 * L + int(dense))
            n = int(round(np.exp(srng.uniform() * (np.log(64) - np.log(16)) + np.log(16))))
            spec = (synth.dense_system(srng, n, n, min(16, n), (1, 2, 3)) if dense
                    else synth.sparse_system(srng, n))
            g = srng.unit_complex()
            gam = np.zeros((L, 2))
            gam[0] = [g.real, g.imag]
            systems[key] = (ctx.load(spec, L), spec, gam, L)
        f, spec, gam, L = systems[key]
        d = np.array(spec.degrees())
        z = np.exp(2j * np.pi * rng.integers(0, d) / d)
        x0 = np.zeros((L, 2, spec.n))
        x0[0, 0], x0[0, 1] = z.real, z.imag
        reqs.append((f, gam, x0, synth.default_params(L, max_steps=19, lin_prec=lin)))

    k = min(16, nreq)
    if seq_rate is None:                        # the plain single-path form
        t0 = time.perf_counter()
        for f, gam, x0, params in reqs[:k]:
            libph.ph_track_path(ctx.h, f, None, gam, x0, dict(params, lin_prec=0),
                                np.zeros_like(x0))
        seq_rate = k / (time.perf_counter() - t0)

    srv = libph.ph_server_create(ctx.h, max_n=64, pool_bytes=8 << 30, queue_cap=1024)
    try:
        def run(arrivals):
            ids = []
            t0 = time.perf_counter()
            for (f, gam, x0, params), ta in zip(reqs, arrivals):
                while time.perf_counter() - t0 < ta:
                    pass
                ids.append(libph.ph_server_submit(ctx.h, srv, f, None, gam, x0, params))
            lats, iters = [], 0
            for jid in ids:
                st, lat = libph.ph_server_wait(ctx.h, srv, jid, 120000)
                lats.append(lat)
                iters += st["newton_iters"]
            return time.perf_counter() - t0, lats, iters

        run([0.0] * min(64, nreq))                       # warm-up
        wall, lats, iters = run([0.0] * nreq)
        cap = nreq / wall
        arrivals = np.cumsum(rng.exponential(1.0 / (0.8 * cap), nreq))
        wall2, lats2, _ = run(list(arrivals))
        # offered loads relative to what sequential single-path tracking sustains
        m = min(sweep_requests, nreq)
        sweep = {}
        for mult in (0.5, 1.0, 2.0):
            arr = np.cumsum(rng.exponential(1.0 / (mult * seq_rate), m))
            w3, l3, _ = run(list(arr))
            sweep[f"{mult:g}x"] = {"offered_per_s": mult * seq_rate, "paths_per_s": m / w3,
                                   "p50_ms": float(np.percentile(l3, 50)),
                                   "p99_ms": float(np.percentile(l3, 99))}
        info = libph.ph_server_info(srv)
    finally:
        libph.ph_server_destroy(srv)

    return {"requests": nreq, "lin_prec": lin,
            "mix": "n log-uniform in [16,64]; dense/sparse 50/50; DD/QD 70/30; "
                   "20 adaptive steps per request; 16 systems per recipe and precision",
            "closed_loop": {"paths_per_s": cap, "corrector_steps_per_s": iters / wall,
                            "p50_ms": float(np.percentile(lats, 50)),
                            "p99_ms": float(np.percentile(lats, 99))},
            "poisson_0.8": {"offered_per_s": 0.8 * cap, "paths_per_s": nreq / wall2,
                            "p50_ms": float(np.percentile(lats2, 50)),
                            "p99_ms": float(np.percentile(lats2, 99))},
            "poisson_vs_sequential_capacity": {"requests_per_rate": m, "rates": sweep},
            "sequential_single_path": {"paths_per_s": seq_rate, "sample": k,
                                       "form": "ph_track_path, all DD/QD"},
            "vs_sequential": cap / seq_rate,
            "kernel_launches": info["kernel_launches"]}


def _planted_worker(job):
    """One planted dense64 workload (its generation is pure Python: spread over
    spawned worker processes)."""
    seed, prec = job
    sys.path.insert(0, ROOT)
    from paper_1501_06625_gb300 import synth
    wl, xs = synth.dense64_planted(seed, prec)
    return wl, xs


def planted_workloads(seeds, prec, workers=16):
    import multiprocessing as mp
    jobs = [(s, prec) for s in seeds]
    if len(jobs) <= 2:
        return [_planted_worker(j) for j in jobs]
    with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
        return pool.map(_planted_worker, jobs)


def _soa(z, L):
    out = np.zeros((L, 2, len(z)))
    out[0, 0], out[0, 1] = np.real(z), np.imag(z)
    return out


def _err_vs(x, xs):
    """max_i |x_i - x*_i| of an [L][2][n] end point against a double vector x*
    (limb by limb from the smallest)."""
    d = x.copy()
    d[0, 0] -= np.real(xs)
    d[0, 1] -= np.imag(xs)
    d = d[::-1].sum(0)
    return float(np.abs(d[0] + 1j * d[1]).max())


def whole_path_leg(libph, synth, ctx, torch, dev, seed, npaths_dd, nsingle, qd_paths):
    """Whole solution paths of the dense n = 64 workload (the headline system's shape) to
    t = 1, each checked against its planted root.

    The all-ones start root's total-degree path does not end at a regular root
    for these systems (no seed tried does within thousands of steps), so every
    path here is planted: synth.dense64_planted adds the constant term that
    makes f(x*) = 0 exactly; tracking x* backwards (start system f, target the
    total-degree system, gamma' = 1/gamma) lands on a start root of
    x_i^{d_i} = 1, and the forward path from that root -- a path of the
    dense64 total-degree homotopy -- ends at x*.  Corrector tolerance on the way
    tol_path = 1e-8, at t = 1 the working precision (1e-24 DD, 1e-52 QD).

    DD: `npaths_dd` systems; the backward paths run through the serving loop
    (untimed preparation).  Timed: the plain single-path form (ph_track_path,
    all DD) on the first `nsingle` paths, one by one (CUDA events); then all
    paths at once through the serving loop, plain (lin_prec 0) and in the
    precision form (lin_prec 3).  QD: `qd_paths` systems, single path.  A path
    counts as successful when it reaches t = 1 within 1e-20 (DD) / 1e-48 (QD)
    of x*."""
    stream = torch.cuda.current_stream(dev)
    out = {}
    for prec, count in (("dd", npaths_dd), ("qd", qd_paths)):
        if count <= 0:
            continue
        L = 2 if prec == "dd" else 4
        tol_ok = 1e-20 if L == 2 else 1e-48
        t0 = time.perf_counter()
        wls = planted_workloads([seed + 100 + i for i in range(count)], prec)
        gen_s = time.perf_counter() - t0
        loaded = []
        for wl, xs in wls:
            f = ctx.load(wl.f, L)
            G = ctx.load(synth.total_degree_start(wl.f), L)
            loaded.append((wl, xs, f, G))
        base = dict(synth.default_params(L), max_steps=4000, tol_path=1e-8,
                    max_newton=3 if L == 2 else 5)
        # backward paths: start roots (untimed); many DD paths through the
        # serving loop, a few QD paths one by one on the whole GPU
        t0 = time.perf_counter()
        starts = []

        def start_of(wl, xl):
            return _soa(synth.nearest_start_root(wl.f, xl[0, 0] + 1j * xl[0, 1]), L)

        if count > 16:
            srv = libph.ph_server_create(ctx.h, max_n=64, pool_bytes=8 << 30, queue_cap=1024)
            try:
                ids = []
                for wl, xs, f, G in loaded:
                    gb = _soa([1.0 / wl.gamma], L).reshape(L, 2)
                    ids.append(libph.ph_server_submit(ctx.h, srv, G, f, gb, _soa(xs, L), base))
                for (wl, xs, f, G), jid in zip(loaded, ids):
                    xl = np.zeros((L, 2, 64))
                    st, _ = libph.ph_server_wait(ctx.h, srv, jid, 600000, x_out=xl)
                    starts.append(start_of(wl, xl) if st["status"] == libph.PH_OK else None)
            finally:
                libph.ph_server_destroy(srv)
        else:
            for wl, xs, f, G in loaded:
                gb = _soa([1.0 / wl.gamma], L).reshape(L, 2)
                xl = np.zeros((L, 2, 64))
                st, _, _ = libph.ph_track_path(ctx.h, G, f, gb, _soa(xs, L), base, xl)
                starts.append(start_of(wl, xl) if st == libph.PH_OK else None)
        prep_s = time.perf_counter() - t0
        idx = [i for i, s0 in enumerate(starts) if s0 is not None]
        row = {"systems": count, "start_roots_found": len(idx), "generation_s": gen_s,
               "backward_s": prep_s, "params": {"tol_path": 1e-8, "max_newton": base["max_newton"],
                                                "max_dt": base["max_dt"]}}
        # the plain single-path form, one path at a time
        single = []
        for i in idx[:nsingle]:
            wl, xs, f, G = loaded[i]
            x0 = torch.tensor(starts[i], device=dev)
            gam = torch.tensor(wl.gamma_soa(), device=dev)
            xo = torch.empty_like(x0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, sd, _ = libph.ph_track_path(ctx.h, f, None, gam, x0, base, xo)
            e1.record(stream)
            e1.synchronize()
            err = _err_vs(xo.cpu().numpy(), xs)
            single.append({"ms": e0.elapsed_time(e1), "status": libph.STATUS_NAMES[st],
                           "steps": sd["steps"], "accepted": sd["accepted"],
                           "newton_iters": sd["newton_iters"], "err_vs_planted": err,
                           "ok": bool(st == libph.PH_OK and err <= tol_ok)})
        if single:
            ms = [r["ms"] for r in single]
            row["single_path"] = {
                "form": "ph_track_path, all " + prec.upper(), "paths": len(single),
                "successful": sum(r["ok"] for r in single),
                "paths_per_s": len(single) / (sum(ms) / 1e3),
                "corrector_steps_per_s": sum(r["newton_iters"] for r in single) / (sum(ms) / 1e3),
                "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                "steps_median": float(np.median([r["steps"] for r in single])),
                "max_err_vs_planted": max(r["err_vs_planted"] for r in single),
                "paths": single if len(single) <= 4 else None}
        # all paths at once through the serving loop
        if L == 2 and len(idx) > nsingle:
            for lin in (0, 3):
                params = dict(base, lin_prec=lin)
                srv = libph.ph_server_create(ctx.h, max_n=64, pool_bytes=8 << 30, queue_cap=1024)
                try:
                    t0 = time.perf_counter()
                    ids = [libph.ph_server_submit(ctx.h, srv, loaded[i][2], None,
                                                  loaded[i][0].gamma_soa(), starts[i], params)
                           for i in idx]
                    lats, iters, oks, errs, f32, f64 = [], 0, 0, [], 0, 0
                    for i, jid in zip(idx, ids):
                        xe = np.zeros((L, 2, 64))
                        st, lat = libph.ph_server_wait(ctx.h, srv, jid, 900000, x_out=xe)
                        e = _err_vs(xe, loaded[i][1])
                        lats.append(lat)
                        errs.append(e)
                        iters += st["newton_iters"]
                        f32 += st["solves_f32"]
                        f64 += st["solves_f64"]
                        oks += int(st["status"] == libph.PH_OK and e <= tol_ok)
                    wall = time.perf_counter() - t0
                finally:
                    libph.ph_server_destroy(srv)
                r = {"form": "serving loop, " + ("all DD" if lin == 0 else
                                                 "precision form (lin_prec 3)"),
                     "paths": len(idx), "successful": oks, "wall_s": wall,
                     "paths_per_s": len(idx) / wall, "corrector_steps_per_s": iters / wall,
                     "p50_ms": float(np.percentile(lats, 50)),
                     "p99_ms": float(np.percentile(lats, 99)),
                     "max_err_vs_planted": float(max(errs)),
                     "solves_f32": f32, "solves_f64": f64}
                if "single_path" in row:
                    r["paths_per_s_vs_single_path"] = r["paths_per_s"] / row["single_path"]["paths_per_s"]
                row["served_lin%d" % lin] = r
        for wl, xs, f, G in loaded:
            ctx.free(f)
            ctx.free(G)
        out[f"dense64_planted_{prec}"] = row
    return out


def sparse512_leg(libph, synth, ctx, torch, dev, seed, steps):
    """The very sparse n = 512 system in QD, total-degree homotopy
    from the all-ones root, adaptive steps (5 Newton iterations, path
    tolerance 1e-8, QD at t = 1): the first `steps` predictor-corrector steps
    through ph_track_path (the MGS solve of the 512 x 512 Jacobian dominates),
    CUDA events."""
    stream = torch.cuda.current_stream(dev)
    wl = synth.sparse512(seed, "qd")
    f = ctx.load(wl.f, wl.L)
    x0 = torch.tensor(wl.x0_soa(), device=dev)
    gam = torch.tensor(wl.gamma_soa(), device=dev)
    xo = torch.empty_like(x0)
    params = dict(wl.params, max_steps=steps - 1, max_newton=5, tol_path=1e-8)
    libph.ph_track_path(ctx.h, f, None, gam, x0, dict(params, max_steps=0), xo)   # graph, tuning
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, sd, _ = libph.ph_track_path(ctx.h, f, None, gam, x0, params, xo)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    kind, size, vms = libph.ph_mgs_variant(ctx.h, 4, 512, 512)
    ctx.free(f)
    return {"workload": wl.name, "steps": sd["steps"], "accepted": sd["accepted"],
            "rejected": sd["rejected"], "newton_iters": sd["newton_iters"],
            "t_final": sd["t_final"], "status": libph.STATUS_NAMES[st], "ms": ms,
            "corrector_steps_per_s": sd["newton_iters"] / (ms * 1e-3),
            "ms_per_corrector_step": ms / max(1, sd["newton_iters"]),
            "mgs_variant": {"kind": libph.MGS_KINDS[kind], "size": size,
                            "ms_grid_cluster_tiled": vms}}


def sparse512_whole_path(libph, synth, ctx, torch, dev, seed, max_steps=4000):
    """One whole path of the sparse n = 512 QD homotopy to t = 1.  The
    all-ones start root's path need not end at a regular root, so the system
    is planted (synth.sparse512_planted: the sparse recipe plus the constant
    terms that make f(x*) = 0 exactly).  x* is tracked backwards (start system
    f, target the total-degree system, gamma' = 1/gamma; untimed), its end
    rounded to the nearest root of x_i^{d_i} = 1, and the forward path from
    that start root -- a path of the n = 512 total-degree homotopy -- is timed
    with CUDA events and checked against x* (success: within 1e-48).  Corrector
    tolerance on the way 1e-8 with 5 Newton iterations, QD at t = 1."""
    stream = torch.cuda.current_stream(dev)
    L = 4
    wl, xs = synth.sparse512_planted(seed, "qd")
    f = ctx.load(wl.f, L)
    G = ctx.load(synth.total_degree_start(wl.f), L)
    base = dict(synth.default_params(L), max_steps=max_steps, tol_path=1e-8, max_newton=5)
    t0 = time.perf_counter()
    gb = _soa([1.0 / wl.gamma], L).reshape(L, 2)
    xl = np.zeros((L, 2, 512))
    stb, sdb, _ = libph.ph_track_path(ctx.h, G, f, gb, _soa(xs, L), base, xl)
    back_s = time.perf_counter() - t0
    out = {"workload": wl.name, "backward_s": back_s, "backward_status": libph.STATUS_NAMES[stb],
           "backward_steps": sdb["steps"], "backward_t_final": sdb["t_final"],
           "params": {"tol_path": 1e-8, "max_newton": 5, "max_dt": base["max_dt"]}}
    if stb == libph.PH_OK:
        x0 = torch.tensor(_soa(synth.nearest_start_root(wl.f, xl[0, 0] + 1j * xl[0, 1]), L),
                          device=dev)
        gam = torch.tensor(wl.gamma_soa(), device=dev)
        xo = torch.empty_like(x0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, sd, _ = libph.ph_track_path(ctx.h, f, None, gam, x0, base, xo)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        err = _err_vs(xo.cpu().numpy(), xs)
        out.update({"status": libph.STATUS_NAMES[st], "ms": ms, "steps": sd["steps"],
                    "accepted": sd["accepted"], "rejected": sd["rejected"],
                    "newton_iters": sd["newton_iters"], "t_final": sd["t_final"],
                    "err_vs_planted": err, "ok": bool(st == libph.PH_OK and err <= 1e-48),
                    "paths_per_s": 1e3 / ms,
                    "corrector_steps_per_s": sd["newton_iters"] / (ms * 1e-3)})
    ctx.free(f)
    ctx.free(G)
    return out


def hard_precision_leg(libph, synth, ctx, torch, dev, seed, steps, decades=8.0, max_dt=1e-6):
    """The planted n = 128 workload where it is hard: precision128's shape with the coefficient
    moduli spread over `decades` decades between the equations (each
    polynomial's terms share a modulus 10^{decades u_i}), so the Jacobian's
    rows differ in scale by up to 10^decades (condition number about 2.5e9 at
    the planted root for 8 decades, 1.9e13 for 12, in numpy; with 12 no step
    of either form converges from x*).
    The path is tracked backwards from x* (start system f, target the
    total-degree system, gamma' = 1/gamma), where the Jacobian is the
    ill-conditioned J_f: the first `steps` steps, single path, plain (lin_prec
    0) against the precision form (lin_prec 1: Newton systems in double), the
    same tolerances; then copies of the path at once through ph_track_paths
    (152 in DD, 32 in QD) with lin_prec 0, 1 and 3 for the FP32/FP64 split."""
    stream = torch.cuda.current_stream(dev)
    out = {}
    for prec in ("dd", "qd"):
        wl, xs = synth.precision128_equations(seed, prec, decades)
        L = wl.L
        f = ctx.load(wl.f, L)
        G = ctx.load(synth.total_degree_start(wl.f), L)
        gi = 1.0 / wl.gamma
        gb = torch.tensor(_soa([gi], L).reshape(L, 2), device=dev)
        x0 = torch.tensor(_soa(xs, L), device=dev)
        mn = 5 if L == 2 else 6
        row = {"steps": steps, "max_newton": mn, "max_dt": max_dt, "decades": decades,
               "cond_at_planted_root_numpy": {8.0: 2.5e9, 12.0: 1.9e13}.get(decades)}
        ref = None
        for lin in (0, 1):
            params = dict(wl.params, max_steps=steps - 1, max_dt=max_dt, max_newton=mn,
                          lin_prec=lin)
            xo = torch.empty_like(x0)
            libph.ph_track_path(ctx.h, G, f, gb, x0, dict(params, max_steps=0), xo)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, sd, _ = libph.ph_track_path(ctx.h, G, f, gb, x0, params, xo)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            x = xo.cpu().numpy()
            r = {"status": libph.STATUS_NAMES[st], "ms": ms, "accepted": sd["accepted"],
                 "rejected": sd["rejected"], "t_final": sd["t_final"],
                 "newton_iters": sd["newton_iters"], "solves_f64": sd["solves_f64"],
                 "escalated": sd["escalated"], "wp_rest": sd["wp_rest"],
                 "cond_estimate": sd["cond"],
                 "ms_per_accepted_step": ms / max(1, sd["accepted"])}
            if ref is None:
                ref = (r, x)
            else:
                if r["t_final"] == ref[0]["t_final"]:
                    d = (x - ref[1])[::-1].sum(0)
                    r["end_point_diff_vs_plain"] = float(np.abs(d[0] + 1j * d[1]).max())
                r["speedup_per_accepted_step"] = (ref[0]["ms_per_accepted_step"]
                                                  / r["ms_per_accepted_step"])
            row[f"single_lin{lin}"] = r
        copies = 152 if L == 2 else 32                 # QD: the plain form takes seconds a step
        bx = torch.tensor(np.repeat(_soa(xs, L)[None], copies, axis=0), device=dev)
        for lin in (0, 1, 3):
            params = dict(wl.params, max_steps=steps - 1, max_dt=max_dt, max_newton=mn,
                          lin_prec=lin)
            bo = torch.empty_like(bx)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats, _ = libph.ph_track_paths(ctx.h, G, f, gb, bx, params, bo)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            acc = sum(x["accepted"] for x in stats)
            row[f"batch{copies}_lin{lin}"] = {
                "ms": ms, "accepted_steps_per_s": acc / (ms * 1e-3),
                "solves_f32": sum(x["solves_f32"] for x in stats),
                "solves_f64": sum(x["solves_f64"] for x in stats),
                "escalated": sum(x["escalated"] for x in stats),
                "wp_rest": sum(x["wp_rest"] for x in stats),
                "cond_estimate_max": float(max(x["cond"] for x in stats))}
        ctx.free(f)
        ctx.free(G)
        out[f"precision128eq_{prec}"] = row
    return out


def large_job_leg(libph, synth, ctx, seed, nsmall=64):
    """The serving loop's large-job route (ph_server_config.big_n = 64): a
    stream of small requests (n log-uniform in [16, 64], dense or sparse,
    DD/QD 70/30, 20-step segments) alone, then the same stream with two large
    jobs submitted in its middle -- a dense n = 128 DD system (128 terms per
    polynomial over 16 variables, 5-step segment) and the sparse n = 320 QD
    system (3-step segment) -- which run alone on the whole GPU by the
    single-path tracker while small-job admission pauses.  Reports each large
    job's latency and the small jobs' p50/p99 without and with them."""
    rng = np.random.default_rng(seed + 2000)
    small = []
    for i in range(nsmall):
        srng = synth.Rng(seed * 104729 + i)
        n = int(round(np.exp(srng.uniform() * (np.log(64) - np.log(16)) + np.log(16))))
        dense = i % 2 == 0
        L = 2 if rng.random() < 0.7 else 4
        spec = (synth.dense_system(srng, n, n, min(16, n), (1, 2, 3)) if dense
                else synth.sparse_system(srng, n))
        g = srng.unit_complex()
        small.append((ctx.load(spec, L), _soa([g], L).reshape(L, 2), _soa(np.ones(n), L),
                      synth.default_params(L, max_steps=19)))
    big = []
    for (n, L, dense, steps) in ((128, 2, True, 5), (320, 4, False, 3)):
        srng = synth.Rng(seed * 7 + n)
        spec = (synth.dense_system(srng, n, n, 16, (1, 2, 3)) if dense
                else synth.sparse_system(srng, n))
        g = srng.unit_complex()
        big.append((ctx.load(spec, L), _soa([g], L).reshape(L, 2), _soa(np.ones(n), L),
                     synth.default_params(L, max_steps=steps - 1, max_newton=3 if L == 2 else 5,
                                          tol_path=1e-8), n, L))
    out = {}
    srv = libph.ph_server_create(ctx.h, max_n=64, pool_bytes=4 << 30, queue_cap=512, big_n=64)
    try:
        for label, with_big in (("small_alone", False), ("with_two_large_jobs", True)):
            ids, bids = [], []
            t0 = time.perf_counter()
            for i, (f, gam, x0, p) in enumerate(small):
                ids.append(libph.ph_server_submit(ctx.h, srv, f, None, gam, x0, p))
                if with_big and i in (nsmall // 4, nsmall // 2):
                    bf, bg, bx, bp, _, _ = big[len(bids)]
                    bids.append(libph.ph_server_submit(ctx.h, srv, bf, None, bg, bx, bp))
            lats = [libph.ph_server_wait(ctx.h, srv, jid, 900000)[1] for jid in ids]
            row = {"small_jobs": len(ids), "wall_s": time.perf_counter() - t0,
                   "small_p50_ms": float(np.percentile(lats, 50)),
                   "small_p99_ms": float(np.percentile(lats, 99))}
            for (bf, bg, bx, bp, n, L), jid in zip(big, bids):
                st, lat = libph.ph_server_wait(ctx.h, srv, jid, 900000)
                row[f"large_n{n}_{'dd' if L == 2 else 'qd'}"] = {
                    "latency_ms": lat, "status": libph.STATUS_NAMES[st["status"]],
                    "steps": st["steps"], "newton_iters": st["newton_iters"]}
            out[label] = row
    finally:
        libph.ph_server_destroy(srv)
    for f, _, _, _ in small:
        ctx.free(f)
    for bf, _, _, _, _, _ in big:
        ctx.free(bf)
    return out


def combine_ranks(dist, torch, tot_ms: float, iters: int, device):
    """Whole-job figures of a replicas run: the slowest rank's timed ms and the
    corrector steps of all ranks (each rank tracks its own path; the only
    collectives are these two reductions).  Without a process group, the
    rank's own figures."""
    if dist is None:
        return tot_ms, float(iters)
    t = torch.tensor([tot_ms, float(iters)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def summarize(ms, stats):
    iters = sum(s["newton_iters"] for s in stats)
    pcs = sum(s["steps"] for s in stats)
    tot = sum(ms) / 1e3
    return {
        "corrector_steps_per_s": iters / tot,
        "pc_steps_per_s": pcs / tot,
        "paths_per_s": len(ms) / tot,
        "p50_segment_ms": float(np.percentile(ms, 50)),
        "p99_segment_ms": float(np.percentile(ms, 99)),
        "path": {"status": stats[-1]["status"], "steps": stats[-1]["steps"],
                 "accepted": stats[-1]["accepted"], "rejected": stats[-1]["rejected"],
                 "newton_iters": stats[-1]["newton_iters"], "t_final": stats[-1]["t_final"]},
        "launches": sum(s["launches"] for s in stats),
    }


def mgs_case(spec: str) -> None:
    """--only-mgs L,N,n,reps: `reps` least-squares solves (ph_mgs_solve, host
    buffers) of one seeded N x n complex matrix with L limbs, then one JSON
    line with the variant the library chose and both variants' measured times.
    A fixed, small launch sequence for kernel profiles: the first solve of a
    shape times 4 launches of each variant, then every solve is one launch."""
    from paper_1501_06625_gb300 import libph
    L, N, n, reps = (int(v) for v in spec.split(","))
    rng = np.random.default_rng(N * 7919 + n)
    A = rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n)) + 2 * np.eye(N, n)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    J = np.zeros((L, 2, n, N))
    J[0, 0], J[0, 1] = A.T.real, A.T.imag
    rhs = np.zeros((L, 2, N))
    rhs[0, 0], rhs[0, 1] = b.real, b.imag
    dx = np.zeros((L, 2, n))
    ctx = libph.Context(0)
    for _ in range(reps):
        libph.ph_mgs_solve(ctx.h, L, N, n, J, rhs, dx)
    kind, size, ms = libph.ph_mgs_variant(ctx.h, L, N, n)
    ctx.close()
    print(json.dumps({"mgs_case": {"L": L, "N": N, "n": n, "solves": reps,
                                   "variant": libph.MGS_KINDS[kind], "size": size,
                                   "ms_grid_cluster_tiled": ms}}))


def monodromy_paths_case(spec: str) -> None:
    """--only-monodromy-paths n,L,paths,steps: one ph_track_paths call (one
    kernel launch) over `paths` copies of the first cyclic n-roots monodromy
    loop, `steps` predictor-corrector steps each, twice; one JSON line with the
    event-timed ms of the second call.  A single long launch for profiles of
    the per-block path kernel on a system with long terms and N > n."""
    import torch
    from paper_1501_06625_gb300 import libph, synth
    n, L, paths, steps = (int(v) for v in spec.split(","))
    F, G, gam, x0 = synth.cyclic_monodromy(1, n)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = libph.Context(0, stream=stream)
    f, g = ctx.load(F, L), ctx.load(G, L)
    xs = np.zeros((paths, L, 2, n))
    xs[:, 0, 0], xs[:, 0, 1] = x0.real, x0.imag
    gs = np.zeros((L, 2))
    gs[0] = [gam.real, gam.imag]
    bx = torch.tensor(xs, dtype=torch.float64, device=dev)
    bo = torch.empty_like(bx)
    bg = torch.tensor(gs, dtype=torch.float64, device=dev)
    params = synth.default_params(L, max_newton=5 if L == 2 else 6, max_steps=steps - 1,
                                  fixed_rows=1)
    ms = 0.0
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, _ = libph.ph_track_paths(ctx.h, f, g, bg, bx, params, bo)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    it = sum(x["newton_iters"] for x in st)
    ctx.close()
    print(json.dumps({"monodromy_paths_case": {"n": n, "L": L, "paths": paths, "steps": steps,
                                               "ms": ms, "newton_iters": it,
                                               "ms_per_iter_per_path": ms * paths / max(1, it)}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", default="dd")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--qd-steps", type=int, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-all-cores-seconds", type=float, default=10.0,
                    help="seconds per core of the all-cores oracle figure (0 skips it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--control", choices=["device", "host"], default="device",
                    help="step control on the device (one graph per path segment) or on the "
                         "host (one graph per step, as in the paper)")
    ap.add_argument("--batch-paths", type=int, default=304,
                    help="paths of the many-path leg (0 skips it)")
    ap.add_argument("--batch-steps", type=int, default=None,
                    help="steps per path of the many-path leg (default: the segment)")
    ap.add_argument("--precision-paths", type=int, default=152,
                    help="paths of the precision-form leg (0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=384,
                    help="requests of the serving leg (0 skips it)")
    ap.add_argument("--no-cyclic", action="store_true", help="skip the cyclic n-roots legs")
    ap.add_argument("--monodromy", action="store_true",
                    help="also run the cyclic n-roots monodromy legs (the paper's one-path runs, "
                         "loops in flight, the degree by loops): outside the hot-path rows")
    ap.add_argument("--whole-paths", type=int, default=304,
                    help="planted dense64 DD paths tracked whole (0 skips the whole-path leg)")
    ap.add_argument("--whole-paths-single", type=int, default=8,
                    help="of these, how many the single-path form tracks one by one")
    ap.add_argument("--whole-paths-qd", type=int, default=3,
                    help="planted dense64 QD paths tracked whole by the single-path form")
    ap.add_argument("--sparse-steps", type=int, default=16,
                    help="predictor-corrector steps of the sparse n = 512 QD path (0 skips)")
    ap.add_argument("--sparse-whole-paths", type=int, default=0,
                    help="1: one whole planted sparse n = 512 QD path to t = 1, backwards "
                         "then forwards (several minutes each way; off by default)")
    ap.add_argument("--large-jobs", type=int, default=1,
                    help="1: the serving loop's large-job route leg (0 skips it)")
    ap.add_argument("--hard-steps", type=int, default=30,
                    help="steps of the ill-conditioned precision128 segment (0 skips)")
    ap.add_argument("--only-mgs", default=None, metavar="L,N,n,reps",
                    help="only time least-squares solves of one shape (for kernel profiles)")
    ap.add_argument("--only-monodromy-paths", default=None, metavar="n,L,paths,steps",
                    help="only time one many-path launch on a monodromy loop (for kernel profiles)")
    ap.add_argument("--monodromy-segment", type=int, default=40,
                    help="steps of the cyclic monodromy paths not tracked whole")
    ap.add_argument("--monodromy-loops", type=int, default=152,
                    help="monodromy loops tracked at once through the serving loop (0 skips)")
    ap.add_argument("--monodromy-degree-64", action="store_true",
                    help="also compute the degree of the cyclic 64-roots set (about two minutes)")
    ap.add_argument("--no-sparse", action="store_true",
                    help="skip the n=512 QD solver roofline measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.only_mgs or args.only_monodromy_paths:
        from paper_1501_06625_gb300 import build
        build.build()
        if args.only_mgs:
            return mgs_case(args.only_mgs)
        return monodromy_paths_case(args.only_monodromy_paths)
    CONTROL["control"] = 1 if args.control == "host" else 0

    import torch
    from paper_1501_06625_gb300 import build, libph, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        # the legs that describe one GPU (serving, precision form, cyclic and
        # monodromy, the n = 512 solve) run in the one-GPU run; a run on N GPUs
        # measures the replicated step and holds its GPUs no longer than that
        args.serve_requests = 0
        args.precision_paths = 0
        args.no_cyclic = True
        args.no_sparse = True
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    legs = {}                                      # wall seconds of each leg
    stream = torch.cuda.current_stream(dev)
    ctx = libph.Context(local, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    wl = synth.dense64(args.seed + rank, args.prec)
    f = ctx.load(wl.f, wl.L)
    peak = libph.ph_fp64_peak(ctx.h, 50.0)            # G lane-ops/s, measured now
    rates = libph.ph_unit_rates(ctx.h)
    unit_rates = {"fp64_fma_pipe_g_per_s": rates[0], "fp64_fma_tensor_core_g_per_s": rates[1],
                  "int32_mad_g_per_s": rates[2]}

    # timed region: barrier + synchronize on both sides, max over ranks
    track_leg(libph, ctx, f, wl, dev, 0, args.warmup, torch, flush)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    ms, stats, xo = track_leg(libph, ctx, f, wl, dev, args.steps, 0, torch, flush)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    if dist:
        dist.barrier()
    s = summarize(ms, stats)
    iters = sum(x["newton_iters"] for x in stats)
    tot_ms = sum(ms)
    tot_ms_max, iters_all = combine_ranks(dist, torch, tot_ms, iters, dev)
    value = iters_all / (tot_ms_max / 1e3)

    # QD leg (same path, quad double)
    qd = None
    if args.prec == "dd" and args.qd_steps != 0:
        wq = synth.dense64(args.seed + rank, "qd")
        fq = ctx.load(wq.f, wq.L)
        kq = args.qd_steps if args.qd_steps is not None else max(1, args.steps // 2)
        msq, statsq, _ = track_leg(libph, ctx, fq, wq, dev, kq, 1, torch, flush)
        qd = summarize(msq, statsq)
        qd.pop("launches")
        qd["note"] = ("the first %d steps from the all-ones root: the degree-0 first "
                      "prediction needs dt ~ 1e-7 for a QD corrector, so these steps are "
                      "mostly rejections (accepted: %d); whole QD paths are in whole_paths"
                      % (SEGMENT[4], statsq[-1]["accepted"]))

    # many-path form: the same system, distinct total-degree start roots, the
    # same segment per path, one persistent kernel (ph_track_paths)
    batch = None
    if args.batch_paths > 0:
        bx0 = torch.tensor(batch_starts(wl, args.batch_paths), dtype=torch.float64, device=dev)
        bxo = torch.empty_like(bx0)
        bgam = torch.tensor(wl.gamma_soa(), dtype=torch.float64, device=dev)
        bparams = seg_params(wl)
        if args.batch_steps:
            bparams["max_steps"] = args.batch_steps - 1
        libph.ph_track_paths(ctx.h, f, None, bgam, bx0, bparams, bxo)   # warm-up
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bstats, _ = libph.ph_track_paths(ctx.h, f, None, bgam, bx0, bparams, bxo)
        e1.record(stream)
        e1.synchronize()
        bms = e0.elapsed_time(e1)
        bit = sum(x["newton_iters"] for x in bstats)
        # FP64 instructions the kernel issues (DD: the fixed-point MGS tally),
        # and the same work counted in the FP64 forms of the single-path kernels
        fx_unit = MGS_UNIT_FIXED_DD if wl.L == 2 else None
        bops = bit * (ad_ops(wl.f, wl.L) + sum_ops(wl.f, wl.L) +
                      mgs_ops(wl.f.N, wl.n, wl.L, unit=fx_unit))
        bops_form = bit * (ad_ops(wl.f, wl.L) + sum_ops(wl.f, wl.L) + mgs_ops(wl.f.N, wl.n, wl.L))
        bach = bops / (bms * 1e-3) / 1e9
        lanes, lane_ms = libph.ph_block_lanes(ctx.h, f)
        tuned = {"lanes_per_output": lanes,
                 "ms_per_iteration_launch_by_lanes": dict(zip(["1", "2", "4", "8", "16", "32"],
                                                              lane_ms))}
        if lane_ms[2] > 0 and min(lane_ms) > 0:
            tuned["gain_vs_4_lanes"] = lane_ms[2] / min(lane_ms)
        batch = {"paths": args.batch_paths, "steps_per_path": bparams["max_steps"] + 1, "ms": bms,
                 "summation_tuning": tuned,
                 "corrector_steps_per_s": bit / (bms * 1e-3),
                 "pc_steps_per_s": sum(x["steps"] for x in bstats) / (bms * 1e-3),
                 "segments_per_s": args.batch_paths / (bms * 1e-3),
                 "vs_single_path": (bit / (bms * 1e-3)) / value,
                 "gpu_launches": 1,
                 "roofline": {"bound": "alu", "kernel": "k_paths (whole step, many paths)",
                              "achieved": bach, "peak": peak, "unit": "G FP64-ops/s",
                              "frac": bach / peak,
                              "ops": "FP64 instructions issued (DD MGS sums in integer units)",
                              "fp64_form_equivalent_frac": bops_form / (bms * 1e-3) / 1e9 / peak}}

    serve = serve_mixed = None
    if args.serve_requests > 0 and rank == 0:
        _t0 = time.perf_counter()
        serve = serve_leg(libph, synth, ctx, args.serve_requests, args.seed)
        serve_mixed = serve_leg(libph, synth, ctx, args.serve_requests, args.seed, lin=3,
                                seq_rate=serve["sequential_single_path"]["paths_per_s"])
        legs['serving'] = time.perf_counter() - _t0

    cyclic = monodromy = None
    if not args.no_cyclic and rank == 0:
        _t0 = time.perf_counter()
        cyclic = cyclic_leg(libph, synth, ctx, torch, dev, peak)
        legs['cyclic'] = time.perf_counter() - _t0
    if args.monodromy and rank == 0:
        monodromy = monodromy_leg(libph, synth, ctx, torch, dev, args.seed,
                                  args.monodromy_segment)
        if args.monodromy_loops > 0:
            monodromy["loops_in_flight"] = monodromy_loops_leg(
                libph, synth, ctx, args.seed, args.monodromy_loops, monodromy)
        monodromy["degree"] = monodromy_degree_leg(
            synth, ctx, args.seed, [(16, 32)] + ([(64, 76)] if args.monodromy_degree_64 else []))

    whole = sparse = hard = large = sparse_whole = None
    if rank == 0 and world == 1:
        if args.whole_paths > 0 or args.whole_paths_qd > 0:
            _t0 = time.perf_counter()
            whole = whole_path_leg(libph, synth, ctx, torch, dev, args.seed, args.whole_paths,
                                   args.whole_paths_single, args.whole_paths_qd)
            legs['whole_paths'] = time.perf_counter() - _t0
        if args.sparse_steps > 0:
            _t0 = time.perf_counter()
            sparse = sparse512_leg(libph, synth, ctx, torch, dev, args.seed, args.sparse_steps)
            legs['sparse512'] = time.perf_counter() - _t0
        if args.sparse_whole_paths > 0:
            _t0 = time.perf_counter()
            sparse_whole = sparse512_whole_path(libph, synth, ctx, torch, dev, args.seed)
            legs['sparse512_whole_path'] = time.perf_counter() - _t0
        if args.large_jobs:
            _t0 = time.perf_counter()
            large = large_job_leg(libph, synth, ctx, args.seed)
            legs['serving_large_jobs'] = time.perf_counter() - _t0
        if args.hard_steps > 0:
            _t0 = time.perf_counter()
            hard = hard_precision_leg(libph, synth, ctx, torch, dev, args.seed, args.hard_steps)
            legs['precision_ill_conditioned'] = time.perf_counter() - _t0

    precision = None
    if args.precision_paths > 0 and rank == 0:
        _t0 = time.perf_counter()
        precision = precision_leg(libph, synth, ctx, torch, dev, flush, args.seed,
                                  args.precision_paths)
        precision.update(precision_path_leg(libph, synth, ctx, torch, dev, flush, args.seed))
        legs['precision'] = time.perf_counter() - _t0

    # end to end through the same call with host buffers
    e2e_v, h2d, d2h = e2e_leg(libph, ctx, f, wl, max(2, args.steps // 2), torch)

    # roofline of the dominant kernel, timed live on the library's stream
    x_mid = torch.tensor(wl.x0_soa(), dtype=torch.float64, device=dev)
    tl = torch.zeros(wl.L, dtype=torch.float64, device=dev)
    tl[0] = 0.05
    gam = torch.tensor(wl.gamma_soa(), dtype=torch.float64, device=dev)
    kms = libph.ph_profile_newton(ctx.h, f, None, gam, 1, tl, x_mid, 20)
    names = ["prep", "monomial_ad", "summation", "mgs"]
    ops = {"monomial_ad": ad_ops(wl.f, wl.L), "summation": sum_ops(wl.f, wl.L),
           "mgs": mgs_ops(wl.f.N, wl.n, wl.L)}
    dom = max(("monomial_ad", "summation", "mgs"), key=lambda k: kms[names.index(k)])
    dms = kms[names.index(dom)]
    achieved = ops[dom] / (dms * 1e-3) / 1e9
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
            "unit": "G FP64-ops/s", "frac": achieved / peak,
            "traffic": MGS_DENSE64_DD_TRAFFIC if dom == "mgs" and wl.L == 2 else None,
            "peak_source": "measured DFMA rate on this GPU in this run (ph_fp64_peak)",
            "kernel_ms": dict(zip(names, kms)), "ops_per_launch": ops[dom]}

    # the n = 512 quad-double solve (sparse system): large enough to be
    # throughput-bound rather than latency-bound
    roof512 = None
    if not args.no_sparse:
        w5 = synth.sparse512(args.seed, "qd")
        f5 = ctx.load(w5.f, w5.L)
        x5 = torch.tensor(w5.x0_soa(), dtype=torch.float64, device=dev)
        g5 = torch.tensor(w5.gamma_soa(), dtype=torch.float64, device=dev)
        t5 = torch.zeros(w5.L, dtype=torch.float64, device=dev)
        t5[0] = 0.5
        k5 = libph.ph_profile_newton(ctx.h, f5, None, g5, 1, t5, x5, 2)
        o5 = mgs_ops(512, 512, 4)
        a5 = o5 / (k5[3] * 1e-3) / 1e9
        roof512 = {"bound": "alu", "kernel": "mgs", "workload": "sparse512_qd", "achieved": a5,
                   "peak": peak, "unit": "G FP64-ops/s", "frac": a5 / peak,
                   "ops": "the solve's work counted in the FP64 forms of the QD primitives; its "
                          "dot products, updates and downdates run as 256-bit integer "
                          "arithmetic, so the fraction can exceed what the FP64 pipe alone "
                          "would reach",
                   "kernel_ms": dict(zip(names, k5)), "ops_per_launch": o5}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        it_c, wall_c, pcs_c = oracle_sample(wl, seconds=args.cpu_seconds)
        cpu = {"value": it_c / wall_c, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {pcs_c} predictor-corrector steps of the {wl.name} path "
                         f"({it_c} corrector steps, {wall_c:.1f} s, one thread)"}
        if args.cpu_all_cores_seconds > 0:
            cpu["all_cores"] = oracle_all_cores(args.seed, args.prec, args.cpu_all_cores_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms_max / len(ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "dd", "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.n, "terms_per_poly": 64, "vars_per_term": 16,
                       "exponents": [1, 2, 3], "homotopy": "total-degree from all-ones, k=1",
                       "seed": args.seed, "precision": "complex double-double",
                       "segment": f"first {SEGMENT[2]} predictor-corrector steps of the path",
                       "l2": "flushed (256 MiB write) between steps",
                       "parallelism": f"replicas x{world}", "control": args.control},
            "segments_per_s": s["paths_per_s"], "pc_steps_per_s": s["pc_steps_per_s"],
            "p50_segment_ms": s["p50_segment_ms"], "p99_segment_ms": s["p99_segment_ms"],
            "path": s["path"], "qd": qd, "batched": batch, "serving": serve,
            "serving_mixed": serve_mixed, "precision": precision, "cyclic": cyclic,
            "cyclic_monodromy_path": monodromy, "whole_paths": whole,
            "sparse512_segment": sparse, "sparse512_whole_path": sparse_whole,
            "precision_ill_conditioned": hard,
            "serving_large_jobs": large,
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": s["launches"], "roofline": roof, "roofline_sparse512_mgs": roof512,
            "cpu_baseline": cpu,
            "clocks": clk, "wall_s_timed": wall, "leg_seconds": legs, "unit_rates": unit_rates,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
