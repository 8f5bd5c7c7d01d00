"""Monodromy loops on the device (Section 4.2): the degree of a solution set
computed numerically, as the paper does for cyclic n-roots.

A loop starts at a known point of the solution set on the slices L, tracks
the homotopy {f = 0, alpha (1-t) L + t K = 0} to the slices K, then
{f = 0, beta (1-t) K + t L = 0} back to L, with random constants alpha and
beta.  Its end point is again a point of the set on L, often another one.
After enough loops with different constants every point of the set on L has
been reached, and their number is the degree.  Every loop is two independent
paths, so many loops run at once through the serving loop (ph_server_*, one
persistent block per path); the host submits and collects them and keeps the
distinct end points.  Host orchestration only: every path runs in the
library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import libph, synth


def _soa(z: np.ndarray, L: int) -> np.ndarray:
    x = np.zeros((L, 2, z.size))
    x[0, 0], x[0, 1] = z.real, z.imag
    return x


def _lead(x: np.ndarray) -> np.ndarray:
    return x[0, 0] + 1j * x[0, 1]


def loops(ctx, loop: dict, L: int, params: dict, rounds: int, per_round: int, seed: int = 1,
          tol: float = 1e-8, patience: int = 1, timeout_ms: int = 600000) -> dict:
    """Monodromy loops (synth.cyclic_monodromy_loop systems) kept `per_round`
    at a time in the serving loop: a loop's way back is submitted as soon as
    its way out ends, and a new loop starts, from the points found so far in
    turn, as soon as one ends, each loop with its own alpha and beta.  No new
    loop starts once `patience * per_round` loops in a row have found no new
    point, or `rounds * per_round` have started; the loops in flight then
    finish (their points count).  Points are distinct when their leading
    limbs differ by more than tol (relative).  params: tracking parameters
    (fixed_rows is set).  Returns {"points": [L][2][n] arrays, "found": count
    after every per_round finished loops, "loops", "failed", "paths",
    "newton_iters"}."""
    F, G = loop["out"]
    Fb, Gb = loop["back"]
    x0 = loop["x0"]
    n = x0.size
    p = dict(params, fixed_rows=1)
    rng = synth.Rng(seed)
    fo, go = ctx.load(F, L), ctx.load(G, L)
    fb, gb = ctx.load(Fb, L), ctx.load(Gb, L)
    srv = libph.ph_server_create(ctx.h, max_n=n, pool_bytes=8 << 30, queue_cap=2 * per_round)
    points = [_soa(x0, L)]
    found = []
    failed = paths = iters = started = finished = since_new = 0
    inflight = {}                                  # job id -> ("out" | "back", submit time)

    def submit(f, g, x, kind):
        gs = np.zeros((L, 2))
        gam = rng.unit_complex()
        gs[0] = [gam.real, gam.imag]
        inflight[libph.ph_server_submit(ctx.h, srv, f, g, gs, x, p)] = (kind, time.monotonic())

    def start_loop():
        nonlocal started
        if started < rounds * per_round and since_new < patience * per_round:
            submit(fo, go, points[started % len(points)], "out")
            started += 1

    try:
        for _ in range(per_round):
            start_loop()
        while inflight:
            progressed = False
            for jid, (kind, t0) in list(inflight.items()):
                x = np.zeros((L, 2, n))
                done, st, _ = libph.ph_server_poll(ctx.h, srv, jid, x)
                if not done:
                    if (time.monotonic() - t0) * 1e3 > timeout_ms:
                        raise RuntimeError("monodromy: a path did not finish in time")
                    continue
                progressed = True
                del inflight[jid]
                paths += 1
                iters += st["newton_iters"]
                ok = st["status"] == libph.PH_OK
                if kind == "out" and ok:
                    submit(fb, gb, x, "back")
                    continue
                finished += 1                      # the loop ends here
                new = False
                if ok:
                    zl = _lead(x)
                    scale = max(1.0, np.abs(zl).max())
                    if all(np.abs(zl - _lead(q)).max() > tol * scale for q in points):
                        points.append(x)
                        new = True
                else:
                    failed += 1
                since_new = 0 if new else since_new + 1
                if finished % per_round == 0:
                    found.append(len(points))
                start_loop()
            if not progressed:
                time.sleep(0.0005)
    finally:
        libph.ph_server_destroy(srv)
        for s_ in (fo, go, fb, gb):
            ctx.free(s_)
    return {"points": points, "found": found, "loops": started, "failed": failed,
            "paths": paths, "newton_iters": iters}


def family_points_on_slices(m: int, coef: np.ndarray, const: np.ndarray) -> np.ndarray:
    """The points of Backelin's family x_{am+b} = w^a v_b, prod_b v_b = 1
    (synth.backelin_point), on the slices coef x + const = 0, in double: x is
    linear in v, so the m - 1 slice equations leave a line v = v_p + s w, and
    prod_b (v_p,b + s w_b) = 1 is a polynomial of degree m in s.  Returns the
    m points, [m][n] complex."""
    w = np.exp(2j * np.pi * np.arange(m) / m)
    A = np.kron(w[:, None], np.eye(m))                  # x = A v, rows a m + b
    Mv = coef @ A                                       # (m - 1) x m
    vp = np.linalg.lstsq(Mv, -const, rcond=None)[0]
    wv = np.linalg.svd(Mv)[2].conj()[-1]                # null vector
    poly = np.array([1.0 + 0j])
    for b in range(m):                                  # prod (vp_b + s w_b)
        poly = np.convolve(poly, np.array([wv[b], vp[b]]))
    poly[-1] -= 1.0
    s = np.roots(poly)
    return np.array([A @ (vp + si * wv) for si in s])
