"""Monodromy loops on the device (Section 4.2): the degree of a solution set
computed numerically, as the paper does for cyclic n-roots.

A loop starts at a known point of the solution set on the slices L, tracks
the homotopy {f = 0, alpha (1-t) L + t K = 0} to the slices K, then
{f = 0, beta (1-t) K + t L = 0} back to L, with random constants alpha and
beta.  Its end point is again a point of the set on L, often another one.
After enough loops with different constants every point of the set on L has
been reached, and their number is the degree.  Every loop is an independent
path, so a round of loops runs at once through the serving loop
(ph_server_*, one persistent block per path); the host only collects the
distinct end points.  Host orchestration only: every path runs in the
library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import libph, synth


def _soa(z: np.ndarray, L: int) -> np.ndarray:
    x = np.zeros((L, 2, z.size))
    x[0, 0], x[0, 1] = z.real, z.imag
    return x


def _lead(x: np.ndarray) -> np.ndarray:
    return x[0, 0] + 1j * x[0, 1]


def _track_all(ctx, srv, f, g, gammas, starts, params, L, timeout_ms):
    """One path per (gamma, start) through the server; returns (end points
    [L][2][n] or None for a failed path, stats)."""
    ids = []
    for gam, x0 in zip(gammas, starts):
        gs = np.zeros((L, 2))
        gs[0] = [gam.real, gam.imag]
        ids.append(libph.ph_server_submit(ctx.h, srv, f, g, gs, x0, params))
    ends, stats = [], []
    for jid, x0 in zip(ids, starts):
        x = np.zeros_like(x0)
        st, _ = libph.ph_server_wait(ctx.h, srv, jid, timeout_ms, x)
        stats.append(st)
        ends.append(x if st["status"] == libph.PH_OK else None)
    return ends, stats


def loops(ctx, loop: dict, L: int, params: dict, rounds: int, per_round: int, seed: int = 1,
          tol: float = 1e-8, patience: int = 1, timeout_ms: int = 600000) -> dict:
    """Runs rounds of `per_round` monodromy loops (synth.cyclic_monodromy_loop
    systems) from the points found so far, each loop with its own alpha and
    beta, until a round adds no new point `patience` times or `rounds` have
    run.  Points are distinct when their leading limbs differ by more than
    tol (relative).  params: tracking parameters (fixed_rows is set).
    Returns {"points": [L][2][n] arrays, "found": count after each round,
    "loops", "failed", "paths", "newton_iters"}."""
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
    found, failed, paths, iters, idle = [], 0, 0, 0, 0
    try:
        for _ in range(rounds):
            starts = [points[i % len(points)] for i in range(per_round)]
            alphas = [rng.unit_complex() for _ in range(per_round)]
            betas = [rng.unit_complex() for _ in range(per_round)]
            mid, s1 = _track_all(ctx, srv, fo, go, alphas, starts, p, L, timeout_ms)
            ok = [i for i, y in enumerate(mid) if y is not None]
            ends, s2 = _track_all(ctx, srv, fb, gb, [betas[i] for i in ok],
                                  [mid[i] for i in ok], p, L, timeout_ms)
            paths += len(s1) + len(s2)
            iters += sum(s["newton_iters"] for s in s1 + s2)
            failed += (per_round - len(ok)) + sum(1 for z in ends if z is None)
            before = len(points)
            for z in ends:
                if z is None:
                    continue
                zl = _lead(z)
                scale = max(1.0, np.abs(zl).max())
                if all(np.abs(zl - _lead(q)).max() > tol * scale for q in points):
                    points.append(z)
            found.append(len(points))
            idle = idle + 1 if len(points) == before else 0
            if idle >= patience:
                break
    finally:
        libph.ph_server_destroy(srv)
        for s in (fo, go, fb, gb):
            ctx.free(s)
    return {"points": points, "found": found, "loops": len(found) * per_round,
            "failed": failed, "paths": paths, "newton_iters": iters}


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
