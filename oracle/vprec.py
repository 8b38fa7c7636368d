"""Reduced-precision emulation of the CG loop (CPU oracle, numpy).

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU leg).

The paper chooses where precision may be lowered by running Nekbone under
Verificarlo's VPREC backend, which rounds the result of every floating-point
operation to a t-bit mantissa while keeping the exponent range (Sec. 2,
"Methodology"; Sec. 3.2, residual versus precision for t = 3..52).  This
module emulates that for the CG loop of the profiling table: every addition,
multiplication and division of the loop -- inside the operator's tensor
contractions, the geometric-factor products, the gather-scatter sums, the
dot products and the vector updates -- is rounded to t mantissa bits
(round to nearest, ties to even).  The set-up (GLL rule, geometry, the
Jacobi diagonal) stays in FP64, as in the paper's "CG only" experiments.
"""
from __future__ import annotations

import math

import numpy as np


def round_t(x, t: int):
    """Round to nearest (ties to even) with a t-bit explicit mantissa (t = 52: FP64)."""
    x = np.asarray(x, dtype=np.float64)
    if t >= 52:
        return x.copy()
    m, e = np.frexp(x)                      # x = m 2^e, 0.5 <= |m| < 1
    scaled = np.ldexp(m, t + 1)             # t + 1 significant bits
    return np.ldexp(np.rint(scaled), e - (t + 1))


def random_rounding(x, t, rng):
    """Monte Carlo arithmetic's random rounding (the paper's Sec. 2 MCA mode):
    inexact(x) = x + 2^(e_x - t) xi, xi uniform in [-1/2, 1/2), with e_x the
    exponent of x (x = m 2^e_x, 1 <= |m| < 2); zero stays zero.  The draws
    xi come from the caller's numpy Generator."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1 -> e_x = e - 1
    xi = rng.random(x.shape) - 0.5
    return np.where(x == 0.0, 0.0, x + np.ldexp(xi, e - 1 - t))


def _contract(D, U, axis, t):
    """sum_l D[o, l] U[..., l along `axis`] with every product and partial sum rounded."""
    n = D.shape[0]
    Um = np.moveaxis(U, axis, -1)            # [..., l]
    acc = np.zeros(Um.shape, dtype=np.float64)
    for l in range(n):
        prod = round_t(Um[..., l:l + 1] * D[None, :, l], t)    # [..., o]
        acc = round_t(acc + prod, t)
    return np.moveaxis(acc, -1, axis)


def ax_local_t(P, u, t):
    """The element operator with every operation rounded to t bits."""
    n = P.n
    U = round_t(u, t).reshape(P.E, n, n, n)          # [e, k, j, i]
    D = round_t(P.D, t)
    ur = _contract(D, U, 3, t)
    us = _contract(D, U, 2, t)
    ut = _contract(D, U, 1, t)
    G = [round_t(g, t) for g in P.G]
    grr, gss, gtt, grs, grt, gst = G
    r = lambda a: round_t(a, t)
    vr = r(r(r(grr * ur) + r(grs * us)) + r(grt * ut))
    vs = r(r(r(grs * ur) + r(gss * us)) + r(gst * ut))
    vt = r(r(r(grt * ur) + r(gst * us)) + r(gtt * ut))
    DT = D.T.copy()
    w = r(r(_contract(DT, vr, 3, t) + _contract(DT, vs, 2, t)) + _contract(DT, vt, 1, t))
    return w.reshape(-1)


def dssum_t(P, v, t):
    """QQ^T with the copies of each global node summed in ascending local
    index, each partial sum rounded (vectorised over nodes: pass k adds the
    k-th copy of every node that has one)."""
    order = np.argsort(P.gid, kind="stable")
    g = P.gid[order]
    first = np.r_[True, g[1:] != g[:-1]]
    start = np.maximum.accumulate(np.where(first, np.arange(len(g)), 0))
    rank = np.arange(len(g)) - start
    out = np.zeros(P.U)
    for k in range(int(rank.max()) + 1 if len(g) else 0):
        sel = order[rank == k]
        gk = P.gid[sel]
        out[gk] = round_t(out[gk] + v[sel], t)
    return out[P.gid]


def sweep(P, b, ts, tol=1e-10, maxit=500):
    """Residual versus mantissa bits (the paper's Sec. 3.2 experiment): for
    each t the iterations taken, the last recursive residual and the lowest
    true FP64 residual reached."""
    rows = []
    for t in ts:
        hist, true = pcg_t(P, b, t, tol=tol, maxit=maxit)
        rows.append({"t": t, "iters": len(hist),
                     "recursive": float(hist[-1]) if len(hist) else float("nan"),
                     "true_min": float(true.min()) if len(true) else float("nan")})
    return rows


def dot_t(a, b, c, t):
    """Sequential sum of rounded products a_i c_i b_i (glsc3)."""
    s = 0.0
    prod = round_t(round_t(a * c, t) * b, t)
    for v in prod:
        s = float(round_t(s + v, t))
    return s


def pcg_t(P, b, t, tol=1e-10, maxit=300):
    """Jacobi PCG (profiling-table order) with every loop operation rounded
    to t mantissa bits.  Returns the per-iteration relative residuals
    sqrt(rtr)/||b||_c (rtr itself computed in t-bit arithmetic) and the true
    FP64 residuals ||b - A x||_c/||b||_c."""
    r_ = lambda a: round_t(a, t)
    minv = r_(P.minv)
    c = P.c
    x = np.zeros(P.L)
    r = r_(b)
    bnorm = math.sqrt(float(np.sum(b * c * b)))
    z = r_(minv * r)
    rtz = dot_t(r, z, c, t)
    p = np.zeros(P.L)
    rtz_old = None
    hist, true = [], []
    for _ in range(maxit):
        beta = 0.0 if rtz_old is None else float(r_(rtz / rtz_old))
        p = r_(z + r_(beta * p))
        w = r_(P.mask * dssum_t(P, ax_local_t(P, p, t), t))
        pap = dot_t(w, p, c, t)
        if not pap > 0:
            break
        alpha = float(r_(rtz / pap))
        x = r_(x + r_(alpha * p))
        r = r_(r - r_(alpha * w))
        rtr = dot_t(r, r, c, t)
        hist.append(math.sqrt(max(rtr, 0.0)) / bnorm)
        true.append(P.true_relres(b, x))
        if hist[-1] <= tol:
            break
        z = r_(minv * r)
        rtz_old = rtz
        rtz = dot_t(r, z, c, t)
    return np.array(hist), np.array(true)
