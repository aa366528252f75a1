"""Optimality Conditions methods (oracle; test infrastructure): Algorithm OC with the bisection on
lambda, Algorithm DOC (damped, exponent q) and Algorithm AOC (average of two OC steps), Sec. 4,
with the overall stopping rule Eq. (OCstop), each linear system solved exactly.

Readings of the paper used here:
  * Algorithm OC step 3(c) writes "x = x^NEW" inside the bisection loop; the old x stays fixed
    during the bisection and x becomes x^NEW(lambda) of the last midpoint evaluated.
  * A lower bound xlow > 0 keeps K(x) nonsingular (Sec. 8.2): x^NEW = min(max(x E / lambda,
    xlow), xbar) with the element energy E_i = u^T K_i u (no factor 1/2, Sec. 4.1).
  * Bisection decisions compare the correctly rounded sum of x^NEW (math.fsum) with V:
    "sum > V" raises the lower end, otherwise the upper end is lowered, exactly as printed.
  * AOC: the compliance of record for iteration k is f^T u at x_k (the first solve of the
    iteration); "feval" counts linear solves.
  * DOC uses the same bisection to fix lambda (the printed algorithm leaves lambda implicit).
"""
import math

import numpy as np

from . import fe


def bisect_lambda(x_old, E, V, xbar, xlow, lam_hi=1e4, lam_lo=0.0, tau=1e-11, q=1.0):
    """Step 3 of Algorithm OC: bisection on lambda so that sum x^NEW = V."""
    Eq = E ** q if q != 1.0 else E
    lam = 0.5 * (lam_hi + lam_lo)
    x_new = None
    steps = 0
    while lam_hi - lam_lo > tau:
        lam = 0.5 * (lam_hi + lam_lo)
        x_new = np.minimum(np.maximum(x_old * Eq / lam, xlow), xbar)
        if math.fsum(x_new) > V:
            lam_lo = lam
        else:
            lam_hi = lam
        steps += 1
    if x_new is None:
        x_new = np.minimum(np.maximum(x_old * Eq / lam, xlow), xbar)
    return x_new, lam, steps


def oc_step(prob, x, xlow=1e-6, q=1.0, tau_lam=1e-11):
    """OC(x): u = K(x)^{-1} f, element energies, bisection.  Returns (x_new, u, c, lambda)."""
    u = prob.solve_u(x)
    E = fe.element_energy(prob.grid, prob.K0, u)
    x_new, lam, _ = bisect_lambda(x, E, prob.V, prob.xbar, xlow, tau=tau_lam, q=q)
    return x_new, u, float(prob.f @ u), lam


def oc_run(prob, x0=None, variant="aoc", tau_oc=1e-5, max_feval=10000, xlow=1e-6, q=0.5,
           tau_lam=1e-11, record=False):
    """Run OC / DOC / AOC until |f^T u_k - f^T u_{k-1}| <= tau_oc or the feval budget is spent."""
    m = prob.m
    x = np.full(m, prob.V / m) if x0 is None else np.array(x0, dtype=float)
    info = dict(feval=0, iters=0, compliance=[], traj=[])
    c_prev = None
    while info["feval"] < max_feval:
        if variant == "aoc":
            x1, u, c, lam = oc_step(prob, x, xlow, 1.0, tau_lam)
            info["feval"] += 1
            if info["feval"] >= max_feval:
                info["compliance"].append(c)
                x = x1
                break
            x2, _, _, _ = oc_step(prob, x1, xlow, 1.0, tau_lam)
            info["feval"] += 1
            x_next = 0.5 * (x1 + x2)
        else:
            qq = 1.0 if variant == "oc" else q
            x_next, u, c, lam = oc_step(prob, x, xlow, qq, tau_lam)
            info["feval"] += 1
        info["iters"] += 1
        info["compliance"].append(c)
        if record:
            info["traj"].append(dict(x=x.copy(), u=u.copy(), c=c, lam=lam))
        x = x_next
        if c_prev is not None and abs(c - c_prev) <= tau_oc:
            break
        c_prev = c
    info["x"] = x
    return x, info
