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
  * Inexact solves (Sec. 6.2): Algorithm PCG with one V-cycle (Algorithm MG) as preconditioner,
    warm-started from the previous u, stopped at ||r|| / ||f|| <= tau; tau starts at tau_0 and
    is multiplied by 0.1 after an iteration whose compliance exceeds the previous iteration's.
    The offending iteration is not redone; the new tau applies from the next solve.
"""
import math

import numpy as np

from . import fe, mg


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


class MGCGSolve:
    """Inexact u = K(x)^{-1} f by multigrid-preconditioned CG (Sec. 5.2, Sec. 6.2): a Galerkin
    hierarchy of K(x) on the free DOFs, damped-Jacobi V-cycles, warm start from the last u.
    ``tau`` is the current relative-residual tolerance; ``iterations`` counts CG iterations."""

    def __init__(self, prob, levels=3, nu1=2, nu2=2, omega=0.6, tau=1e-4, maxit=1000):
        self.prob, self.levels, self.nu1, self.nu2, self.omega = prob, levels, nu1, nu2, omega
        self.tau, self.maxit = tau, maxit
        self.u = None
        self.iterations = 0

    def __call__(self, x):
        prob = self.prob
        K = prob.K_free(x)
        levs = mg.hierarchy(prob.grid, prob.fixed, K, self.levels)
        z0 = None if self.u is None else self.u[prob.free]
        z, it, _ = mg.pcg(K, prob.f[prob.free],
                          lambda r: mg.vcycle(levs, r, self.nu1, self.nu2, self.omega),
                          z0=z0, tol=self.tau, maxit=self.maxit)
        self.iterations += it
        u = np.zeros(prob.grid.n_dofs)
        u[prob.free] = z
        self.u = u
        return u


def oc_step(prob, x, xlow=1e-6, q=1.0, tau_lam=1e-11, solve=None):
    """OC(x): u = K(x)^{-1} f, element energies, bisection.  Returns (x_new, u, c, lambda).
    ``solve``: the linear solver (default: exact banded Cholesky)."""
    u = prob.solve_u(x) if solve is None else solve(x)
    E = fe.element_energy(prob.grid, prob.K0, u)
    x_new, lam, _ = bisect_lambda(x, E, prob.V, prob.xbar, xlow, tau=tau_lam, q=q)
    return x_new, u, float(prob.f @ u), lam


def oc_run(prob, x0=None, variant="aoc", tau_oc=1e-5, max_feval=10000, xlow=1e-6, q=0.5,
           tau_lam=1e-11, record=False, solve=None, adaptive_tol=False):
    """Run OC / DOC / AOC until |f^T u_k - f^T u_{k-1}| <= tau_oc or the feval budget is spent.
    ``solve``: the linear solver (default exact); with an MGCGSolve and ``adaptive_tol`` the
    tolerance follows the Sec. 6.2 rule (info["tau"] lists the tolerance of each iteration)."""
    m = prob.m
    x = np.full(m, prob.V / m) if x0 is None else np.array(x0, dtype=float)
    info = dict(feval=0, iters=0, compliance=[], traj=[], tau=[])
    c_prev = None
    while info["feval"] < max_feval:
        if solve is not None and hasattr(solve, "tau"):
            info["tau"].append(solve.tau)
        if variant == "aoc":
            x1, u, c, lam = oc_step(prob, x, xlow, 1.0, tau_lam, solve)
            info["feval"] += 1
            if info["feval"] >= max_feval:
                info["compliance"].append(c)
                x = x1
                break
            x2, _, _, _ = oc_step(prob, x1, xlow, 1.0, tau_lam, solve)
            info["feval"] += 1
            x_next = 0.5 * (x1 + x2)
        else:
            qq = 1.0 if variant == "oc" else q
            x_next, u, c, lam = oc_step(prob, x, xlow, qq, tau_lam, solve)
            info["feval"] += 1
        info["iters"] += 1
        info["compliance"].append(c)
        if record:
            info["traj"].append(dict(x=x.copy(), u=u.copy(), c=c, lam=lam))
        x = x_next
        if adaptive_tol and c_prev is not None and c > c_prev:
            solve.tau *= 0.1
        if c_prev is not None and abs(c - c_prev) <= tau_oc:
            break
        c_prev = c
    info["x"] = x
    return x, info
