"""Adjoint gradient of a linear functional of the displacement (oracle; test infrastructure).

For L(x) = w^T u(x) with K(x) u = f (Eq. (to)): K(x) lambda = w, dL/dx_e = -lambda_e^T K0 u_e.
For the compliance (w = f) lambda = u and dL/dx_e = -u_e^T K0 u_e, the energy term of KKT3
(Sec. 2).  No counterpart in the paper's algorithms; the closed form is pinned by central finite
differences in the tests.
"""
import numpy as np

from . import fe
from .linsolve import SPDSolver


def grad_linear_functional(prob, x, w, u=None):
    """(dL/dx, u, lambda) for L = w^T u, solving both systems exactly."""
    K = prob.K_free(x)
    solver = SPDSolver(K, prob.grid, prob.free)
    if u is None:
        u = np.zeros(prob.grid.n_dofs)
        u[prob.free] = solver.solve(prob.f[prob.free])
    lam = np.zeros(prob.grid.n_dofs)
    lam[prob.free] = solver.solve(np.asarray(w, dtype=float)[prob.free])
    le = fe.element_values(prob.grid, lam)
    ue = fe.element_values(prob.grid, u)
    g = -np.einsum("ei,ij,ej->e", le, prob.K0, ue)
    return g, u, lam
