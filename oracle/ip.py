"""Primal-dual interior-point method for the VTS minimum-compliance problem (oracle; test
infrastructure).  Restates Sec. 2 (KKT conditions, perturbed complementarity, Newton system
Eq. (nwt), its reduction Eq. (nwtr) and the augmented SPD system Eq. (nwtr2), (nwtr2Z),
(nwtr2rhs)) and Sec. 3 (the algorithm, barrier update sigma = 0.2, the 0.9 step-length rule,
the Newton and IP stopping rules), with every Newton system solved exactly (bordering with
banded Cholesky).

Readings of the paper used here (where it is ambiguous or its printed formulas disagree):
  * Newton row 3 (Eq. (nwt)): the printed symmetric matrix is kept and the right-hand side of
    row 3 is F3_i = -1/2 u^T K_i u - lambda - phi_i + psi_i; with that choice the direction
    solves J d = -F for the Jacobian J of the KKT map F (checked against a finite-difference
    Jacobian).  Res1 = f - K(x) u, Res2 = V - sum x, Res4 = s - phi x, Res5 = r - psi (xbar - x).
  * Eq. (phipsi2): d_psi = (xbar - x)^{-1} (Res5 + Psi d_x) (plus sign; the one that reproduces
    Eq. (nwtr)); Eq. (phipsi1): d_phi = X^{-1} (Res4 - Phi d_x).
  * Eq. (nwtr2Za) is garbled in print; d_x is recovered from row 3 of Eq. (nwtr):
    d_x = D^{-1} (B(u)^T d_u + e d_lambda - tilde Res3), D = X^{-1} Phi + (xbar - x)^{-1} Psi.
  * Norms in the Newton stopping rule are Euclidean; the test runs after the update, at the
    new iterate, with the current s and r.
  * Step length: the 0.9 fraction-to-boundary rule is applied to x (both bounds) and also to
    phi and psi (KKT6 requires them non-negative); ``step_rule="x_only"`` is the literal
    reading that bounds only x.  The minimum over an empty set is +inf.
  * The initial u is the exact solution of K(x0) u = f.
Vectors u are full length (zeros on fixed DOFs); solves act on the free DOFs.
"""
import numpy as np
import scipy.sparse as sp

from . import fe
from .linsolve import SPDSolver, solve_arrow


class Problem:
    """min 1/2 f^T u  s.t.  K(x) u = f, sum x = V, 0 <= x <= xbar  (Eq. (to))."""

    def __init__(self, grid, K0, fixed, f, V, xbar):
        self.grid, self.K0 = grid, np.asarray(K0, dtype=float)
        self.fixed = np.asarray(fixed, dtype=bool)
        self.free = fe.free_dofs(self.fixed)
        self.f = np.asarray(f, dtype=float) * (~self.fixed)
        self.V, self.xbar = float(V), float(xbar)
        self.m = grid.n_elems

    def K_free(self, x):
        K = fe.assemble(self.grid, self.K0, x)
        return K[self.free][:, self.free].tocsr()

    def solve_u(self, x):
        """Exact u = K(x)^{-1} f (full length, zeros on fixed DOFs)."""
        K = self.K_free(x)
        u = np.zeros(self.grid.n_dofs)
        u[self.free] = SPDSolver(K, self.grid, self.free).solve(self.f[self.free])
        return u


def kkt_residuals(prob, K0, u, lam, x, phi, psi, s, r):
    """Res1, Res2, F3 (row-3 right-hand side), Res4, Res5, tilde Res3, D and g_e = K0 u_e."""
    grid = prob.grid
    Kx = fe.assemble(grid, K0, x)
    res1 = prob.f - Kx @ u
    res1[prob.fixed] = 0.0
    res2 = prob.V - np.sum(x)
    ue = fe.element_values(grid, u)
    g = ue @ K0.T                                   # g_e = K0 u_e, the columns of B(u)
    energy_half = 0.5 * np.einsum("ei,ei->e", ue, g)
    f3 = -energy_half - lam - phi + psi
    res4 = s - phi * x
    res5 = r - psi * (prob.xbar - x)
    rt3 = f3 - res4 / x + res5 / (prob.xbar - x)
    D = phi / x + psi / (prob.xbar - x)
    return res1, res2, f3, res4, res5, rt3, D, g


def newton_direction(prob, z, s, r):
    """Exact Newton direction via the augmented system Eq. (nwtr2) (bordering), then d_x from
    row 3 of Eq. (nwtr) and d_phi, d_psi from Eq. (phipsi1)-(phipsi2)."""
    u, lam, x, phi, psi = z
    grid, K0 = prob.grid, prob.K0
    res1, res2, f3, res4, res5, rt3, D, g = kkt_residuals(prob, K0, u, lam, x, phi, psi, s, r)
    # Z_uu = K(x) + sum_e g_e g_e^T / D_e (element-local rank-one terms), Z_ul, Z_ll
    Ke = x[:, None, None] * K0[None] + np.einsum("ei,ej->eij", g, g) / D[:, None, None]
    Zuu = fe.assemble_elementwise(grid, Ke)[prob.free][:, prob.free].tocsr()
    z_ul = fe.scatter_add(grid, g / D[:, None])[prob.free]
    z_ll = float(np.sum(1.0 / D))
    rhs_u = (res1 + fe.scatter_add(grid, g * (rt3 / D)[:, None]))[prob.free]
    rhs_l = res2 + float(np.sum(rt3 / D))
    solver = SPDSolver(Zuu, grid, prob.free)
    du_free, dlam = solve_arrow(solver, z_ul, z_ll, rhs_u, rhs_l)
    du = np.zeros(grid.n_dofs)
    du[prob.free] = du_free
    Btdu = np.einsum("ei,ei->e", g, fe.element_values(grid, du))
    dx = (Btdu + dlam - rt3) / D
    dphi = (res4 - phi * dx) / x
    dpsi = (res5 + psi * dx) / (prob.xbar - x)
    return (du, dlam, dx, dphi, dpsi), dict(Zuu=Zuu, z_ul=z_ul, z_ll=z_ll, rhs_u=rhs_u, rhs_l=rhs_l)


def _ratio_min(v, dv, sign):
    """min over {i: sign*dv_i < 0} of -v_i/dv_i (fraction to the boundary), +inf if empty."""
    mask = sign * dv < 0
    if not np.any(mask):
        return np.inf
    return float(np.min(-v[mask] / dv[mask]))


def step_length(prob, z, d, frac=0.9, step_rule="all"):
    """Sec. 3.3: alpha = min(alpha_l, alpha_u, 1) with the 0.9 rule (optionally also on phi, psi)."""
    _, _, x, phi, psi = z
    _, _, dx, dphi, dpsi = d
    a_l = frac * _ratio_min(x, dx, +1)
    a_u = frac * _ratio_min(prob.xbar - x, -dx, +1)
    alphas = [a_l, a_u, 1.0]
    if step_rule == "all":
        alphas += [frac * _ratio_min(phi, dphi, +1), frac * _ratio_min(psi, dpsi, +1)]
    return min(alphas)


def newton_criterion(prob, z, s, r):
    """||Res1|| / ||f|| + ||tilde Res3|| / (||phi|| + ||psi||) at z (Sec. 3.4)."""
    u, lam, x, phi, psi = z
    res1, _, _, _, _, rt3, _, _ = kkt_residuals(prob, prob.K0, u, lam, x, phi, psi, s, r)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f)
            + np.linalg.norm(rt3) / (np.linalg.norm(phi) + np.linalg.norm(psi)))


def kkt_criterion(prob, z, s, r):
    """The scaled KKT residual of the Remark in Sec. 3.4:
    ||Res1|| / ||f|| + ||tilde Res3|| / (||phi|| + ||psi||) + phi^T x / (||phi|| ||x||)
    + psi^T (xbar - x) / (||psi|| ||xbar - x||).  (The printed last denominator repeats
    ||phi|| ||x||; the reading here scales each complementarity term by its own factors.)"""
    u, lam, x, phi, psi = z
    res1, _, _, _, _, rt3, _, _ = kkt_residuals(prob, prob.K0, u, lam, x, phi, psi, s, r)
    xu = prob.xbar - x
    nphi, npsi = np.linalg.norm(phi), np.linalg.norm(psi)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f) + np.linalg.norm(rt3) / (nphi + npsi)
            + float(phi @ x) / (nphi * np.linalg.norm(x))
            + float(psi @ xu) / (npsi * np.linalg.norm(xu)))


def ip_run(prob, sigma=0.2, tau_nwt=0.1, tau_ip=1e-8, frac=0.9, step_rule="all",
           max_newton=500, record=False, stop_rule="barrier", tau_kkt=1e-6, methods=None):
    """Sec. 3.1 algorithm.  Returns (z, info); info counts IP iterations (barrier reductions),
    Newton steps and linear solves (feval), and optionally the per-step trajectory.
    stop_rule "barrier": stop once max(s, r) <= tau_IP (Eq. (crit:ip)); "kkt": stop once the
    scaled KKT residual of the Remark in Sec. 3.4 (kkt_criterion, after each Newton step) is
    <= tau_kkt.  (The Remark names no tolerance of its own; at tau_IP = 1e-8 the tilde Res3
    term stalls near 1e-7, from the rounding of Res4 / x at tiny x, so the test takes its own.)
    ``methods`` = (direction, Newton criterion, KKT criterion) of another model of the same
    form (the SIMP model of Sec. 9); the default is this module's VTS functions."""
    direction, criterion, kkt = methods or (newton_direction, newton_criterion, kkt_criterion)
    m = prob.m
    x = np.full(m, prob.V / m)
    u = prob.solve_u(x)
    z = [u, 1.0, x, np.ones(m), np.ones(m)]
    s = r = 1.0
    info = dict(newton=0, ip=0, feval=1, traj=[])
    while info["newton"] < max_newton:
        d, _ = direction(prob, z, s, r)
        info["feval"] += 1
        alpha = step_length(prob, z, d, frac, step_rule)
        z = [z[0] + alpha * d[0], z[1] + alpha * d[1], z[2] + alpha * d[2],
             z[3] + alpha * d[3], z[4] + alpha * d[4]]
        info["newton"] += 1
        crit = criterion(prob, z, s, r)
        if record:
            info["traj"].append(dict(u=z[0].copy(), lam=z[1], x=z[2].copy(), phi=z[3].copy(),
                                     psi=z[4].copy(), s=s, r=r, alpha=alpha, crit=crit))
        if stop_rule == "kkt" and kkt(prob, z, s, r) <= tau_kkt:
            break
        if crit <= tau_nwt:
            s *= sigma
            r *= sigma
            info["ip"] += 1
            if stop_rule == "barrier" and max(s, r) <= tau_ip:
                break
    info["s"], info["r"] = s, r
    info["compliance"] = float(prob.f @ z[0])
    return z, info


def full_newton_matrix(prob, z):
    """Dense matrix of Eq. (nwt) (size n_free + 1 + 3m) for brute-force checks on tiny grids."""
    u, lam, x, phi, psi = z
    grid, K0 = prob.grid, prob.K0
    free = prob.free
    nf, m = free.size, prob.m
    K = fe.assemble(grid, K0, x)[free][:, free].toarray()
    ue = fe.element_values(grid, u)
    g = ue @ K0.T
    B = np.zeros((grid.n_dofs, m))
    edofs = grid.element_dofs()
    for e in range(m):
        B[edofs[e], e] += g[e]
    B = B[free]
    N = nf + 1 + 3 * m
    J = np.zeros((N, N))
    iu, il, ix, iph, ips = 0, nf, nf + 1, nf + 1 + m, nf + 1 + 2 * m
    J[iu:il, iu:il] = K
    J[iu:il, ix:iph] = B
    J[il, ix:iph] = 1.0
    J[ix:iph, iu:il] = B.T
    J[ix:iph, il] = 1.0
    J[ix:iph, iph:ips] = np.eye(m)
    J[ix:iph, ips:] = -np.eye(m)
    J[iph:ips, ix:iph] = np.diag(phi)
    J[iph:ips, iph:ips] = np.diag(x)
    J[ips:, ix:iph] = -np.diag(psi)
    J[ips:, ips:] = np.diag(prob.xbar - x)
    return J


def kkt_map(prob, z, s, r):
    """F(z) = [K(x)u - f; sum x - V; -1/2 u^T K_i u - lambda - phi + psi; phi x - s;
    psi (xbar - x) - r] on the free DOFs (KKT1-3, KKT4p, KKT5p)."""
    u, lam, x, phi, psi = z
    K = fe.assemble(prob.grid, prob.K0, x)
    F1 = (K @ u - prob.f)[prob.free]
    F2 = np.sum(x) - prob.V
    F3 = -0.5 * fe.element_energy(prob.grid, prob.K0, u) - lam - phi + psi
    F4 = phi * x - s
    F5 = psi * (prob.xbar - x) - r
    return np.concatenate([F1, [F2], F3, F4, F5])
