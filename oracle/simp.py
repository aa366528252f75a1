"""The SIMP model with a density filter and its interior-point method (oracle; test infrastructure).

Restates Sec. 9 ("The SIMP model of topology optimization"):
  * the density filter x~ = W x, with hat W_ij = max(0, r_min - dist(i, j)) and every column of W
    divided by its sum (W_{:i} = hat W_{:i} / sum_j hat W_ij, as printed); dist is the Manhattan
    distance between element centres, in element widths;
  * the equilibrium hat K(x~) u = f with hat K(x~) = sum_i x~_i^p K_i;
  * the modified KKT row 3: -1/2 u^T [p sum_j W_ji x~_j^(p-1) K_j] u - lambda - phi_i + psi_i = 0;
  * the Newton system Eq. (nwtr) (and so Eq. (nwtr2)) with B(u) replaced by
    hat B(u) = (p sum_j W_j1 x~_j^(p-1) K_j u, ..., p sum_j W_jm x~_j^(p-1) K_j u).
The rest of the method (Sec. 2-3: the barrier update, the 0.9 step rule, the Newton and IP stopping
rules, the initial point) is the convex method's, taken from ``oracle.ip``.

Readings used here:
  * The Newton matrix is the printed one with B -> hat B and nothing else changed: the second
    derivative of row 3 in x (non-zero for p > 1) is left out, as the paper's "vanilla" method
    for the non-convex problem does.  The right-hand side is the SIMP residuals
    (Res1 = f - hat K(x~) u, F3 the modified row 3).
  * The volume constraint sum x = V and the bounds 0 <= x <= xbar act on x, not on x~.
  * Column normalisation as printed; since every column of W sums to 1, sum x~ = sum x.

In matrix form hat B(u) = B(u) diag(c) W with c = p x~^(p-1) and B(u) = (K_1 u, ..., K_m u); the
oracle builds exactly that product of sparse matrices and solves the bordered system exactly.
"""
import numpy as np
import scipy.sparse as sp

from . import fe, ip
from .linsolve import SPDSolver, solve_arrow


def filter_matrix(grid, rmin):
    """W of Sec. 9 as a sparse m x m matrix: hat W_ij = max(0, rmin - |di| - |dj| (- |dk|)) over
    element pairs of the grid (element index i = ex + nx (ey + ny ez)), columns normalised."""
    nx, ny, nz = grid.nx, grid.ny, max(grid.nz, 1)
    R = int(np.ceil(rmin)) - 1
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    idx = ex + nx * (ey + ny * ez)
    rows, cols, vals = [], [], []
    dzs = range(-R, R + 1) if grid.dim == 3 else [0]
    for dz in dzs:
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                w = rmin - (abs(dx) + abs(dy) + abs(dz))
                if w <= 0:
                    continue
                jx, jy, jz = ex + dx, ey + dy, ez + dz
                ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
                rows.append(idx[ok])
                cols.append((jx + nx * (jy + ny * jz))[ok])
                vals.append(np.full(int(ok.sum()), float(w)))
    m = grid.n_elems
    What = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(m, m)).tocsr()
    colsum = np.asarray(What.sum(axis=0)).ravel()
    return (What @ sp.diags(1.0 / colsum)).tocsr()


class SimpProblem(ip.Problem):
    """min 1/2 f^T u  s.t.  hat K(W x) u = f, sum x = V, 0 <= x <= xbar (Sec. 9)."""

    def __init__(self, grid, K0, fixed, f, V, xbar, p=3.0, rmin=2.0):
        super().__init__(grid, K0, fixed, f, V, xbar)
        self.p, self.rmin = float(p), float(rmin)
        self.W = filter_matrix(grid, rmin)

    def filtered(self, x):
        """x~ = W x, rho = x~^p (the stiffness coefficients) and c = p x~^(p-1)."""
        xt = self.W @ np.asarray(x, dtype=float)
        return xt, xt ** self.p, self.p * xt ** (self.p - 1.0)

    def K_free(self, x):
        _, rho, _ = self.filtered(x)
        K = fe.assemble(self.grid, self.K0, rho)
        return K[self.free][:, self.free].tocsr()


def columns_B(grid, g):
    """B(u) = (K_1 u, ..., K_m u) as a sparse n x m matrix: column e holds g_e = K0 u_e on the
    DOFs of element e."""
    edofs = grid.element_dofs()
    m, ne = edofs.shape
    cols = np.repeat(np.arange(m), ne)
    return sp.coo_matrix((g.ravel(), (edofs.ravel(), cols)), shape=(grid.n_dofs, m)).tocsr()


def simp_residuals(prob, u, lam, x, phi, psi, s, r):
    """Res1, Res2, F3 (the modified row 3), Res4, Res5, tilde Res3, D and hat B(u)."""
    grid, K0 = prob.grid, prob.K0
    _, rho, c = prob.filtered(x)
    res1 = prob.f - fe.assemble(grid, K0, rho) @ u
    res1[prob.fixed] = 0.0
    res2 = prob.V - np.sum(x)
    ue = fe.element_values(grid, u)
    g = ue @ K0.T
    E = np.einsum("ei,ei->e", ue, g)
    f3 = -0.5 * (prob.W.T @ (c * E)) - lam - phi + psi
    res4 = s - phi * x
    res5 = r - psi * (prob.xbar - x)
    rt3 = f3 - res4 / x + res5 / (prob.xbar - x)
    D = phi / x + psi / (prob.xbar - x)
    Bh = (columns_B(grid, g) @ sp.diags(c) @ prob.W).tocsr()
    return res1, res2, f3, res4, res5, rt3, D, Bh


def newton_direction(prob, z, s, r):
    """Exact direction of Eq. (nwtr2) with hat B(u) in place of B(u) (bordering with banded
    Cholesky), then d_x from row 3 of Eq. (nwtr) and d_phi, d_psi from Eq. (phipsi1)-(phipsi2)."""
    u, lam, x, phi, psi = z
    res1, res2, f3, res4, res5, rt3, D, Bh = simp_residuals(prob, u, lam, x, phi, psi, s, r)
    _, rho, _ = prob.filtered(x)
    Dinv = 1.0 / D
    Z = fe.assemble(prob.grid, prob.K0, rho) + Bh @ sp.diags(Dinv) @ Bh.T
    Zuu = Z.tocsr()[prob.free][:, prob.free].tocsr()
    z_ul = (Bh @ Dinv)[prob.free]
    z_ll = float(np.sum(Dinv))
    rhs_u = (res1 + Bh @ (rt3 * Dinv))[prob.free]
    rhs_l = res2 + float(np.sum(rt3 * Dinv))
    du_free, dlam = solve_arrow(SPDSolver(Zuu, prob.grid, prob.free), z_ul, z_ll, rhs_u, rhs_l)
    du = np.zeros(prob.grid.n_dofs)
    du[prob.free] = du_free
    dx = (Bh.T @ du + dlam - rt3) * Dinv
    dphi = (res4 - phi * dx) / x
    dpsi = (res5 + psi * dx) / (prob.xbar - x)
    return (du, dlam, dx, dphi, dpsi), dict(Zuu=Zuu, z_ul=z_ul, z_ll=z_ll, rhs_u=rhs_u,
                                            rhs_l=rhs_l)


def newton_criterion(prob, z, s, r):
    """||Res1|| / ||f|| + ||tilde Res3|| / (||phi|| + ||psi||) (Sec. 3.4) with the SIMP
    residuals."""
    u, lam, x, phi, psi = z
    res1, _, _, _, _, rt3, _, _ = simp_residuals(prob, u, lam, x, phi, psi, s, r)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f)
            + np.linalg.norm(rt3) / (np.linalg.norm(phi) + np.linalg.norm(psi)))


def kkt_criterion(prob, z, s, r):
    """The scaled KKT residual of the Remark in Sec. 3.4 with the SIMP residuals (the same
    reading of its last denominator as ``oracle.ip.kkt_criterion``)."""
    u, lam, x, phi, psi = z
    xu = prob.xbar - x
    nphi, npsi = np.linalg.norm(phi), np.linalg.norm(psi)
    return (newton_criterion(prob, z, s, r)
            + float(phi @ x) / (nphi * np.linalg.norm(x))
            + float(psi @ xu) / (npsi * np.linalg.norm(xu)))


def ip_run(prob, **kw):
    """The algorithm of Sec. 3.1 on the SIMP problem (keywords as ``oracle.ip.ip_run``)."""
    return ip.ip_run(prob, methods=(newton_direction, newton_criterion, kkt_criterion), **kw)


def kkt_map(prob, z, s, r):
    """F(z) = [hat K(W x) u - f; sum x - V; modified row 3; phi x - s; psi (xbar - x) - r] on the
    free DOFs (Sec. 9 with KKT2, KKT4p, KKT5p)."""
    u, lam, x, phi, psi = z
    _, rho, c = prob.filtered(x)
    F1 = (fe.assemble(prob.grid, prob.K0, rho) @ u - prob.f)[prob.free]
    F2 = np.sum(x) - prob.V
    F3 = -0.5 * (prob.W.T @ (c * fe.element_energy(prob.grid, prob.K0, u))) - lam - phi + psi
    F4 = phi * x - s
    F5 = psi * (prob.xbar - x) - r
    return np.concatenate([F1, [F2], F3, F4, F5])
