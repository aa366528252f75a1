"""Geometric multigrid and multigrid-preconditioned CG (oracle; test infrastructure).

Restates Sec. 5 (Algorithm MG: V-cycle correction scheme; Algorithm PCG with one V-cycle as
preconditioner) and the transfer operators of Sec. 7 (nine-point bilinear prolongation with
stencil [1/4 1/2 1/4; 1/2 1 1/2; 1/4 1/2 1/4], restriction = its transpose, the IP multiplier
lambda transferred by the identity).  The 3D analogue uses the 27-point trilinear stencil.

Everything here is explicit sparse algebra: P is an assembled sparse matrix and the coarse
operators are the Galerkin products A_{k-1} = P^T A_k P of Sec. 5.1.

Readings of the paper used here:
  * coarse boundary conditions (not stated in the paper): a coarse DOF is fixed iff the fine DOF
    at the same node is fixed; P maps free coarse DOFs to free fine DOFs,
    P = P_full[free_fine][:, free_coarse];
  * the smoother (named only as "typically Gauss-Seidel"): damped Jacobi
    z <- z + omega diag(A)^{-1} (b - A z), nu1 pre- and nu2 post-sweeps;
  * the coarsest level (written k = 0 in Algorithm MG while levels run 1..l) is level 1,
    solved exactly (dense Cholesky);
  * the CG stopping rule "||rho|| ||b|| <= tol" is read as ||rho||_2 / ||b||_2 <= tol.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fe


def _interp_1d(nc):
    """1-D linear interpolation from nc+1 coarse nodes to 2nc+1 fine nodes (sparse)."""
    rows, cols, vals = [], [], []
    for i in range(2 * nc + 1):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc + 1, nc + 1))


def coarse_grid(grid):
    if grid.nx % 2 or grid.ny % 2 or (grid.dim == 3 and grid.nz % 2):
        raise ValueError("grid is not coarsenable by 2 in every direction")
    if grid.dim == 2:
        return fe.Grid(grid.nx // 2, grid.ny // 2)
    return fe.Grid(grid.nx // 2, grid.ny // 2, grid.nz // 2)


def prolongation_full(grid_c):
    """Bilinear (trilinear) prolongation on all DOFs, coarse grid_c -> the 2x finer grid.

    Tensor product of 1-D linear interpolation; node ids run x fastest, so the node matrix is
    kron(Pz, kron(Py, Px)); DOFs are interleaved per node, hence the final kron with I_dim.
    """
    Px, Py = _interp_1d(grid_c.nx), _interp_1d(grid_c.ny)
    Pn = sp.kron(Py, Px)
    if grid_c.dim == 3:
        Pn = sp.kron(_interp_1d(grid_c.nz), Pn)
    return sp.kron(Pn, sp.identity(grid_c.dim)).tocsr()


def coarse_fixed(grid_f, fixed_f):
    """Coarse DOF fixed iff the fine DOF at the coincident node is fixed (injection)."""
    grid_c = coarse_grid(grid_f)
    d = grid_f.dim
    fixed_f = np.asarray(fixed_f, dtype=bool).reshape(-1, d)
    if d == 2:
        nodes = fixed_f.reshape(grid_f.ny + 1, grid_f.nx + 1, d)[::2, ::2]
    else:
        nodes = fixed_f.reshape(grid_f.nz + 1, grid_f.ny + 1, grid_f.nx + 1, d)[::2, ::2, ::2]
    return grid_c, nodes.reshape(-1).copy()


def prolongation(grid_f, fixed_f):
    """P restricted to free DOFs: (free fine) x (free coarse).  Returns (P, grid_c, fixed_c)."""
    grid_c, fixed_c = coarse_fixed(grid_f, fixed_f)
    Pf = prolongation_full(grid_c)
    P = Pf[fe.free_dofs(fixed_f)][:, fe.free_dofs(fixed_c)]
    return P.tocsr(), grid_c, fixed_c


class Level:
    def __init__(self, A, P=None):
        self.A = sp.csr_matrix(A)   # operator on this level
        self.P = P                  # prolongation from the next coarser level to this one
        self.diag = self.A.diagonal()


def hierarchy(grid, fixed, A_fine, n_levels, arrow=False):
    """Galerkin hierarchy (Sec. 5.1): levels[0] finest ... levels[-1] coarsest.

    A_fine acts on the free DOFs (plus one trailing lambda unknown if ``arrow``); the lambda
    unknown is carried to every level by the identity (Sec. 7).
    """
    levels = []
    A = sp.csr_matrix(A_fine)
    g, fx = grid, np.asarray(fixed, dtype=bool)
    for k in range(n_levels):
        if k == n_levels - 1:
            levels.append(Level(A))
            break
        P, gc, fxc = prolongation(g, fx)
        if arrow:
            P = sp.block_diag((P, sp.identity(1))).tocsr()
        levels.append(Level(A, P))
        A = (P.T @ A @ P).tocsr()
        g, fx = gc, fxc
    coarsest = levels[-1]
    coarsest.chol = sla.cho_factor(coarsest.A.toarray(), lower=True)
    return levels


def jacobi(level, b, z, nu, omega):
    """nu damped-Jacobi sweeps z <- z + omega D^{-1} (b - A z)."""
    for _ in range(nu):
        z = z + omega * (b - level.A @ z) / level.diag
    return z


def mgm(levels, k, z, b, nu1, nu2, omega):
    """Algorithm MG, function mgm (Sec. 5.1): one V-cycle correction step at level index k."""
    lev = levels[k]
    if k == len(levels) - 1:
        return sla.cho_solve(lev.chol, b)
    z = jacobi(lev, b, z, nu1, omega)
    r_c = lev.P.T @ (b - lev.A @ z)
    v = mgm(levels, k + 1, np.zeros(r_c.shape[0]), r_c, nu1, nu2, omega)
    z = z + lev.P @ v
    return jacobi(lev, b, z, nu2, omega)


def vcycle(levels, b, nu1=2, nu2=2, omega=0.6):
    """One V-cycle from the zero initial guess: the preconditioner y = M^{-1} b of Algorithm PCG."""
    return mgm(levels, 0, np.zeros_like(b), b, nu1, nu2, omega)


def pcg(A, b, precond, z0=None, tol=1e-8, maxit=1000):
    """Algorithm PCG (Sec. 5.2) with the paper's sign convention r = A z - b, p = -y.

    Stops when ||r||_2 / ||b||_2 <= tol (tested before the first and after every iteration) or
    after maxit iterations.  Returns (z, iterations, history of ||r||/||b||).
    """
    z = np.zeros_like(b) if z0 is None else np.array(z0, dtype=float)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    r = A @ z - b
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= tol:
        return z, 0, hist
    y = precond(r)
    p = -y
    it = 0
    for it in range(1, maxit + 1):
        Ap = A @ p
        ry = float(r @ y)
        alpha = ry / float(p @ Ap)
        z = z + alpha * p
        r_new = r + alpha * Ap
        y_new = precond(r_new)
        beta = float(r_new @ y_new) / ry
        p = -y_new + beta * p
        r, y = r_new, y_new
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            break
    return z, it, hist
