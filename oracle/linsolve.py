"""Exact SPD solves for the oracle (test infrastructure).

The exact solution u = K(x)^{-1} f is the result that MGCG approximates (Sec. 5-6).  The paper
uses MATLAB backslash (CHOLMOD); the oracle uses LAPACK banded Cholesky (pbtrf/pbtrs through
scipy.linalg) on the free DOFs, with the nodes re-ordered so that the shortest grid direction
runs fastest, which keeps the band narrow (Sec. 6.1, the banded structure of K and Z).

The IP matrix Z of Eq. (nwtr2Z) is banded plus one dense row and column (the arrow of
Sec. 6.1); it is solved by bordering: two banded solves with the leading block and a scalar
Schur complement for the last unknown.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def band_ordering(grid, free):
    """Permutation of the free DOF indices (positions in ``free``) that runs the shortest grid
    direction fastest.  Returns perm such that free[perm] is the new order."""
    d = grid.dim
    node = free // d
    comp = free % d
    nx1, ny1 = grid.nx + 1, grid.ny + 1
    i = node % nx1
    j = (node // nx1) % ny1
    if d == 2:
        coords = [i, j]
    else:
        k = node // (nx1 * ny1)
        coords = [i, j, k]
    extents = [grid.nx, grid.ny] + ([grid.nz] if d == 3 else [])
    # sort key: longest direction slowest, shortest fastest, component fastest of all
    order = np.argsort(extents)[::-1]
    keys = [comp] + [coords[a] for a in order[::-1]]
    return np.lexsort(keys)


class BandedCholesky:
    """Cholesky factor of a sparse SPD matrix A stored in LAPACK lower band form."""

    def __init__(self, A, perm):
        A = sp.csr_matrix(A)
        self.perm = np.asarray(perm)
        Ap = A[self.perm][:, self.perm].tocoo()
        low = Ap.row >= Ap.col
        r, c, v = Ap.row[low], Ap.col[low], Ap.data[low]
        self.n = A.shape[0]
        self.bw = int((r - c).max()) if r.size else 0
        ab = np.zeros((self.bw + 1, self.n))
        np.add.at(ab, (r - c, c), v)
        self.cb = sla.cholesky_banded(ab, lower=True, check_finite=False)

    def solve(self, b):
        b = np.asarray(b, dtype=float)
        y = np.empty_like(b)
        y[self.perm] = sla.cho_solve_banded((self.cb, True), b[self.perm], check_finite=False)
        return y


class SPDSolver:
    """Exact solver for an SPD matrix on the free DOFs of a grid.

    Banded Cholesky where the band fits in ``max_band_bytes``; otherwise a sparse direct LU
    (SuperLU), which is still an exact direct method.  ``kind`` says which was used.
    """

    def __init__(self, A, grid, free, max_band_bytes=8 << 30):
        perm = band_ordering(grid, free)
        n = A.shape[0]
        Ap = sp.csr_matrix(A)[perm][:, perm].tocoo()
        bw = int(np.abs(Ap.row - Ap.col).max()) if Ap.nnz else 0
        if (bw + 1) * n * 8 <= max_band_bytes:
            self.kind = "banded-cholesky"
            self._f = BandedCholesky(A, perm)
            self.solve = self._f.solve
        else:
            self.kind = "superlu"
            lu = spla.splu(sp.csc_matrix(A), permc_spec="COLAMD")
            self.solve = lambda b: lu.solve(np.asarray(b, dtype=float))


def solve_arrow(solver_uu, z_ul, z_ll, r_u, r_l):
    """Solve [[Z_uu, z_ul], [z_ul^T, z_ll]] [d_u; d_l] = [r_u; r_l] by bordering.

    Z_uu w1 = r_u, Z_uu w2 = z_ul, s = z_ll - z_ul^T w2 (Schur complement of Z_uu),
    d_l = (r_l - z_ul^T w1) / s, d_u = w1 - d_l w2.
    """
    w1 = solver_uu.solve(r_u)
    w2 = solver_uu.solve(z_ul)
    s = z_ll - float(z_ul @ w2)
    d_l = (r_l - float(z_ul @ w1)) / s
    return w1 - d_l * w2, d_l
