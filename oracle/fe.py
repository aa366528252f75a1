"""Finite-element data of the variable-thickness-sheet problem (oracle; test infrastructure).

Restates Eq. (to) and the discretisation of Sec. 7 of Kocvara & Mohammed (arXiv 1606.06201):
square bilinear (Q1) elements for u, one constant density x_i per element, isotropic
material E = 1, nu = 0.3, K(x) = sum_i x_i K_i where K_i is the element matrix K0 scattered
to the element's DOFs.  Plane stress for the 2D sheet (thickness x_i, unit reference
thickness).  The 3D trilinear hexahedron is the direct analogue (no counterpart in the
paper, which is 2D only).

Numbering (also the layout of every vector the oracle accepts):
  2D: node (i, j) -> i + (nx+1) j;  DOF 2*node + c (c = 0: x, 1: y);
      element (ex, ey) -> ex + nx ey; local nodes counter-clockwise from (ex, ey):
      (ex,ey), (ex+1,ey), (ex+1,ey+1), (ex,ey+1).
  3D: node (i, j, k) -> i + (nx+1)(j + (ny+1) k);  DOF 3*node + c;
      element ex + nx (ey + ny ez); local nodes: the bottom face (z = ez) counter-clockwise
      as in 2D, then the top face (z = ez+1) in the same order.
"""
import numpy as np
import scipy.sparse as sp


class Grid:
    """Structured grid of nx x ny (x nz) unit elements."""

    def __init__(self, nx, ny, nz=0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dim = 3 if nz else 2

    @property
    def n_nodes(self):
        n = (self.nx + 1) * (self.ny + 1)
        return n * (self.nz + 1) if self.dim == 3 else n

    @property
    def n_dofs(self):
        return self.dim * self.n_nodes

    @property
    def n_elems(self):
        m = self.nx * self.ny
        return m * self.nz if self.dim == 3 else m

    def node_id(self, i, j, k=0):
        if self.dim == 2:
            return i + (self.nx + 1) * j
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def element_nodes(self):
        """(m, 4) or (m, 8) global node ids of each element, local order as in the module doc."""
        nx, ny, nz = self.nx, self.ny, self.nz
        if self.dim == 2:
            ey, ex = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
            ex, ey = ex.ravel(), ey.ravel()
            n00 = ex + (nx + 1) * ey
            return np.stack([n00, n00 + 1, n00 + 1 + (nx + 1), n00 + (nx + 1)], axis=1)
        ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
        sx, sxy = 1, (nx + 1)
        plane = (nx + 1) * (ny + 1)
        n000 = ex + (nx + 1) * (ey + (ny + 1) * ez)
        bottom = [n000, n000 + sx, n000 + sx + sxy, n000 + sxy]
        top = [b + plane for b in bottom]
        return np.stack(bottom + top, axis=1)

    def element_dofs(self):
        """(m, 8) or (m, 24) global DOF ids per element in local DOF order (node-major)."""
        en = self.element_nodes()
        d = self.dim
        return (d * en[:, :, None] + np.arange(d)[None, None, :]).reshape(en.shape[0], -1)


def _gauss2():
    """Two-point Gauss-Legendre rule on [0, 1]: points and weights."""
    g = 0.5 / np.sqrt(3.0)
    return np.array([0.5 - g, 0.5 + g]), np.array([0.5, 0.5])


def elasticity_matrix(dim, E=1.0, nu=0.3):
    """Constitutive matrix D: plane stress (2D, Voigt [xx, yy, xy]) or isotropic 3D
    (Voigt [xx, yy, zz, yz, xz, xy]), engineering shear strains."""
    if dim == 2:
        c = E / (1.0 - nu * nu)
        return c * np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, 0.5 * (1.0 - nu)]])
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def element_stiffness(dim, E=1.0, nu=0.3, h=1.0, D=None):
    """Element stiffness K0 = int B^T D B over one square (cube) element of side h with unit
    thickness, by tensor Gauss quadrature (2 points per direction; exact for Q1/trilinear).

    Sec. 7: square elements, bilinear u, E = 1, nu = 0.3.  In 2D K0 does not depend on h;
    in 3D it scales with h.  D: another constitutive matrix (Voigt order as elasticity_matrix),
    for an anisotropic material; default the isotropic one of E, nu.
    """
    D = elasticity_matrix(dim, E, nu) if D is None else np.asarray(D, dtype=float)
    pts, wts = _gauss2()
    if dim == 2:
        corners = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=float)
        K = np.zeros((8, 8))
        for a, wa in zip(pts, wts):
            for b, wb in zip(pts, wts):
                # shape functions N_k = prod (1 - |xi - corner|) on the unit square
                dN = np.zeros((4, 2))
                for k, (cx, cy) in enumerate(corners):
                    fx = a if cx else 1.0 - a
                    fy = b if cy else 1.0 - b
                    sx = 1.0 if cx else -1.0
                    sy = 1.0 if cy else -1.0
                    dN[k] = [sx * fy / h, sy * fx / h]
                B = np.zeros((3, 8))
                B[0, 0::2] = dN[:, 0]
                B[1, 1::2] = dN[:, 1]
                B[2, 0::2] = dN[:, 1]
                B[2, 1::2] = dN[:, 0]
                K += wa * wb * h * h * (B.T @ D @ B)
        return K
    corners = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                        [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=float)
    K = np.zeros((24, 24))
    for a, wa in zip(pts, wts):
        for b, wb in zip(pts, wts):
            for c, wc in zip(pts, wts):
                dN = np.zeros((8, 3))
                for k, (cx, cy, cz) in enumerate(corners):
                    f = [a if cx else 1.0 - a, b if cy else 1.0 - b, c if cz else 1.0 - c]
                    s = [1.0 if cx else -1.0, 1.0 if cy else -1.0, 1.0 if cz else -1.0]
                    dN[k] = [s[0] * f[1] * f[2] / h, s[1] * f[0] * f[2] / h, s[2] * f[0] * f[1] / h]
                B = np.zeros((6, 24))
                B[0, 0::3] = dN[:, 0]
                B[1, 1::3] = dN[:, 1]
                B[2, 2::3] = dN[:, 2]
                B[3, 1::3] = dN[:, 2]
                B[3, 2::3] = dN[:, 1]
                B[4, 0::3] = dN[:, 2]
                B[4, 2::3] = dN[:, 0]
                B[5, 0::3] = dN[:, 1]
                B[5, 1::3] = dN[:, 0]
                K += wa * wb * wc * h ** 3 * (B.T @ D @ B)
    return K


def assemble(grid, K0, x):
    """K(x) = sum_i x_i K_i as a sparse n x n matrix (Eq. (to)), no boundary conditions."""
    edofs = grid.element_dofs()
    ne = edofs.shape[1]
    rows = np.repeat(edofs, ne, axis=1).ravel()
    cols = np.tile(edofs, (1, ne)).ravel()
    vals = (np.asarray(x, dtype=float)[:, None] * K0.ravel()[None, :]).ravel()
    n = grid.n_dofs
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def assemble_elementwise(grid, Ke):
    """sum_i L_i^T Ke[i] L_i for per-element dense matrices Ke (m, ne, ne)."""
    edofs = grid.element_dofs()
    ne = edofs.shape[1]
    rows = np.repeat(edofs, ne, axis=1).ravel()
    cols = np.tile(edofs, (1, ne)).ravel()
    n = grid.n_dofs
    return sp.coo_matrix((np.asarray(Ke).reshape(-1), (rows, cols)), shape=(n, n)).tocsr()


def free_dofs(fixed):
    """Indices of the DOFs that are not fixed (fixed: bool array of length n)."""
    return np.flatnonzero(~np.asarray(fixed, dtype=bool))


def element_values(grid, u):
    """u_e for every element: (m, ne) gather of a full-length vector."""
    return np.asarray(u)[grid.element_dofs()]


def element_energy(grid, K0, u):
    """u_e^T K0 u_e for every element (no factor 1/2)."""
    ue = element_values(grid, u)
    return np.einsum("ei,ij,ej->e", ue, K0, ue)


def apply_K(grid, K0, x, u, chunk=1 << 20):
    """K(x) u = sum_e x_e L_e^T K0 L_e u (Eq. (to)) without assembling K, for grids too large for
    a sparse matrix: element gathers, the element product, and a weighted bincount as the scatter,
    in chunks of elements."""
    edofs = grid.element_dofs()
    x = np.asarray(x, dtype=float)
    u = np.asarray(u, dtype=float)
    out = np.zeros(grid.n_dofs)
    for e0 in range(0, edofs.shape[0], chunk):
        ed = edofs[e0:e0 + chunk]
        ve = (u[ed] @ K0.T) * x[e0:e0 + chunk, None]
        out += np.bincount(ed.ravel(), weights=ve.ravel(), minlength=grid.n_dofs)
    return out


def scatter_add(grid, ve):
    """sum_e L_e^T ve[e]: element vectors (m, ne) to a full-length vector."""
    out = np.zeros(grid.n_dofs)
    np.add.at(out, grid.element_dofs().ravel(), np.asarray(ve).ravel())
    return out
