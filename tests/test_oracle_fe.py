"""Pins for the oracle's finite-element data (Eq. (to), Sec. 7): element stiffness by exact symbolic
integration, rank and rigid-body null space, closed-form entries, assembly against a dense
loop assembly, the patch test, the energy identity and the paper's printed variable counts."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fe
from oracle.ip import Problem
from paper_1606_06201_gb300 import workloads as W


def _sympy_K0(dim, nu):
    sympy = pytest.importorskip("sympy")
    X = sympy.symbols("x0:%d" % dim)
    E = sympy.Integer(1)
    nu = sympy.Rational(nu).limit_denominator(1000)
    corners = [(0, 0), (1, 0), (1, 1), (0, 1)] if dim == 2 else \
        [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    N = []
    for c in corners:
        p = sympy.Integer(1)
        for a, ca in zip(X, c):
            p *= a if ca else (1 - a)
        N.append(p)
    ncomp = dim
    ndof = len(corners) * ncomp
    # displacement field components as sums over DOFs; strains by symbolic differentiation
    def strain_of_dof(k):
        node, comp = divmod(k, ncomp)
        u = [sympy.Integer(0)] * dim
        u[comp] = N[node]
        g = [[sympy.diff(u[i], X[j]) for j in range(dim)] for i in range(dim)]
        if dim == 2:
            return [g[0][0], g[1][1], g[0][1] + g[1][0]]
        return [g[0][0], g[1][1], g[2][2], g[1][2] + g[2][1], g[0][2] + g[2][0], g[0][1] + g[1][0]]
    if dim == 2:
        c = E / (1 - nu ** 2)
        D = sympy.Matrix([[c, c * nu, 0], [c * nu, c, 0], [0, 0, c * (1 - nu) / 2]])
    else:
        lam = E * nu / ((1 + nu) * (1 - 2 * nu))
        mu = E / (2 * (1 + nu))
        D = sympy.zeros(6, 6)
        for i in range(3):
            for j in range(3):
                D[i, j] = lam + (2 * mu if i == j else 0)
        for i in range(3, 6):
            D[i, i] = mu
    eps = [sympy.Matrix(strain_of_dof(k)) for k in range(ndof)]
    K = np.zeros((ndof, ndof))
    for a in range(ndof):
        for b in range(a, ndof):
            integrand = sympy.expand((eps[a].T * D * eps[b])[0, 0])
            val = integrand
            for v in X:
                val = sympy.integrate(val, (v, 0, 1))
            K[a, b] = K[b, a] = float(val)
    return K


def test_K0_2d_exact_integration():
    K0 = fe.element_stiffness(2, 1.0, 0.3)
    Kx = _sympy_K0(2, 0.3)
    np.testing.assert_allclose(K0, Kx, rtol=0, atol=1e-14)


def test_K0_2d_closed_form_entries():
    nu = 0.3
    K0 = fe.element_stiffness(2, 1.0, nu)
    c = 1.0 / (1.0 - nu * nu)
    # diagonal: int (dN/dx)^2 D11 + (dN/dy)^2 D33 = c (1/3 + (1-nu)/6)
    np.testing.assert_allclose(np.diag(K0), c * (0.5 - nu / 6.0), rtol=1e-14)
    # x-y coupling at one node: (D12 + D33)/4 = c (1 + nu)/8
    np.testing.assert_allclose(K0[0, 1], c * (1.0 + nu) / 8.0, rtol=1e-14)
    assert abs(K0[0, 0] - 0.45 / 0.91) < 1e-15 + 1e-15 * 0.5


@pytest.mark.parametrize("dim", [2, 3])
def test_K0_rank_and_rigid_modes(dim):
    K0 = fe.element_stiffness(dim, 1.0, 0.3)
    assert np.allclose(K0, K0.T, atol=1e-15)
    ev = np.linalg.eigvalsh(K0)
    nrigid = 3 if dim == 2 else 6
    assert np.all(ev[:nrigid] < 1e-13) and ev[nrigid] > 1e-3
    corners = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float) if dim == 2 else \
        np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float)
    modes = []
    for c in range(dim):
        t = np.zeros((len(corners), dim)); t[:, c] = 1.0
        modes.append(t.ravel())
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (0, 2)]
    for a, b in pairs:
        rot = np.zeros((len(corners), dim))
        rot[:, a] = -corners[:, b]
        rot[:, b] = corners[:, a]
        modes.append(rot.ravel())
    for mvec in modes:
        assert np.abs(K0 @ mvec).max() < 1e-14


def test_K0_3d_exact_integration_and_closed_form():
    nu = 0.3
    K0 = fe.element_stiffness(3, 1.0, nu)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    # diagonal: (lam + 2 mu)/9 + 2 mu/9 (each squared derivative integrates to 1/9)
    np.testing.assert_allclose(np.diag(K0), (lam + 4 * mu) / 9.0, rtol=1e-14)
    Kx = _sympy_K0(3, nu)
    np.testing.assert_allclose(K0, Kx, rtol=0, atol=1e-14)
    # K0 scales with the element size h in 3D and is h-independent in 2D
    np.testing.assert_allclose(fe.element_stiffness(3, 1.0, nu, h=2.0), 2.0 * K0, rtol=1e-14)
    np.testing.assert_allclose(fe.element_stiffness(2, 1.0, nu, h=2.0), fe.element_stiffness(2, 1.0, nu), rtol=1e-14)


def _dense_assembly(grid, K0, x):
    """Loop-by-loop dense assembly straight from the numbering conventions."""
    n = grid.n_dofs
    K = np.zeros((n, n))
    d = grid.dim
    e = 0
    rng_z = range(grid.nz) if d == 3 else [None]
    for ez in rng_z:
        for ey in range(grid.ny):
            for ex in range(grid.nx):
                if d == 2:
                    nodes = [(ex, ey), (ex + 1, ey), (ex + 1, ey + 1), (ex, ey + 1)]
                    ids = [i + (grid.nx + 1) * j for i, j in nodes]
                else:
                    base = [(ex, ey), (ex + 1, ey), (ex + 1, ey + 1), (ex, ey + 1)]
                    ids = [i + (grid.nx + 1) * (j + (grid.ny + 1) * ez) for i, j in base] + \
                          [i + (grid.nx + 1) * (j + (grid.ny + 1) * (ez + 1)) for i, j in base]
                dofs = [d * nid + c for nid in ids for c in range(d)]
                for a, ga in enumerate(dofs):
                    for b, gb in enumerate(dofs):
                        K[ga, gb] += x[e] * K0[a, b]
                e += 1
    return K


@pytest.mark.parametrize("shape", [(1, 1, 0), (2, 1, 0), (3, 2, 0), (2, 1, 1), (2, 2, 2)])
def test_assembly_matches_dense_loops(shape):
    grid = fe.Grid(*shape)
    K0 = fe.element_stiffness(grid.dim)
    x = np.random.default_rng(0).uniform(0.1, 1.0, grid.n_elems)
    np.testing.assert_allclose(fe.assemble(grid, K0, x).toarray(), _dense_assembly(grid, K0, x),
                               rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape", [(1, 1, 0), (3, 2, 0), (2, 2, 2), (5, 3, 2)])
def test_matrix_free_apply_matches_dense_loops(shape):
    """apply_K (chunked gathers and a weighted bincount) against the dense assembly by loops,
    with chunks smaller than the element count so that the chunk seams are crossed."""
    grid = fe.Grid(*shape)
    K0 = fe.element_stiffness(grid.dim)
    rng = np.random.default_rng(3)
    x = rng.uniform(0.1, 1.0, grid.n_elems)
    u = rng.standard_normal(grid.n_dofs)
    np.testing.assert_allclose(fe.apply_K(grid, K0, x, u, chunk=2), _dense_assembly(grid, K0, x) @ u,
                               rtol=0, atol=1e-13 * np.abs(u).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_test_uniform_strain(dim):
    grid = fe.Grid(4, 3) if dim == 2 else fe.Grid(3, 3, 2)
    K0 = fe.element_stiffness(dim)
    K = fe.assemble(grid, K0, np.ones(grid.n_elems))
    rng = np.random.default_rng(1)
    G = rng.standard_normal((dim, dim))
    nx1, ny1 = grid.nx + 1, grid.ny + 1
    nid = np.arange(grid.n_nodes)
    coords = [nid % nx1, (nid // nx1) % ny1] + ([nid // (nx1 * ny1)] if dim == 3 else [])
    coords = np.stack(coords, axis=1).astype(float)
    u = (coords @ G.T).ravel()
    fint = (K @ u).reshape(-1, dim)
    interior = np.all([(coords[:, a] > 0) & (coords[:, a] < [grid.nx, grid.ny, grid.nz][a])
                       for a in range(dim)], axis=0)
    assert interior.any()
    assert np.abs(fint[interior]).max() < 1e-12


def test_energy_identity_at_solution():
    cfg = W.cantilever_2d(8, 4, 0.5)
    grid = fe.Grid(8, 4)
    K0 = fe.element_stiffness(2)
    prob = Problem(grid, K0, cfg["fixed"], cfg["f"], cfg["V"], 1.0)
    x = np.random.default_rng(2).uniform(0.2, 1.0, grid.n_elems)
    u = prob.solve_u(x)
    e = fe.element_energy(grid, K0, u)
    c = prob.f @ u
    K = fe.assemble(grid, K0, x)
    np.testing.assert_allclose(np.sum(x * e), c, rtol=1e-12)
    np.testing.assert_allclose(u @ (K @ u), c, rtol=1e-12)


def test_variable_counts_printed_in_tables():
    # problem "abc" = a x b coarsest mesh with c levels -> (a 2^(c-1)) x (b 2^(c-1)) finest
    # tab:1 223 -> 144 variables (free DOFs, +1 for lambda in IP: 145)
    nx, ny = 2 * 4, 2 * 4
    assert int(np.count_nonzero(W.clamp_xmin(nx, ny) == 0)) == 144
    # tab:3 429 -> 1,050,624
    nx, ny = 4 * 256, 2 * 256
    assert int(np.count_nonzero(W.clamp_xmin(nx, ny) == 0)) == 1050624
    # Example 3 counts all DOFs: 822 -> 170, 828 -> 526,850
    assert W.n_dofs(16, 4) == 170
    assert W.n_dofs(8 * 128, 2 * 128) == 526850
    # configuration sizes: 64x32 has 4,290 DOFs (4,224 free); 512x256 has 263,682 (263,168 free)
    assert W.n_dofs(64, 32) == 4290 and int(np.count_nonzero(W.clamp_xmin(64, 32) == 0)) == 4224
    assert W.n_dofs(512, 256) == 263682
    assert int(np.count_nonzero(W.clamp_xmin(512, 256) == 0)) == 263168


def test_cholesky_matches_dense_solve():
    from oracle.linsolve import SPDSolver
    for shape in [(6, 4, 0), (4, 8, 0), (3, 2, 2)]:
        grid = fe.Grid(*shape)
        K0 = fe.element_stiffness(grid.dim)
        fixed = W.clamp_xmin(*shape).astype(bool)
        free = fe.free_dofs(fixed)
        x = np.random.default_rng(3).uniform(0.05, 1.0, grid.n_elems)
        K = fe.assemble(grid, K0, x)[free][:, free]
        b = np.random.default_rng(4).standard_normal(free.size)
        s = SPDSolver(K, grid, free)
        assert s.kind == "banded-cholesky"
        np.testing.assert_allclose(s.solve(b), np.linalg.solve(K.toarray(), b), rtol=1e-10, atol=1e-12)
