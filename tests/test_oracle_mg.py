"""Pins for the oracle's multigrid (Sec. 5, transfers of Sec. 7): exact reproduction of bilinear and
trilinear fields, the variational property P^T K_h P = K_2h, V-cycle symmetry, PCG against a dense
solve, the identity transfer of the IP multiplier."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fe, mg
from oracle.ip import Problem
from oracle.linsolve import SPDSolver
from paper_1606_06201_gb300 import workloads as W


@pytest.mark.parametrize("shape", [(3, 2, 0), (2, 2, 1)])
def test_prolongation_reproduces_multilinear_fields(shape):
    gc = fe.Grid(*shape)
    P = mg.prolongation_full(gc)
    d = gc.dim
    rng = np.random.default_rng(0)
    coef = rng.standard_normal((d, 8))

    def field(coords):
        x, y = coords[:, 0], coords[:, 1]
        z = coords[:, 2] if d == 3 else np.zeros_like(x)
        basis = np.stack([np.ones_like(x), x, y, z, x * y, x * z, y * z, x * y * z], axis=1)
        return (basis @ coef.T).ravel()

    def node_coords(g, scale):
        nid = np.arange(g.n_nodes)
        nx1, ny1 = g.nx + 1, g.ny + 1
        c = [nid % nx1, (nid // nx1) % ny1] + ([nid // (nx1 * ny1)] if d == 3 else [])
        return np.stack(c, axis=1) * scale

    gf = fe.Grid(2 * gc.nx, 2 * gc.ny, 2 * gc.nz)
    uc = field(node_coords(gc, 1.0))
    uf = field(node_coords(gf, 0.5))
    np.testing.assert_allclose(P @ uc, uf, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [(4, 2, 0), (2, 2, 2)])
def test_galerkin_equals_coarse_discretisation(shape):
    """Nested Q1 spaces: P^T K_h(x) P = K_2h(x_c) when x is constant on each coarse element's
    children (K0 is h-independent in 2D and scales with h in 3D)."""
    gc = fe.Grid(*shape)
    gf = fe.Grid(2 * gc.nx, 2 * gc.ny, 2 * gc.nz)
    d = gc.dim
    rng = np.random.default_rng(1)
    xc = rng.uniform(0.1, 1.0, gc.n_elems)
    # fine densities inherited from the parent coarse element
    if d == 2:
        xf = np.repeat(np.repeat(xc.reshape(gc.ny, gc.nx), 2, axis=0), 2, axis=1).ravel()
    else:
        xf = np.repeat(np.repeat(np.repeat(xc.reshape(gc.nz, gc.ny, gc.nx), 2, 0), 2, 1), 2, 2).ravel()
    K0 = fe.element_stiffness(d)
    Kf = fe.assemble(gf, K0, xf)
    P = mg.prolongation_full(gc)
    Kc = fe.assemble(gc, fe.element_stiffness(d, h=2.0), xc)
    np.testing.assert_allclose((P.T @ Kf @ P).toarray(), Kc.toarray(), rtol=0, atol=1e-13)
    # with the clamped boundary: restriction of both sides to the free DOFs
    fixed = W.clamp_xmin(gf.nx, gf.ny, gf.nz).astype(bool)
    Pb, gcc, fixed_c = mg.prolongation(gf, fixed)
    freef, freec = fe.free_dofs(fixed), fe.free_dofs(fixed_c)
    np.testing.assert_allclose((Pb.T @ Kf[freef][:, freef] @ Pb).toarray(),
                               Kc[freec][:, freec].toarray(), rtol=0, atol=1e-13)
    assert np.array_equal(fixed_c, W.clamp_xmin(gc.nx, gc.ny, gc.nz).astype(bool))


def _setup(nx=16, ny=8, levels=3):
    grid = fe.Grid(nx, ny)
    K0 = fe.element_stiffness(2)
    fixed = W.clamp_xmin(nx, ny).astype(bool)
    free = fe.free_dofs(fixed)
    x = W.log_uniform_field((ny, nx), 5)
    K = fe.assemble(grid, K0, x)[free][:, free]
    return grid, fixed, free, K, mg.hierarchy(grid, fixed, K, levels)


def test_vcycle_is_symmetric_and_positive():
    grid, fixed, free, K, levels = _setup()
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal((2, free.size))
    Ma, Mb = mg.vcycle(levels, a, 2, 2, 0.6), mg.vcycle(levels, b, 2, 2, 0.6)
    assert abs(Ma @ b - a @ Mb) <= 1e-12 * abs(Ma @ b)
    assert a @ Ma > 0 and b @ Mb > 0
    # unequal pre/post sweeps break the symmetry (the test would catch a swapped nu)
    Na, Nb = mg.vcycle(levels, a, 2, 1, 0.6), mg.vcycle(levels, b, 2, 1, 0.6)
    assert abs(Na @ b - a @ Nb) > 1e-8 * abs(Na @ b)


def test_vcycle_two_level_with_exact_smoother_limit():
    """One level = the exact coarsest solve: the V-cycle equals A^{-1} b."""
    grid, fixed, free, K, _ = _setup(8, 4)
    levels = mg.hierarchy(grid, fixed, K, 1)
    b = np.random.default_rng(3).standard_normal(free.size)
    np.testing.assert_allclose(mg.vcycle(levels, b), np.linalg.solve(K.toarray(), b), rtol=1e-10)


def test_pcg_converges_to_cholesky():
    grid, fixed, free, K, levels = _setup(32, 16, 4)
    b = np.random.default_rng(4).standard_normal(free.size)
    z, it, hist = mg.pcg(K, b, lambda r: mg.vcycle(levels, r), tol=1e-12)
    exact = SPDSolver(K, grid, free).solve(b)
    assert hist[-1] <= 1e-12 and it < 60
    assert np.linalg.norm(z - exact) <= 1e-9 * np.linalg.norm(exact)
    # without preconditioner on a tiny SPD system, CG is exact after n steps (brute force)
    A = np.array([[4.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 2.0]])
    bb = np.array([1.0, -2.0, 0.5])
    zz, _, _ = mg.pcg(sp.csr_matrix(A), bb, lambda r: r.copy(), tol=1e-14, maxit=3)
    np.testing.assert_allclose(zz, np.linalg.solve(A, bb), rtol=1e-12)


def test_pcg_iterations_flat_in_problem_size():
    """Soft pin (Sec. 7, flat CG counts under refinement): uniform x, iterations to 1e-8 barely grow."""
    its = []
    for nx, ny, L in [(16, 8, 2), (32, 16, 3), (64, 32, 4)]:
        grid = fe.Grid(nx, ny)
        fixed = W.clamp_xmin(nx, ny).astype(bool)
        free = fe.free_dofs(fixed)
        K = fe.assemble(grid, fe.element_stiffness(2), np.full(nx * ny, 0.5))[free][:, free]
        levels = mg.hierarchy(grid, fixed, K, L)
        b = W.point_load(nx, ny, 0, (nx, ny // 2), 1)[free]
        _, it, _ = mg.pcg(K, b, lambda r: mg.vcycle(levels, r), tol=1e-8)
        its.append(it)
    assert max(its) - min(its) <= 4, its


def test_arrow_hierarchy_transfers_lambda_by_identity():
    grid, fixed, free, K, _ = _setup(8, 4)
    rng = np.random.default_rng(5)
    zl = 0.01 * rng.standard_normal(free.size)
    Z = sp.bmat([[K + sp.diags(np.full(free.size, 0.1)), zl[:, None]], [zl[None, :], np.array([[7.0]])]]).tocsr()
    levels = mg.hierarchy(grid, fixed, Z, 2, arrow=True)
    P, _, _ = mg.prolongation(grid, fixed)
    Zc = levels[1].A.toarray()
    np.testing.assert_allclose(Zc[:-1, -1], P.T @ zl, rtol=1e-13)
    assert Zc[-1, -1] == 7.0
