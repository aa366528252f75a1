"""CUDA path against the CPU oracle through the C ABI: the matrix-free operator K(x) v, Galerkin
coarse operators, one V-cycle (Algorithm MG), the full MGCG solve (Algorithm PCG) in FP64 and
mixed precision, batched right-hand sides, element energies and the adjoint gradient."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fe, mg
from oracle.linsolve import SPDSolver
from paper_1606_06201_gb300 import workloads as W

from gpu_helpers import dev, host, oracle_hierarchy, oracle_K_free, rel_err, topo_lib, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES_2D = [(1, 1, 0, 1), (2, 1, 0, 1), (6, 4, 0, 2), (16, 8, 0, 3), (64, 32, 0, 3), (96, 40, 0, 4)]
SHAPES_3D = [(2, 2, 2, 2), (4, 2, 2, 2), (6, 4, 2, 2), (8, 4, 4, 3)]


def _x(nx, ny, nz, seed=11):
    shape = (nz, ny, nx) if nz else (ny, nx)
    return W.log_uniform_field(shape, seed)


@pytest.mark.parametrize("generic", [False, True])
@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D + [(61, 31, 0, 1), (200, 48, 0, 3)])
def test_apply_K_matches_assembled(shape, generic):
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny, nz)
    x = _x(nx, ny, nz)
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, generic_kernels=generic)
    s.set_density(dev(torch, x))
    v = W.random_vector(s.n, 3, fixed)
    y = host(s.apply_K(dev(torch, v)))
    K, free, _ = oracle_K_free(nx, ny, nz, x, fixed.astype(bool))
    ref = np.zeros(s.n)
    ref[free] = K @ v[free]
    assert np.all(y[fixed.astype(bool)] == 0.0)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(16, 8, 0, 3), (64, 32, 0, 4), (200, 48, 0, 4), (8, 4, 4, 3)])
def test_galerkin_level_matrices_match_sparse_rap(shape):
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny, nz)
    x = _x(nx, ny, nz, 12)
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels)
    s.set_density(dev(torch, x))
    levs, _, _, _ = oracle_hierarchy(nx, ny, nz, x, fixed, levels)
    g = fe.Grid(nx, ny, nz)
    fx = fixed.astype(bool)
    for k in range(1, levels):
        from oracle.mg import coarse_fixed
        g, fx = coarse_fixed(g, fx)
        Ae = s.level_matrices(k)
        free = fe.free_dofs(fx)
        A = fe.assemble_elementwise(g, Ae)[free][:, free].toarray()
        ref = levs[k].A.toarray()
        np.testing.assert_allclose(A, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_galerkin_level_matrices_large_2d_fp64():
    """FP64 levels of a 512 x 256 hierarchy, where the first coarse level (32768 elements) is
    built with one thread per coarse element and the deeper ones (8192 elements and fewer) with
    one per entry: the assembled operators against the oracle's sparse P^T A P, compared as
    sparse matrices."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, levels = 512, 256, 5
    fixed = W.clamp_xmin(nx, ny)
    x = _x(nx, ny, 0, 16)
    s = topo.Solver(nx, ny, fixed=fixed, levels=levels)
    s.set_density(dev(torch, x))
    levs, _, _, _ = oracle_hierarchy(nx, ny, 0, x, fixed, levels)
    from oracle.mg import coarse_fixed
    g = fe.Grid(nx, ny)
    fx = fixed.astype(bool)
    for k in range(1, levels):
        g, fx = coarse_fixed(g, fx)
        free = fe.free_dofs(fx)
        A = fe.assemble_elementwise(g, s.level_matrices(k))[free][:, free].tocsr()
        ref = levs[k].A.tocsr()
        diff = (A - ref).tocoo()
        scale = np.abs(ref.data).max()
        assert diff.nnz == 0 or np.abs(diff.data).max() <= 1e-13 * scale, k
    s.close()


@pytest.mark.parametrize("shape", [(64, 32, 0, 5), (200, 48, 0, 4), (8, 4, 4, 3)])
@pytest.mark.parametrize("generic", [False, True])
def test_fp32_hierarchy_matrices_match_sparse_rap(shape, generic):
    """Mixed solvers with fixed damping build the coarse matrices below the coarsest level in FP32
    (from FP32 densities and FP32 child tables) and the coarsest in FP64 from FP32 inputs: each
    level against the oracle's FP64 Galerkin product to FP32 accuracy."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny, nz)
    x = _x(nx, ny, nz, 15)
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, precision=topo.MIXED,
                    generic_kernels=generic)
    s.set_density(dev(torch, x))
    levs, _, _, _ = oracle_hierarchy(nx, ny, nz, x, fixed, levels)
    from oracle.mg import coarse_fixed
    g = fe.Grid(nx, ny, nz)
    fx = fixed.astype(bool)
    checked = 0
    for k in range(1, levels):
        g, fx = coarse_fixed(g, fx)
        if k == 1 and not nz and not generic:
            continue  # matrix-free in mixed precision
        Ae = s.level_matrices(k)
        free = fe.free_dofs(fx)
        A = fe.assemble_elementwise(g, Ae)[free][:, free].toarray()
        ref = levs[k].A.toarray()
        np.testing.assert_allclose(A, ref, rtol=0, atol=2e-6 * np.abs(ref).max())
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("generic", [False, True])
@pytest.mark.parametrize("shape", [(16, 8, 0, 3), (64, 32, 0, 3), (96, 40, 0, 4), (8, 4, 4, 3)])
@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (0, 1)])
def test_vcycle_fp64_matches_oracle(shape, nu, generic):
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny, nz)
    x = _x(nx, ny, nz, 13)
    omega = 0.6 if not nz else 0.5
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, nu1=nu[0], nu2=nu[1], omega=omega,
                    generic_kernels=generic)
    s.set_density(dev(torch, x))
    levs, free, _, _ = oracle_hierarchy(nx, ny, nz, x, fixed, levels)
    r = W.random_vector(s.n, 5, fixed)
    y = host(s.apply_vcycle(dev(torch, r)))
    ref = np.zeros(s.n)
    ref[free] = mg.vcycle(levs, r[free], nu[0], nu[1], omega)
    assert rel_err(y, ref) <= 1e-12


@pytest.mark.parametrize("contrast", [1e-3, 1e-9])
def test_small_coarsest_inverse_newton_schulz_and_fallback(contrast):
    """Coarsest level of 90 DOFs (32 x 16 grid, 3 levels): inverted by FP32 Gauss-Jordan and FP64
    Newton-Schulz steps; with a 1e-9 density block the coarsest matrix is too ill-conditioned for
    the FP32 start, the accuracy check fails and the Cholesky kernels recompute the inverse.  Both
    V-cycles against the oracle's (tolerance: the conditioning of the extreme case)."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, levels = 32, 16, 3
    fixed = W.clamp_xmin(nx, ny)
    x = np.ones(nx * ny)
    xe = x.reshape(ny, nx)
    xe[4:12, 8:24] = contrast
    s = topo.Solver(nx, ny, fixed=fixed, levels=levels, omega=0.6)
    s.set_density(dev(torch, x))
    levs, free, _, _ = oracle_hierarchy(nx, ny, 0, x, fixed, levels)
    r = W.random_vector(s.n, 9, fixed)
    y = host(s.apply_vcycle(dev(torch, r)))
    ref = np.zeros(s.n)
    ref[free] = mg.vcycle(levs, r[free], 2, 2, 0.6)
    assert rel_err(y, ref) <= (1e-12 if contrast > 1e-6 else 1e-6)


@pytest.mark.parametrize("shape", [(64, 32, 0, 3), (128, 64, 0, 5), (8, 4, 4, 2)])
def test_vcycle_mixed_close_to_fp64(shape):
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny, nz)
    x = _x(nx, ny, nz, 14)
    s64 = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels)
    s32 = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, precision=topo.MIXED)
    xd = dev(torch, x)
    s64.set_density(xd)
    s32.set_density(xd)
    r = dev(torch, W.random_vector(s64.n, 6, fixed))
    assert rel_err(host(s32.apply_vcycle(r)), host(s64.apply_vcycle(r))) <= 1e-4


def _solve_case(torch, topo, nx, ny, nz, levels, precision, tol, seed=21):
    fixed = W.clamp_xmin(nx, ny, nz)
    x = _x(nx, ny, nz, seed)
    f = W.normal_load(fixed, seed + 1)
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, precision=precision)
    s.set_density(dev(torch, x))
    u, info = s.solve(dev(torch, f), tol=tol)
    K, free, grid = oracle_K_free(nx, ny, nz, x, fixed.astype(bool))
    exact = np.zeros(s.n)
    exact[free] = SPDSolver(K, grid, free).solve(f[free])
    return host(u), exact, f, info, s


@pytest.mark.parametrize("shape", [(64, 32, 0, 3), (96, 40, 0, 4), (256, 128, 0, 6), (8, 4, 4, 3)])
def test_solve_fp64_matches_cholesky(shape):
    torch = torch_cuda()
    topo = topo_lib()
    u, exact, f, info, _ = _solve_case(torch, topo, *shape, topo.FP64, 1e-13)
    assert info.status == topo.OK and info.rel_residual <= 1e-13
    assert rel_err(u, exact) <= 1e-10
    assert abs(f @ u - f @ exact) <= 1e-10 * abs(f @ exact)


@pytest.mark.parametrize("shape", [(64, 32, 0, 3), (256, 128, 0, 6), (8, 4, 4, 3)])
def test_solve_mixed_matches_cholesky(shape):
    torch = torch_cuda()
    topo = topo_lib()
    u, exact, f, info, _ = _solve_case(torch, topo, *shape, topo.MIXED, 1e-8)
    assert info.status == topo.OK and info.rel_residual <= 1e-8
    assert rel_err(u, exact) <= 1e-6
    assert abs(f @ u - f @ exact) <= 1e-6 * abs(f @ exact)


def test_solve_warm_start_and_zero_rhs():
    torch = torch_cuda()
    topo = topo_lib()
    u, exact, f, info, s = _solve_case(torch, topo, 64, 32, 0, 3, topo.FP64, 1e-10)
    u2, info2 = s.solve(dev(torch, f), u=dev(torch, u), tol=1e-10, use_x0=True)
    assert info2.iterations <= 1
    z, info3 = s.solve(dev(torch, np.zeros(s.n)), tol=1e-8)
    assert info3.iterations == 0 and float(host(z).max()) == 0.0


def test_batched_rhs_equal_individual_solves():
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny = 64, 32
    fixed = W.clamp_xmin(nx, ny)
    x = dev(torch, _x(nx, ny, 0, 31))
    F = np.stack([W.normal_load(fixed, 40 + k) for k in range(3)])
    sb = topo.Solver(nx, ny, fixed=fixed, levels=3, nrhs=3)
    sb.set_density(x)
    U, info = sb.solve(dev(torch, F), tol=1e-12)
    s1 = topo.Solver(nx, ny, fixed=fixed, levels=3)
    s1.set_density(x)
    for k in range(3):
        u, _ = s1.solve(dev(torch, F[k]), tol=1e-12)
        np.testing.assert_allclose(host(U)[k], host(u), rtol=0, atol=1e-14 * np.abs(host(u)).max())


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_modes_give_identical_bits(precision):
    """The replayed 4-iteration graph and the one-launch conditional-while graph run the same
    kernels in the same order: same iterates bit for bit, same counts, also when one right-hand
    side (zero) stops at once and another hits max_iter."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny = 64, 32
    fixed = W.clamp_xmin(nx, ny)
    x = dev(torch, _x(nx, ny, 0, 33))
    F = np.stack([W.normal_load(fixed, 50), np.zeros(fixed.size), W.normal_load(fixed, 51)])
    out = []
    for mode in (0, 1):
        s = topo.Solver(nx, ny, fixed=fixed, levels=3, nrhs=3, precision=precision, max_iter=30)
        s.set_graph_mode(mode)
        s.set_density(x)
        U, info = s.solve(dev(torch, F), tol=1e-10)
        U2, info2 = s.solve(dev(torch, F), tol=1e-30, allow_not_converged=True)
        out.append((host(U), info.iterations, host(U2), info2.iterations, info2.status))
        s.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][2], out[1][2])
    assert out[0][1] == out[1][1] and out[0][3] == out[1][3] and out[0][4] == out[1][4]
    with pytest.raises(topo.TopoError):
        topo.Solver(nx, ny, fixed=fixed, levels=3).set_graph_mode(2)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,nu,nrhs", [((256, 128, 0, 6), (2, 2), 1),
                                           ((128, 64, 0, 5), (1, 1), 2),
                                           ((96, 40, 0, 4), (0, 1), 1),
                                           ((256, 64, 0, 6), (2, 3), 3)])
def test_fused_deep_levels_give_identical_bits(precision, shape, nu, nrhs):
    """The deep levels of the V-cycle in one cluster launch run the same per-node arithmetic as
    the per-sweep launches: V-cycle outputs and whole solves agree bit for bit."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny)
    x = dev(torch, _x(nx, ny, 0, 37))
    R = np.stack([W.random_vector(fixed.size, 60 + k, fixed) for k in range(nrhs)])
    F = np.stack([W.normal_load(fixed, 70 + k) for k in range(nrhs)])
    out = []
    for fused in (False, True):
        s = topo.Solver(nx, ny, fixed=fixed, levels=levels, precision=precision, nu1=nu[0],
                        nu2=nu[1], nrhs=nrhs, max_iter=200)
        s.set_vcycle_fusion(fused)
        s.set_density(x)
        y = host(s.apply_vcycle(dev(torch, R)))
        # (nu1, nu2) = (0, 1) is not a symmetric preconditioner: CG may stall, the bits still agree
        u, info = s.solve(dev(torch, F), tol=1e-9, allow_not_converged=True)
        out.append((y, host(u), info.iterations))
        s.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,nu,nrhs,generic,omega_auto",
                         [((256, 128, 0, 6), (2, 2), 1, False, False),
                          ((96, 40, 0, 4), (1, 1), 2, False, False),
                          ((128, 64, 0, 5), (2, 1), 3, True, False),
                          ((64, 32, 0, 4), (0, 2), 1, False, True)])
def test_coarse_prolongation_with_first_post_sweep_gives_identical_bits(
        precision, shape, nu, nrhs, generic, omega_auto, monkeypatch):
    """On the 2D levels with stored element matrices, the kernel that forms v = z + P z_c for the
    3 x 3 neighbours of a node and sweeps on it gives the bits of the separate prolongation and
    sweep kernels (TOPO_COARSE_PROLONG=0): V-cycle outputs and whole solves."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny)
    x = dev(torch, _x(nx, ny, 0, 39))
    R = np.stack([W.random_vector(fixed.size, 80 + k, fixed) for k in range(nrhs)])
    F = np.stack([W.normal_load(fixed, 90 + k) for k in range(nrhs)])
    out = []
    for sep in ("0", "1"):
        monkeypatch.setenv("TOPO_COARSE_PROLONG", sep)
        s = topo.Solver(nx, ny, fixed=fixed, levels=levels, precision=precision, nu1=nu[0],
                        nu2=nu[1], nrhs=nrhs, max_iter=200, generic_kernels=generic,
                        omega_auto=omega_auto)
        s.set_density(x)
        y = host(s.apply_vcycle(dev(torch, R if nrhs > 1 else R[0])))
        u, info = s.solve(dev(torch, F if nrhs > 1 else F[0]), tol=1e-9,
                          allow_not_converged=True)
        out.append((y, host(u), info.iterations))
        s.close()
    monkeypatch.delenv("TOPO_COARSE_PROLONG")
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_levels_with_power_iteration_damping_give_identical_bits(precision):
    """Per-level damping from the power iteration (omega folded into the inverse diagonals):
    the fused kernels take each level's own damping, so fused and unfused V-cycles and solves
    agree bit for bit."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, levels = 256, 128, 6
    fixed = W.clamp_xmin(nx, ny)
    x = dev(torch, _x(nx, ny, 0, 38))
    r = W.random_vector(fixed.size, 61, fixed)
    f = W.normal_load(fixed, 71)
    out = []
    for fused in (False, True):
        s = topo.Solver(nx, ny, fixed=fixed, levels=levels, precision=precision, omega_auto=True)
        s.set_vcycle_fusion(fused)
        s.set_density(x)
        y = host(s.apply_vcycle(dev(torch, r)))
        u, info = s.solve(dev(torch, f), tol=1e-9)
        out.append((y, host(u), info.iterations))
        s.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("precision", [0, 1])
def test_pair_arithmetic_outer_operator_reaches_tight_tolerances(precision):
    """The outer operator in float pairs (about 48 bits): solves to 1e-11 whose true residual, by
    the oracle's sparse matrix, is at that level; and the same iteration count (within one) and
    solution (to the conditioning of the solve) as the FP64 operator."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, levels = 256, 128, 6
    fixed = W.clamp_xmin(nx, ny)
    x = _x(nx, ny, 0, 39)
    f = W.normal_load(fixed, 40)
    K, free, _ = oracle_K_free(nx, ny, 0, x, fixed.astype(bool))
    res = {}
    for mode in (0, 1):
        s = topo.Solver(nx, ny, fixed=fixed, levels=levels, precision=precision)
        s.set_outer_precision(mode)
        s.set_density(dev(torch, x))
        u, info = s.solve(dev(torch, f), tol=1e-11)
        uh = host(u)
        r = np.linalg.norm(f[free] - K @ uh[free]) / np.linalg.norm(f[free])
        assert r <= 3e-11, (mode, r)
        res[mode] = (uh, info.iterations)
        s.close()
    assert abs(res[0][1] - res[1][1]) <= 1
    assert rel_err(res[1][0], res[0][0]) <= 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_pair_arithmetic_hex_outer_operator(precision):
    """The 3D Walsh-Hadamard outer operator in float pairs, batched (3 load cases): solves to
    1e-11 whose true residual by the oracle's sparse matrix is at that level, and the FP64
    operator's iteration counts (within one) and solutions (to 1e-9)."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = 16, 8, 8, 3
    cfg = W.random_field_3d(nx, ny, nz, n_rhs=3)
    K, free, _ = oracle_K_free(nx, ny, nz, cfg["x"], cfg["fixed"].astype(bool))
    res = {}
    for mode in (0, 1):
        s = topo.Solver(nx, ny, nz, fixed=cfg["fixed"], levels=levels, precision=precision, nrhs=3)
        s.set_outer_precision(mode)
        s.set_density(dev(torch, cfg["x"]))
        U, info = s.solve(dev(torch, cfg["f"]), tol=1e-11)
        Uh = host(U)
        for r in range(3):
            f = cfg["f"][r]
            rr = np.linalg.norm(f[free] - K @ Uh[r][free]) / np.linalg.norm(f[free])
            assert rr <= 3e-11, (mode, r, rr)
        res[mode] = (Uh, info.iterations)
        s.close()
    assert abs(res[0][1] - res[1][1]) <= 1
    assert rel_err(res[1][0], res[0][0]) <= 1e-9


@pytest.mark.parametrize("precision,nrhs", [(0, 1), (1, 1), (1, 3)])
def test_solve_from_host_buffers_matches_device_solve(precision, nrhs):
    """topo_solve_host (copies in and out inside the call, b copied while the hierarchy is built)
    gives the bits of topo_set_density + topo_solve on device buffers."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny = 128, 64
    fixed = W.clamp_xmin(nx, ny)
    x = _x(nx, ny, 0, 17)
    F = np.stack([W.normal_load(fixed, 80 + k) for k in range(nrhs)])
    s = topo.Solver(nx, ny, fixed=fixed, levels=4, precision=precision, nrhs=nrhs)
    s.set_density(dev(torch, x))
    u_dev, info_dev = s.solve(dev(torch, F), tol=1e-9)
    xh = torch.as_tensor(x).contiguous().pin_memory()
    fh = torch.as_tensor(F).contiguous().pin_memory()
    uh = torch.full_like(fh, float("nan")).pin_memory()
    info = s.solve_host(xh, fh, uh, tol=1e-9)
    assert info.status == topo.OK and info.iterations == info_dev.iterations
    np.testing.assert_array_equal(uh.numpy(), host(u_dev))
    # pageable host memory works too
    uh2 = torch.zeros_like(fh)
    s.solve_host(torch.as_tensor(x).contiguous(), torch.as_tensor(F).contiguous(), uh2, tol=1e-9)
    np.testing.assert_array_equal(uh2.numpy(), host(u_dev))
    s.close()


def test_profiling_times_every_kernel_kind_and_keeps_results():
    """Profiling inserts event nodes only: the iterate is bit-identical to an unprofiled solve,
    and every kernel kind of the iteration is timed once per CG iteration."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny = 128, 64
    fixed = W.clamp_xmin(nx, ny)
    x = dev(torch, _x(nx, ny, 0, 35))
    f = dev(torch, W.normal_load(fixed, 36))
    s = topo.Solver(nx, ny, fixed=fixed, levels=4, precision=topo.MIXED)
    s.set_density(x)
    u0, info0 = s.solve(f, tol=1e-9)
    s.set_profiling(True)  # the outer operator only
    u1, info1 = s.solve(f, tol=1e-9)
    assert torch.equal(u0, u1) and info0.iterations == info1.iterations
    assert s.profile()[1] == info1.iterations
    assert all(s.profile_kernel(k)[1] == 0 for k in range(1, len(topo.Solver.PROFILE_KINDS)))
    s.set_profiling_mask((1 << len(topo.Solver.PROFILE_KINDS)) - 1)
    u2, info2 = s.solve(f, tol=1e-9)
    assert torch.equal(u0, u2) and info0.iterations == info2.iterations
    fused_restriction = topo.Solver.PROFILE_KINDS.index("fine_restriction")
    ge3 = topo.Solver.PROFILE_KINDS.index("vcycle_levels_ge3")
    for k in range(len(topo.Solver.PROFILE_KINDS)):
        ms, cnt = s.profile_kernel(k)
        if k == fused_restriction:  # one kernel with the residual (timed as fine_residual)
            assert cnt == 0, (k, ms, cnt)
        elif k >= ge3:  # levels >= 3 of 4: inside the fused deep part; none beyond
            assert cnt in (0, info2.iterations) and (k == ge3 or cnt == 0), (k, ms, cnt)
        else:
            assert cnt == info2.iterations and ms > 0.0, (k, ms, cnt)
    assert s.profile() == s.profile_kernel(0)
    s.set_vcycle_fusion(False)  # separate kernels: every kind timed
    s.set_profiling_mask((1 << len(topo.Solver.PROFILE_KINDS)) - 1)  # (resets the sums)
    u3, info3 = s.solve(f, tol=1e-9)
    assert torch.equal(u0, u3) and info0.iterations == info3.iterations
    for k in range(len(topo.Solver.PROFILE_KINDS)):
        ms, cnt = s.profile_kernel(k)
        if k > ge3:  # levels >= 4 of a 4-level hierarchy: none
            assert cnt == 0, (k, ms, cnt)
        else:
            assert cnt == info3.iterations and ms > 0.0, (k, ms, cnt)
    with pytest.raises(topo.TopoError):
        s.set_profiling_mask(1 << len(topo.Solver.PROFILE_KINDS))
    with pytest.raises(topo.TopoError):
        s.profile_kernel(len(topo.Solver.PROFILE_KINDS))
    s.close()


def test_energy_gradient_and_compliance():
    torch = torch_cuda()
    topo = topo_lib()
    u, exact, f, info, s = _solve_case(torch, topo, 16, 8, 0, 2, topo.FP64, 1e-13)
    grid = fe.Grid(16, 8)
    K0 = fe.element_stiffness(2)
    ud = dev(torch, u)
    E = host(s.element_energy(ud))
    ue = fe.element_values(grid, u)
    # rounding bound of a bilinear form: a few ulps of |u_e|^T |K0| |u_e| (cancellation-free scale)
    scale_u = np.einsum("ei,ij,ej->e", np.abs(ue), np.abs(K0), np.abs(ue))
    assert np.all(np.abs(E - fe.element_energy(grid, K0, u)) <= 64 * 2.2e-16 * scale_u + 1e-300)
    w = W.random_vector(s.n, 9, W.clamp_xmin(16, 8))
    g = host(s.grad_x(dev(torch, w), ud))
    we = fe.element_values(grid, w)
    ref = -np.einsum("ei,ij,ej->e", we, K0, ue)
    scale_w = np.einsum("ei,ij,ej->e", np.abs(we), np.abs(K0), np.abs(ue))
    assert np.all(np.abs(g - ref) <= 64 * 2.2e-16 * scale_w + 1e-300)
    c = s.compliance(dev(torch, f), ud)
    assert abs(c[0] - f @ u) <= 1e-14 * (np.abs(f) @ np.abs(u))


def test_invalid_density_and_breakdown_paths():
    torch = torch_cuda()
    topo = topo_lib()
    s = topo.Solver(16, 8, fixed=W.clamp_xmin(16, 8), levels=2)
    bad = np.full(128, 0.5)
    bad[3] = np.nan
    with pytest.raises(topo.TopoError) as e:
        s.set_density(dev(torch, bad))
    assert e.value.status == topo.E_INVALID_ARG
    bad[3] = -1.0
    with pytest.raises(topo.TopoError):
        s.set_density(dev(torch, bad))
    s.set_density(dev(torch, np.full(128, 0.5)))
    f = dev(torch, W.normal_load(W.clamp_xmin(16, 8), 3))
    # max_iter = 1 cannot reach 1e-12: NOT_CONVERGED, with the iterate still returned
    s1 = topo.Solver(16, 8, fixed=W.clamp_xmin(16, 8), levels=2, max_iter=1)
    s1.set_density(dev(torch, np.full(128, 0.5)))
    u, info = s1.solve(f, tol=1e-12, allow_not_converged=True)
    assert info.status == topo.E_NOT_CONVERGED and info.iterations == 1
    with pytest.raises(topo.TopoError):
        s1.solve(f, tol=1e-12)


def test_full_size_standalone_solve_residual():
    """2048 x 1024 grid (4.2M DOFs, 9 levels) in the timed configuration: the true residual of the
    returned u, by the oracle's sparse matrix, meets the tolerance in both precisions."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg = W.random_field_2d(2048, 1024)
    K, free, _ = oracle_K_free(2048, 1024, 0, cfg["x"], cfg["fixed"].astype(bool))
    f = cfg["f"]
    for prec in (topo.FP64, topo.MIXED):
        s = topo.Solver(2048, 1024, fixed=cfg["fixed"], levels=9, precision=prec)
        s.set_density(dev(torch, cfg["x"]))
        u, info = s.solve(dev(torch, f), tol=1e-8)
        uh = host(u)
        res = np.linalg.norm(f[free] - K @ uh[free]) / np.linalg.norm(f[free])
        assert info.status == topo.OK
        assert res <= 2e-8, (prec, res, info.iterations)
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_3d_point_loads_match_cholesky(precision):
    """3D workload recipe at 16x8x8 (3 levels): 8 unit -z point loads on the x = nx face solved
    together; each displacement against the oracle's exact solve."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg = W.random_field_3d(16, 8, 8, n_rhs=8)
    s = topo.Solver(16, 8, 8, fixed=cfg["fixed"], levels=3, precision=precision, nrhs=8)
    s.set_density(dev(torch, cfg["x"]))
    tol = 1e-12 if precision == 0 else 1e-9
    U, info = s.solve(dev(torch, cfg["f"]), tol=tol)
    assert info.status == topo.OK
    K, free, grid = oracle_K_free(16, 8, 8, cfg["x"], cfg["fixed"].astype(bool))
    solver = SPDSolver(K, grid, free)
    Uh = host(U)
    for r in range(8):
        exact = np.zeros(s.n)
        exact[free] = solver.solve(cfg["f"][r][free])
        assert rel_err(Uh[r], exact) <= (1e-10 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_chebyshev_smoother_solves_and_is_symmetric(precision):
    """Chebyshev smoothing (degree nu on D^{-1} A_k, interval from the power iteration): the solve
    still matches the exact solution and, in FP64, the V-cycle is a symmetric operator."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, L = 128, 64, 5
    fixed = W.clamp_xmin(nx, ny)
    x = _x(nx, ny, 0, 41)
    f = W.normal_load(fixed, 42)
    s = topo.Solver(nx, ny, fixed=fixed, levels=L, precision=precision, smoother=topo.CHEBYSHEV)
    s.set_density(dev(torch, x))
    tol = 1e-12 if precision == 0 else 1e-9
    u, info = s.solve(dev(torch, f), tol=tol)
    K, free, grid = oracle_K_free(nx, ny, 0, x, fixed.astype(bool))
    exact = np.zeros(s.n)
    exact[free] = SPDSolver(K, grid, free).solve(f[free])
    assert info.status == topo.OK
    assert rel_err(host(u), exact) <= (1e-10 if precision == 0 else 1e-6)
    if precision == 0:
        a = W.random_vector(s.n, 43, fixed)
        c = W.random_vector(s.n, 44, fixed)
        Ma = host(s.apply_vcycle(dev(torch, a)))
        Mc = host(s.apply_vcycle(dev(torch, c)))
        assert abs(Ma @ c - a @ Mc) <= 1e-11 * abs(Ma @ c)
        assert a @ Ma > 0
    # a second density: the power iterations start from the first build's vectors
    x2 = _x(nx, ny, 0, 45)
    s.set_density(dev(torch, x2))
    u2, info2 = s.solve(dev(torch, f), tol=tol)
    K2, _, _ = oracle_K_free(nx, ny, 0, x2, fixed.astype(bool))
    exact2 = np.zeros(s.n)
    exact2[free] = SPDSolver(K2, grid, free).solve(f[free])
    assert info2.status == topo.OK
    assert rel_err(host(u2), exact2) <= (1e-10 if precision == 0 else 1e-6)


@pytest.mark.parametrize("shape", [(16, 8, 8, 3, 4), (256, 128, 0, 6, 1)])
def test_autotuner_picks_a_converging_setting(tmp_path, shape):
    """The autotuner times full solves over damped Jacobi (omega, nu), the Chebyshev degree and,
    in 2D, the strip height of the finest-level sweeps; it caches the fastest converging setting
    per (grid, precision, batch) and that setting solves to the tolerance."""
    torch = torch_cuda()
    topo = topo_lib()
    from paper_1606_06201_gb300 import autotune
    nx, ny, nz, levels, nrhs = shape
    if nz:
        cfg = W.random_field_3d(nx, ny, nz, n_rhs=nrhs)
    else:
        cfg = W.random_field_2d(nx, ny)
    x, F = dev(torch, cfg["x"]), dev(torch, cfg["f"])
    path = str(tmp_path / "tune.json")
    best = autotune.autotune(nx, ny, nz, cfg["fixed"], x, F, levels=levels, precision=topo.MIXED,
                             nrhs=nrhs, tol=1e-8, omegas=(0.3, 0.5), sweeps=(1, 2),
                             cheb_degrees=(1, 2), rows=(0, 4, 8), cache_path=path)
    assert best["smoother"] in ("jacobi", "chebyshev") and best["nu"] in (1, 2)
    assert best["ms"] > 0 and best["tried"] == 6 + (0 if nz else 2)
    assert best["rows"] in ((0,) if nz else (0, 4, 8))
    import json
    assert list(json.load(open(path)).values())[0] == best
    s = autotune.solver_for(best, nx, ny, nz, cfg["fixed"], levels, precision=topo.MIXED,
                            nrhs=nrhs)
    s.set_density(x)
    _, info = s.solve(F, tol=1e-8)
    assert info.status == topo.OK and info.rel_residual <= 1e-8


@pytest.mark.parametrize("shape", [(64, 32, 0, 4), (16, 8, 8, 3)])
@pytest.mark.parametrize("kind", ["chebyshev", "omega_auto"])
def test_batched_power_iteration_smoothers_equal_individual_solves(shape, kind):
    """Chebyshev smoothing and the adaptive damping take lambda_max from a build-time power
    iteration on one vector per level: a batch of right-hand sides gets the same smoother as a
    single solve, and the batched solutions equal the individual ones."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny, nz)
    x = dev(torch, _x(nx, ny, nz, 47))
    F = np.stack([W.normal_load(fixed, 80 + k) for k in range(3)])
    kw = dict(smoother=topo.CHEBYSHEV) if kind == "chebyshev" else dict(omega_auto=True)
    sb = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, nrhs=3, **kw)
    sb.set_density(x)
    U, info = sb.solve(dev(torch, F), tol=1e-12)
    assert info.status == topo.OK
    s1 = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, **kw)
    s1.set_density(x)
    for k in range(3):
        u, _ = s1.solve(dev(torch, F[k]), tol=1e-12)
        np.testing.assert_allclose(host(U)[k], host(u), rtol=0, atol=1e-12 * np.abs(host(u)).max())
    sb.close()
    s1.close()


def test_bounded_wait_expiry_stops_the_solve_with_timeout_and_the_solver_recovers():
    """The deep V-cycle levels wait for their bulk copies with a bound on the global timer.  With
    the bound set to 0 the first wait gives up at once: the copies still land under a second
    bounded wait, the CG stops with TOPO_E_TIMEOUT, and the context stays usable: with the bound
    restored the next solve gives the bits of the solve before."""
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny = 256, 128
    fixed = W.clamp_xmin(nx, ny)
    x = dev(torch, _x(nx, ny, 0, 51))
    f = dev(torch, W.normal_load(fixed, 52))
    s = topo.Solver(nx, ny, fixed=fixed, levels=6, precision=topo.MIXED)
    s.set_density(x)
    u0, info0 = s.solve(f, tol=1e-8)
    assert info0.status == topo.OK
    s.set_wait_limit_ns(0)
    with pytest.raises(topo.TopoError) as e:
        s.solve(f, tol=1e-8)
    assert e.value.status == topo.E_TIMEOUT
    s.set_wait_limit_ns(10**9)
    u1, info1 = s.solve(f, tol=1e-8)
    assert info1.status == topo.OK and info1.iterations == info0.iterations
    np.testing.assert_array_equal(host(u1), host(u0))
    s.close()
