"""The 3D batched and differentiation workloads at their full sizes, through the C ABI.

Full-size direct solves are beyond the oracle, so these tests check what holds at any size, with
the oracle's matrix-free K(x)u (Eq. (to)):
- the true residual of every returned solution meets the solve tolerance;
- the adjoint gradient equals -lam_e^T K0 u_e, evaluated by the oracle on the GPU's own u and lam;
- central differences of the energy functional on 32 seeded high-sensitivity elements agree with
  the compliance gradient (differentiation sizes; the 12.8M-DOF scale run checks the residual and
  the gradient formula).
"""
import numpy as np
import pytest

from oracle import fe
from paper_1606_06201_gb300 import workloads as W

from gpu_helpers import dev, host, topo_lib, torch_cuda

pytestmark = pytest.mark.gpu


def _true_residual(grid, K0, x, fixed, f, u):
    """||f - K(x) u|| / ||f|| over the free DOFs."""
    free = fe.free_dofs(fixed)
    r = f - fe.apply_K(grid, K0, x, u)
    return float(np.linalg.norm(r[free]) / np.linalg.norm(f[free]))


def _energy_bound(grid, K0, a, b):
    """Rounding bound of a_e^T K0 b_e per element: 64 eps |a_e|^T |K0| |b_e| (the products of
    large displacements cancel to small energies)."""
    return 64 * np.finfo(float).eps * np.einsum("ei,ij,ej->e", np.abs(fe.element_values(grid, a)),
                                                 np.abs(K0), np.abs(fe.element_values(grid, b)))


def test_3d_128x64x64_eight_load_cases_batched_with_autotuned_smoother(tmp_path):
    """Eight unit point loads on a 128 x 64 x 64 hex grid (1.6M DOFs, 5 levels) solved as one
    batched mixed-precision MGCG with the autotuner's smoother setting: every load case meets 1e-8
    in the true residual."""
    torch = torch_cuda()
    topo = topo_lib()
    from paper_1606_06201_gb300.autotune import autotune, solver_for
    nx, ny, nz, levels = 128, 64, 64, 5
    cfg = W.random_field_3d(nx, ny, nz, n_rhs=8)
    x = dev(torch, cfg["x"])
    F = dev(torch, cfg["f"])
    best = autotune(nx, ny, nz, cfg["fixed"], x, F, levels, precision=topo.MIXED, nrhs=8,
                    tol=1e-8, sweeps=(1, 2), cheb_degrees=(1, 2), reps=1,
                    cache_path=str(tmp_path / "tune.json"))
    s = solver_for(best, nx, ny, nz, cfg["fixed"], levels, precision=topo.MIXED, nrhs=8)
    s.set_density(x)
    U, info = s.solve(F, tol=1e-8)
    assert info.status == topo.OK
    grid = fe.Grid(nx, ny, nz)
    K0 = fe.element_stiffness(3)
    Uh = host(U)
    for r in range(8):
        res = _true_residual(grid, K0, cfg["x"], cfg["fixed"].astype(bool), cfg["f"][r], Uh[r])
        assert res <= 2e-8, (r, res, info.iterations)
    s.close()


@pytest.mark.parametrize("shape,levels", [((64, 32, 32), 4), ((1024, 512, 0), 8)])
def test_differentiation_workloads_full_size(shape, levels):
    """Compliance and a linear functional on the differentiation workloads (3D 64 x 32 x 32, 2D
    1024 x 512), mixed precision: forward and adjoint residuals, the gradient formulas against the
    oracle on the GPU's u and lam, and central differences (h = 1e-6) on 32 seeded elements of high
    sensitivity."""
    torch = torch_cuda()
    topo = topo_lib()
    from paper_1606_06201_gb300 import autograd as AG
    nx, ny, nz = shape
    cfg = W.random_density_problem(nx, ny, nz, seed_x=4)
    s = topo.Solver(nx, ny, nz, fixed=cfg["fixed"], levels=levels, precision=topo.MIXED)
    grid = fe.Grid(nx, ny, nz)
    K0 = fe.element_stiffness(grid.dim)
    fixed = cfg["fixed"].astype(bool)
    w = W.random_vector(s.n, 5, cfg["fixed"])
    f = dev(torch, cfg["f"])
    wt = dev(torch, w)
    # compliance: dc/dx_e = -u_e^T K0 u_e
    xt = dev(torch, cfg["x"]).requires_grad_(True)
    c = AG.compliance(xt, f, s, tol=1e-10)
    c.backward()
    u, _ = s.solve(f, tol=1e-10)
    uh = host(u)
    assert _true_residual(grid, K0, cfg["x"], fixed, cfg["f"], uh) <= 2e-10
    g_ref = -fe.element_energy(grid, K0, uh)
    assert np.all(np.abs(host(xt.grad) - g_ref) <= _energy_bound(grid, K0, uh, uh))
    # linear functional w^T u: adjoint K lam = w, dL/dx_e = -lam_e^T K0 u_e
    xt2 = dev(torch, cfg["x"]).requires_grad_(True)
    uu = AG.displacement(xt2, f, s, tol=1e-10)
    (wt * uu).sum().backward()
    s.set_density(dev(torch, cfg["x"]))
    lam, _ = s.solve(wt, tol=1e-10)
    lh = host(lam)
    assert _true_residual(grid, K0, cfg["x"], fixed, w, lh) <= 2e-10
    ue = fe.element_values(grid, uh)
    le = fe.element_values(grid, lh)
    g2_ref = -np.einsum("ei,ij,ej->e", le, K0, ue)
    assert np.all(np.abs(host(xt2.grad) - g2_ref) <= _energy_bound(grid, K0, lh, uh))
    # Central differences.  At these sizes one element moves the compliance by |g_e| h, about
    # 1e-6..1e-4 of c for h = 1e-6 on a typical element, below what any FP64 evaluation of c
    # resolves; so the 32 seeded elements are drawn from the 1% with the largest sensitivity, and
    # the differences are taken of the energy functional Pi(u) = 2 f^T u - u^T K(x) u, which equals
    # c at the solution and errs only quadratically in the solve error, from FP64 solves to 1e-13.
    # The gradient they are compared with comes from a mixed forward solve to 1e-12.
    xt3 = dev(torch, cfg["x"]).requires_grad_(True)
    AG.compliance(xt3, f, s, tol=1e-12).backward()
    g = host(xt3.grad)
    top = np.argsort(np.abs(g))[-max(32, s.m // 100):]
    idx = np.random.default_rng(6).choice(top, 32, replace=False)
    sfd = topo.Solver(nx, ny, nz, fixed=cfg["fixed"], levels=levels, precision=topo.FP64)
    h = 1e-6
    fd = np.empty(idx.size)
    for q, e in enumerate(idx):
        vals = []
        for sign in (1.0, -1.0):
            xp = cfg["x"].copy()
            xp[e] += sign * h
            sfd.set_density(dev(torch, xp))
            up, _ = sfd.solve(f, tol=1e-13)
            vals.append(2.0 * float(f @ up) - float(up @ sfd.apply_K(up)))
        fd[q] = (vals[0] - vals[1]) / (2 * h)
    assert np.linalg.norm(g[idx] - fd) <= 1e-5 * np.linalg.norm(fd)
    sfd.close()
    s.close()


def test_3d_scale_run_256x128x128_forward_backward():
    """The 12.8M-DOF scale run (256 x 128 x 128, 6 levels, mixed): forward solve and the compliance
    gradient; the true residual meets the tolerance and the gradient equals -u_e^T K0 u_e on every
    element, both by the oracle on the GPU's u."""
    torch = torch_cuda()
    topo = topo_lib()
    from paper_1606_06201_gb300 import autograd as AG
    nx, ny, nz, levels = 256, 128, 128, 6
    cfg = W.random_density_problem(nx, ny, nz, seed_x=4)
    s = topo.Solver(nx, ny, nz, fixed=cfg["fixed"], levels=levels, precision=topo.MIXED)
    f = dev(torch, cfg["f"])
    xt = dev(torch, cfg["x"]).requires_grad_(True)
    c = AG.compliance(xt, f, s, tol=1e-8)
    c.backward()
    u, info = s.solve(f, tol=1e-8)
    uh = host(u)
    grid = fe.Grid(nx, ny, nz)
    K0 = fe.element_stiffness(3)
    assert _true_residual(grid, K0, cfg["x"], cfg["fixed"].astype(bool), cfg["f"], uh) <= 2e-8
    g_ref = -fe.element_energy(grid, K0, uh)
    assert np.all(np.abs(host(xt.grad) - g_ref) <= _energy_bound(grid, K0, uh, uh))
    cv = float(c.detach())
    assert abs(cv - float(cfg["f"] @ uh)) <= 1e-12 * abs(cv)
    s.close()
