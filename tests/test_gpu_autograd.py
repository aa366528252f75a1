"""Differentiable solves: torch.autograd gradients from the adjoint MGCG against the oracle's
adjoint gradient and against central finite differences (h = 1e-6) on 32 seeded elements, for the
compliance and for a random linear functional of u, in 2D and 3D, FP64 and mixed precision."""
import numpy as np
import pytest

from oracle import fe, grad as ograd, ip as oip
from paper_1606_06201_gb300 import workloads as W

from gpu_helpers import dev, host, topo_lib, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [((64, 32, 0), 3), ((8, 4, 4), 2)]


def _setup(shape, levels, precision):
    torch = torch_cuda()
    topo = topo_lib()
    from paper_1606_06201_gb300 import autograd as AG
    nx, ny, nz = shape
    cfg = W.random_density_problem(nx, ny, nz, seed_x=4)
    s = topo.Solver(nx, ny, nz, fixed=cfg["fixed"], levels=levels, precision=precision)
    grid = fe.Grid(nx, ny, nz)
    prob = oip.Problem(grid, fe.element_stiffness(grid.dim), cfg["fixed"], cfg["f"], 1.0, 1.0)
    return torch, topo, AG, cfg, s, prob


@pytest.mark.parametrize("shape,levels", CASES)
@pytest.mark.parametrize("which", ["compliance", "linear"])
def test_gradient_matches_oracle_and_fd(shape, levels, which):
    torch, topo, AG, cfg, s, prob = _setup(shape, levels, 0)
    x = dev(torch, cfg["x"]).requires_grad_(True)
    f = dev(torch, cfg["f"])
    w = W.random_vector(s.n, 7, cfg["fixed"])
    wt = dev(torch, w)
    if which == "compliance":
        L = AG.compliance(x, f, s, tol=1e-13)
        g_ref, _, _ = ograd.grad_linear_functional(prob, cfg["x"], prob.f)
    else:
        u = AG.displacement(x, f, s, tol=1e-13)
        L = (wt * u).sum()
        g_ref, _, _ = ograd.grad_linear_functional(prob, cfg["x"], w)
    L.backward()
    g = host(x.grad)
    assert np.linalg.norm(g - g_ref) <= 1e-9 * np.linalg.norm(g_ref)
    # central differences through the GPU forward solve
    idx = np.random.default_rng(5).choice(s.m, 32, replace=False)
    h = 1e-6
    fd = np.empty(idx.size)
    for k, e in enumerate(idx):
        vals = []
        for sign in (1.0, -1.0):
            xp = cfg["x"].copy()
            xp[e] += sign * h
            s.set_density(dev(torch, xp))
            up, _ = s.solve(f, tol=1e-13)
            vals.append(float((wt if which == "linear" else f) @ up))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    assert np.linalg.norm(g[idx] - fd) <= 1e-5 * np.linalg.norm(fd)


@pytest.mark.parametrize("shape,levels", CASES)
def test_gradient_mixed_precision(shape, levels):
    torch, topo, AG, cfg, s, prob = _setup(shape, levels, 1)
    x = dev(torch, cfg["x"]).requires_grad_(True)
    f = dev(torch, cfg["f"])
    w = W.random_vector(s.n, 8, cfg["fixed"])
    u = AG.displacement(x, f, s, tol=1e-10)
    (dev(torch, w) * u).sum().backward()
    g_ref, _, _ = ograd.grad_linear_functional(prob, cfg["x"], w)
    assert np.linalg.norm(host(x.grad) - g_ref) <= 1e-6 * np.linalg.norm(g_ref)
