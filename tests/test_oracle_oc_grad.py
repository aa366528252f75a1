"""Pins for the oracle's OC methods (Sec. 4) and the adjoint gradient: the bisection hits the
volume, the OC fixed-point property E_i = lambda on inactive elements, mirror symmetry, and the
gradient against central finite differences."""
import math

import numpy as np
import pytest

from oracle import fe, grad, ip, oc
from paper_1606_06201_gb300 import workloads as W


def _problem(nx, ny, volfrac=0.5):
    cfg = W.cantilever_2d(nx, ny, volfrac)
    return ip.Problem(fe.Grid(nx, ny), fe.element_stiffness(2), cfg["fixed"], cfg["f"], cfg["V"], 1.0)


def test_bisection_meets_volume():
    rng = np.random.default_rng(0)
    x = rng.uniform(0.1, 0.9, 200)
    E = rng.uniform(0.01, 3.0, 200)
    V = 0.4 * 200
    x_new, lam, steps = oc.bisect_lambda(x, E, V, 1.0, 1e-6)
    # 1e4 / 2^k <= 1e-11 first at k = 50
    assert steps == math.ceil(math.log2(1e4 / 1e-11))
    assert abs(math.fsum(x_new) - V) <= 1e-6 * V
    assert np.all(x_new >= 1e-6) and np.all(x_new <= 1.0)
    # brute force: sum x_new(lambda) is non-increasing in lambda and crosses V at the returned lambda
    s_lo = math.fsum(np.minimum(np.maximum(x * E / (lam * (1 - 1e-9)), 1e-6), 1.0))
    s_hi = math.fsum(np.minimum(np.maximum(x * E / (lam * (1 + 1e-9)), 1e-6), 1.0))
    assert s_hi <= V + 1e-6 and s_lo >= V - 1e-6


def test_oc_fixed_point_and_symmetry():
    prob = _problem(16, 8)
    x, info = oc.oc_run(prob, variant="aoc", tau_oc=0.0, max_feval=2000, xlow=1e-9)
    x1, u, c, lam = oc.oc_step(prob, x, xlow=1e-9)
    E = fe.element_energy(prob.grid, prob.K0, u)
    inside = (x > 1e-3) & (x < 1.0 - 1e-3)
    assert inside.sum() > 10
    np.testing.assert_allclose(E[inside], lam, rtol=1e-3)
    X = x.reshape(8, 16)
    np.testing.assert_allclose(X, X[::-1], rtol=0, atol=1e-8)
    # plain OC zig-zags; AOC and DOC both decrease the compliance from the uniform start
    for variant in ("aoc", "doc"):
        _, inf2 = oc.oc_run(prob, variant=variant, tau_oc=0.0, max_feval=20)
        assert inf2["compliance"][-1] < inf2["compliance"][0]


@pytest.mark.parametrize("which", ["compliance", "random"])
def test_gradient_matches_central_differences(which):
    cfg = W.random_density_problem(12, 6, seed_x=4)
    grid = fe.Grid(12, 6)
    prob = ip.Problem(grid, fe.element_stiffness(2), cfg["fixed"], cfg["f"], 1.0, 1.0)
    x = cfg["x"]
    w = prob.f if which == "compliance" else W.random_vector(grid.n_dofs, 7, cfg["fixed"])
    g, u, lam = grad.grad_linear_functional(prob, x, w)
    if which == "compliance":
        np.testing.assert_allclose(lam, u, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(g, -fe.element_energy(grid, prob.K0, u), rtol=1e-12)
    idx = np.random.default_rng(5).choice(prob.m, 32, replace=False)
    h = 1e-6
    fd = np.empty(idx.size)
    for k, e in enumerate(idx):
        xp, xm = x.copy(), x.copy()
        xp[e] += h
        xm[e] -= h
        fd[k] = (w @ prob.solve_u(xp) - w @ prob.solve_u(xm)) / (2 * h)
    assert np.linalg.norm(g[idx] - fd) <= 1e-5 * np.linalg.norm(fd)


def test_inexact_oc_adaptive_tolerance_rule():
    """Sec. 6.2 in the oracle: with MGCG solves the tolerance of iteration k is tau_0 * 0.1^j, j
    the number of earlier iterations whose compliance rose; with a tight tau_0 the inexact run
    reproduces the exact-solve run."""
    prob = _problem(32, 16)
    sol = oc.MGCGSolve(prob, levels=3, tau=0.1)
    _, info = oc.oc_run(prob, variant="oc", tau_oc=0.0, max_feval=30, solve=sol,
                        adaptive_tol=True)
    c, taus = info["compliance"], info["tau"]
    rises = 0
    for k in range(len(c)):
        assert taus[k] == pytest.approx(0.1 * 0.1 ** rises, rel=1e-15), k
        if k >= 1 and c[k] > c[k - 1]:
            rises += 1
    assert rises >= 1
    tight = oc.MGCGSolve(prob, levels=3, tau=1e-12)
    _, inexact = oc.oc_run(prob, variant="aoc", tau_oc=0.0, max_feval=20, solve=tight,
                           adaptive_tol=True)
    _, exact = oc.oc_run(prob, variant="aoc", tau_oc=0.0, max_feval=20)
    np.testing.assert_allclose(inexact["compliance"], exact["compliance"], rtol=1e-9)
    np.testing.assert_allclose(inexact["x"], exact["x"], rtol=0, atol=1e-8)
