"""Pins for the oracle's interior-point method (Sec. 2-3): the Newton direction against a
finite-difference Jacobian of the KKT map and against a dense solve of the full system Eq. (nwt),
the barrier schedule (12 IP iterations at tau_IP = 1e-8, tab:IP), feasibility invariants, the
brute-force optimum of a two-element problem, mirror symmetry, and agreement with long-run OC
(convexity of the VTS problem)."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import fe, ip, oc
from paper_1606_06201_gb300 import workloads as W


def _problem(nx, ny, volfrac=0.5, xbar=1.0):
    cfg = W.cantilever_2d(nx, ny, volfrac)
    grid = fe.Grid(nx, ny)
    return ip.Problem(grid, fe.element_stiffness(2), cfg["fixed"], cfg["f"], cfg["V"], xbar)


def _random_interior_state(prob, seed):
    rng = np.random.default_rng(seed)
    m = prob.m
    x = rng.uniform(0.2, 0.8, m) * prob.xbar
    u = np.zeros(prob.grid.n_dofs)
    u[prob.free] = rng.standard_normal(prob.free.size)
    return [u, 0.7, x, rng.uniform(0.5, 2.0, m), rng.uniform(0.5, 2.0, m)]


def _pack(prob, z):
    u, lam, x, phi, psi = z
    return np.concatenate([u[prob.free], [lam], x, phi, psi])


def _unpack(prob, v):
    nf, m = prob.free.size, prob.m
    u = np.zeros(prob.grid.n_dofs)
    u[prob.free] = v[:nf]
    return [u, v[nf], v[nf + 1:nf + 1 + m], v[nf + 1 + m:nf + 1 + 2 * m], v[nf + 1 + 2 * m:]]


@pytest.mark.parametrize("shape", [(2, 2), (4, 2)])
def test_newton_direction_solves_fd_jacobian(shape):
    prob = _problem(*shape)
    s, r = 0.3, 0.2
    z = _random_interior_state(prob, 0)
    d, _ = ip.newton_direction(prob, z, s, r)
    v0 = _pack(prob, z)
    N = v0.size
    J = np.zeros((N, N))
    h = 1e-6
    for k in range(N):
        e = np.zeros(N); e[k] = h
        J[:, k] = (ip.kkt_map(prob, _unpack(prob, v0 + e), s, r)
                   - ip.kkt_map(prob, _unpack(prob, v0 - e), s, r)) / (2 * h)
    F = ip.kkt_map(prob, z, s, r)
    dv = _pack(prob, d)
    assert np.linalg.norm(J @ dv + F) <= 1e-7 * (np.linalg.norm(F) + np.linalg.norm(J) * np.linalg.norm(dv))


@pytest.mark.parametrize("shape", [(2, 2), (4, 2)])
def test_newton_direction_matches_full_system(shape):
    """Dense solve of the printed Eq. (nwt) with right-hand side (Res1, Res2, F3, Res4, Res5)."""
    prob = _problem(*shape)
    s, r = 0.05, 0.08
    z = _random_interior_state(prob, 1)
    d, _ = ip.newton_direction(prob, z, s, r)
    J = ip.full_newton_matrix(prob, z)
    res1, res2, f3, res4, res5, _, _, _ = ip.kkt_residuals(prob, prob.K0, *z, s, r)
    rhs = np.concatenate([res1[prob.free], [res2], f3, res4, res5])
    dd = np.linalg.solve(J, rhs)
    np.testing.assert_allclose(_pack(prob, d), dd, rtol=1e-10, atol=1e-10 * np.abs(dd).max())


def test_ip_schedule_and_invariants():
    prob = _problem(16, 8)
    z, info = ip.ip_run(prob, record=True)
    # barrier s = r = 0.2^k: the k-th reduction reaches 1e-8 at k = ceil(ln 1e-8 / ln 0.2) = 12
    assert info["ip"] == 12
    assert info["s"] <= 1e-8 < info["s"] / 0.2
    for st in info["traj"]:
        assert np.all(st["x"] > 0) and np.all(st["x"] < prob.xbar)
        assert np.all(st["phi"] > 0) and np.all(st["psi"] > 0)
    # Res2 is linear: after one step with alpha the volume residual shrinks by (1 - alpha)
    assert abs(np.sum(info["traj"][0]["x"]) - prob.V) <= 1e-12 * prob.V * max(1, 1 - info["traj"][0]["alpha"]) \
        or info["traj"][0]["alpha"] < 1
    assert abs(np.sum(z[2]) - prob.V) <= 1e-11 * prob.V
    # KKT at termination: equilibrium, stationarity and complementarity all small
    res1, res2, f3, res4, res5, _, _, _ = ip.kkt_residuals(prob, prob.K0, *z, 0.0, 0.0)
    assert np.linalg.norm(res1) <= 1e-6 * np.linalg.norm(prob.f)
    assert np.abs(f3).max() <= 1e-6 * (1 + np.abs(z[1]))
    assert np.abs(res4).max() <= 1e-6 and np.abs(res5).max() <= 1e-6
    # Newton steps in the paper's range for Example-2 shapes (25-33; soft: V differs)
    assert 15 <= info["newton"] <= 45


def test_two_element_brute_force_optimum():
    """2x1 grid, x2 = V - x1: a bounded 1-D scan of f^T u(x1) gives the optimum."""
    prob = _problem(2, 1, volfrac=0.5, xbar=1.0)

    def compliance(x1):
        return float(prob.f @ prob.solve_u(np.array([x1, prob.V - x1])))

    res = minimize_scalar(compliance, bounds=(1e-9, prob.V - 1e-9), method="bounded",
                          options=dict(xatol=1e-12))
    z, info = ip.ip_run(prob)
    np.testing.assert_allclose(info["compliance"], res.fun, rtol=1e-7)
    np.testing.assert_allclose(z[2][0], res.x, atol=1e-5)
    x_oc, oinfo = oc.oc_run(prob, variant="aoc", tau_oc=0.0, max_feval=400, xlow=1e-9)
    np.testing.assert_allclose(oinfo["compliance"][-1], res.fun, rtol=1e-7)


def test_ip_solution_is_mirror_symmetric():
    prob = _problem(16, 8)
    z, _ = ip.ip_run(prob)
    X = z[2].reshape(8, 16)
    np.testing.assert_allclose(X, X[::-1], rtol=0, atol=1e-9)


def test_ip_and_long_run_oc_agree():
    """Convex VTS problem: IP and a long AOC run reach the same optimal compliance."""
    prob = _problem(8, 4)
    _, info = ip.ip_run(prob)
    _, oinfo = oc.oc_run(prob, variant="aoc", tau_oc=0.0, max_feval=3000, xlow=1e-10)
    np.testing.assert_allclose(oinfo["compliance"][-1], info["compliance"], rtol=2e-5)


def test_kkt_stop_rule_gives_almost_the_same_solution():
    """Remark in Sec. 3.4: stopping once the scaled KKT residual is small leads to almost the same
    results as the barrier rule max(s, r) <= tau_IP.  With tau_kkt = 1e-4 the run stops at the
    first Newton step whose residual meets it, and x agrees with the barrier rule's to 1e-3."""
    for shape in ((16, 8), (32, 16)):
        prob = _problem(*shape)
        zb, ib = ip.ip_run(prob)
        zk, ik = ip.ip_run(prob, stop_rule="kkt", tau_kkt=1e-4, record=True)
        kkt = [ip.kkt_criterion(prob, [t["u"], t["lam"], t["x"], t["phi"], t["psi"]], t["s"],
                                t["r"]) for t in ik["traj"]]
        assert kkt[-1] <= 1e-4 and all(k > 1e-4 for k in kkt[:-1]), shape
        assert np.max(np.abs(zb[2] - zk[2])) <= 1e-3, shape
        assert abs(ib["compliance"] - ik["compliance"]) <= 1e-6 * ib["compliance"], shape


def test_kkt_criterion_vanishes_at_a_kkt_point_and_sums_its_terms():
    """The scaled KKT residual is the sum of its four non-negative terms: zero residuals and zero
    complementarity give 0; a complementarity product alone gives exactly its scaled value."""
    prob = _problem(8, 4)
    m = prob.m
    rng = np.random.default_rng(3)
    x = rng.uniform(0.1, 0.9, m)
    u = prob.solve_u(x)
    # phi = psi = 0 would divide by zero: one entry each, on elements where the bound is apart
    phi = np.zeros(m)
    psi = np.zeros(m)
    phi[0], psi[1] = 2.0, 3.0
    z = [u, 0.0, x, phi, psi]
    # with s = phi x and r = psi (xbar - x) elementwise the barrier residuals vanish; Res3 does not
    val = ip.kkt_criterion(prob, z, 0.0, 0.0)
    comp = phi[0] * x[0] / (2.0 * np.linalg.norm(x)) + psi[1] * (1 - x[1]) / (3.0 * np.linalg.norm(1 - x))
    res1, _, _, _, _, rt3, _, _ = ip.kkt_residuals(prob, prob.K0, u, 0.0, x, phi, psi, 0.0, 0.0)
    expect = (np.linalg.norm(res1) / np.linalg.norm(prob.f) + np.linalg.norm(rt3) / 5.0 + comp)
    assert abs(val - expect) <= 1e-12 * expect


def test_example3_corner_supported_solution_is_mirror_symmetric():
    """Example 3's setting (two lower corners fixed, load at the lower edge's middle node) is
    symmetric about the vertical centre line, and so is the IP solution of the convex problem."""
    nx, ny = 16, 4
    cfg = W.corner_supported_2d(nx, ny, 0.5)
    prob = ip.Problem(fe.Grid(nx, ny), fe.element_stiffness(2), cfg["fixed"], cfg["f"], cfg["V"],
                      cfg["xbar"])
    z, info = ip.ip_run(prob)
    assert info["ip"] == 12 and max(info["s"], info["r"]) <= 1e-8
    x = z[2].reshape(ny, nx)
    assert np.max(np.abs(x - x[:, ::-1])) <= 1e-9
    assert abs(x.sum() - cfg["V"]) <= 1e-9 * cfg["V"]

