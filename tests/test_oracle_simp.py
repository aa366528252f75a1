"""Pins for the oracle's SIMP model with the density filter (Sec. 9): the filter matrix against a
brute-force double loop over element pairs and its closed-form interior and corner columns, the
reduction to the convex VTS method at p = 1 and r_min = 1 (W = I), the Newton direction against a
finite-difference Jacobian of the SIMP KKT map with the dropped second-derivative block, the
modified KKT row 3 as the gradient of the strain energy, mirror symmetry and feasibility of a
full IP run on an Example-4-shaped beam."""
import numpy as np
import pytest

from oracle import fe, ip, simp
from paper_1606_06201_gb300 import workloads as W


def _problem(nx, ny, volfrac=0.4, xbar=3.0, p=3.0, rmin=2.0, nz=0):
    if nz:
        fixed = W.clamp_xmin(nx, ny, nz)
        f = W.point_load(nx, ny, nz, (nx, ny // 2, nz // 2), 1)
        return simp.SimpProblem(fe.Grid(nx, ny, nz), fe.element_stiffness(3), fixed, f,
                                volfrac * nx * ny * nz, xbar, p=p, rmin=rmin)
    cfg = W.cantilever_2d(nx, ny, volfrac)
    return simp.SimpProblem(fe.Grid(nx, ny), fe.element_stiffness(2), cfg["fixed"], cfg["f"],
                            cfg["V"], xbar, p=p, rmin=rmin)


def _brute_force_filter(grid, rmin):
    """hat W_ij = max(0, rmin - Manhattan distance of the centres), columns divided by their sums,
    by a plain double loop over all element pairs."""
    nz = max(grid.nz, 1)
    cen = [(ex, ey, ez) for ez in range(nz) for ey in range(grid.ny) for ex in range(grid.nx)]
    m = len(cen)
    Wh = np.zeros((m, m))
    for i in range(m):
        for j in range(m):
            dist = sum(abs(a - b) for a, b in zip(cen[i], cen[j]))
            Wh[i, j] = max(0.0, rmin - dist)
    return Wh / Wh.sum(axis=0)[None, :]


@pytest.mark.parametrize("shape,rmin", [((5, 4, 0), 2.0), ((6, 3, 0), 2.5), ((4, 3, 0), 3.0),
                                        ((3, 3, 2), 2.0), ((4, 2, 3), 2.7)])
def test_filter_matches_brute_force(shape, rmin):
    grid = fe.Grid(*shape)
    Wo = simp.filter_matrix(grid, rmin).toarray()
    np.testing.assert_allclose(Wo, _brute_force_filter(grid, rmin), rtol=0, atol=1e-15)
    np.testing.assert_allclose(Wo.sum(axis=0), 1.0, rtol=0, atol=1e-14)


def test_filter_closed_form_columns():
    """r_min = 2: an interior column holds 2/6 on its element and 1/6 on the four edge
    neighbours; a corner column 2/4 and 1/4 on its two neighbours; r_min = 1 gives W = I."""
    grid = fe.Grid(5, 4)
    Wd = simp.filter_matrix(grid, 2.0).toarray()
    i = 2 + 5 * 2
    col = Wd[:, i]
    assert col[i] == pytest.approx(2 / 6, abs=1e-15)
    for j in (i - 1, i + 1, i - 5, i + 5):
        assert col[j] == pytest.approx(1 / 6, abs=1e-15)
    assert np.count_nonzero(col) == 5
    c0 = Wd[:, 0]
    assert c0[0] == pytest.approx(0.5) and c0[1] == pytest.approx(0.25) and c0[5] == pytest.approx(0.25)
    assert np.count_nonzero(c0) == 3
    np.testing.assert_array_equal(simp.filter_matrix(grid, 1.0).toarray(), np.eye(grid.n_elems))


def _interior_state(prob, seed):
    rng = np.random.default_rng(seed)
    m = prob.m
    u = np.zeros(prob.grid.n_dofs)
    u[prob.free] = rng.standard_normal(prob.free.size)
    return [u, 0.7, rng.uniform(0.2, 0.8, m) * prob.xbar, rng.uniform(0.5, 2.0, m),
            rng.uniform(0.5, 2.0, m)]


def test_p1_rmin1_reduces_to_the_convex_method():
    """With p = 1 and W = I the SIMP problem is the VTS problem of Eq. (to): the same direction
    and the same IP trajectory."""
    cfg = W.cantilever_2d(8, 4, 0.5)
    grid, K0 = fe.Grid(8, 4), fe.element_stiffness(2)
    pv = ip.Problem(grid, K0, cfg["fixed"], cfg["f"], cfg["V"], 1.0)
    ps = simp.SimpProblem(grid, K0, cfg["fixed"], cfg["f"], cfg["V"], 1.0, p=1.0, rmin=1.0)
    z = _interior_state(pv, 3)
    dv, _ = ip.newton_direction(pv, z, 0.1, 0.2)
    ds, _ = simp.newton_direction(ps, z, 0.1, 0.2)
    for a, b in zip(dv, ds):
        np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-11 * (1 + np.max(np.abs(a))))
    zv, iv = ip.ip_run(pv, max_newton=12)
    zs, is_ = simp.ip_run(ps, max_newton=12)
    assert iv["ip"] == is_["ip"] and iv["newton"] == is_["newton"]
    np.testing.assert_allclose(zs[2], zv[2], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(zs[0], zv[0], rtol=1e-8, atol=1e-12 * np.abs(zv[0]).max())


def _pack(prob, z):
    u, lam, x, phi, psi = z
    return np.concatenate([u[prob.free], [lam], x, phi, psi])


def _unpack(prob, v):
    nf, m = prob.free.size, prob.m
    u = np.zeros(prob.grid.n_dofs)
    u[prob.free] = v[:nf]
    return [u, v[nf], v[nf + 1:nf + 1 + m], v[nf + 1 + m:nf + 1 + 2 * m], v[nf + 1 + 2 * m:]]


@pytest.mark.parametrize("shape,rmin", [((4, 2), 2.0), ((4, 4), 2.5), ((2, 2, 2), 2.0)])
def test_direction_solves_fd_jacobian_without_the_xx_block(shape, rmin):
    """The direction solves J d = -F for the finite-difference Jacobian J of the SIMP KKT map once
    its (row 3, x) block, the second derivative that the method leaves out, is set to zero.  Every
    other block (hat K, hat B in rows 1 and 3, the filter) comes from the map itself."""
    prob = _problem(*shape[:2], rmin=rmin, nz=shape[2] if len(shape) == 3 else 0)
    s, r = 0.3, 0.2
    z = _interior_state(prob, 0)
    d, _ = simp.newton_direction(prob, z, s, r)
    v0 = _pack(prob, z)
    N = v0.size
    J = np.zeros((N, N))
    h = 1e-6
    for k in range(N):
        e = np.zeros(N)
        e[k] = h
        J[:, k] = (simp.kkt_map(prob, _unpack(prob, v0 + e), s, r)
                   - simp.kkt_map(prob, _unpack(prob, v0 - e), s, r)) / (2 * h)
    nf, m = prob.free.size, prob.m
    r3 = slice(nf + 1, nf + 1 + m)
    assert np.abs(J[r3, r3]).max() > 1e-3  # the left-out block is not zero for p = 3
    J[r3, r3] = 0.0
    F = simp.kkt_map(prob, z, s, r)
    dv = _pack(prob, d)
    assert np.linalg.norm(J @ dv + F) <= 1e-7 * (np.linalg.norm(F) + np.linalg.norm(J) * np.linalg.norm(dv))


def test_row3_energy_term_is_the_gradient_of_the_strain_energy():
    """-(F3 + lambda + phi - psi) = d/dx [1/2 u^T hat K(W x) u] at fixed u (central differences)."""
    prob = _problem(5, 4, rmin=2.5)
    z = _interior_state(prob, 5)
    u, lam, x, phi, psi = z
    F3 = simp.kkt_map(prob, z, 0.1, 0.1)[prob.free.size + 1:prob.free.size + 1 + prob.m]
    grad = -(F3 + lam + phi - psi)

    def energy(xx):
        _, rho, _ = prob.filtered(xx)
        return 0.5 * u @ (fe.assemble(prob.grid, prob.K0, rho) @ u)

    h = 1e-6
    fd = np.array([(energy(x + h * np.eye(prob.m)[i]) - energy(x - h * np.eye(prob.m)[i])) / (2 * h)
                   for i in range(prob.m)])
    np.testing.assert_allclose(grad, fd, rtol=1e-7, atol=1e-9 * np.abs(fd).max())


def test_example4_shaped_run_is_feasible_and_mirror_symmetric():
    """Sec. 9.1 shape (Example 2 beam, xbar = 3, r_min = 2, p = 3) on 16 x 8: the run ends with
    max(s, r) <= tau_IP after 12 barrier reductions, sum x = V, 0 < x < xbar, and the design is
    symmetric about the beam's mid-line (the load, supports and filter are)."""
    prob = _problem(16, 8)
    z, info = simp.ip_run(prob, max_newton=400)
    x = z[2]
    assert info["ip"] == 12 and max(info["s"], info["r"]) <= 1e-8
    assert abs(x.sum() - prob.V) <= 1e-8 * prob.V
    assert x.min() > 0 and x.max() < prob.xbar
    xm = x.reshape(8, 16)
    np.testing.assert_allclose(xm, xm[::-1], rtol=0, atol=1e-6 * prob.xbar)
    assert np.isfinite(info["compliance"]) and info["compliance"] > 0
