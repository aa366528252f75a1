"""Pins for three oracle functions whose earlier checks could not tell a plausible mistake from
the right formula: the damped OC update (Algorithm DOC, Sec. 4.2), the Newton stopping rule of
Sec. 3.4 and the scaled KKT residual of the Remark in Sec. 3.4.

Each pin computes its expected value by a route that does not go through the function under
test: closed forms of the bisection's root, an algebraic simplification of tilde Res3, element
energies from the assembled operator, and points built so that single KKT rows vanish.  Each pin
is also run against mistakes planted in copies of the oracle's functions (on the CPU): every
planted mistake must make the pin fail, which shows that the pin can see it.
"""
import math

import numpy as np
import pytest

from oracle import fe, ip, oc
from paper_1606_06201_gb300 import workloads as W


# --------------------------------------------------------------------------------------------
# Algorithm DOC (Sec. 4.2): x_i^NEW = min(x_i (u^T K_i u)^q / lambda, xbar), lambda from the
# same bisection as Algorithm OC.
# --------------------------------------------------------------------------------------------

def _check_doc_step(bisect):
    """Closed form of one damped step when no bound binds: sum x^NEW = V fixes
    lambda = sum x_i E_i^q / V and x^NEW = V x E^q / sum x E^q."""
    rng = np.random.default_rng(11)
    m = 64
    x = rng.uniform(0.3, 0.5, m)
    E = rng.uniform(20.0, 40.0, m)          # lambda near 2.5 for q = 1/2, far from 1
    V = 0.4 * m
    for q in (0.5, 1.0 / 3.0):
        xq = x * E ** q
        lam_exact = math.fsum(xq) / V
        x_exact = xq / lam_exact
        assert np.all((x_exact > 1e-6) & (x_exact < 1.0))   # no bound binds
        x_new, lam, _ = bisect(x, E, V, 1.0, 1e-6, q=q)
        assert abs(lam - lam_exact) <= 1e-10, (q, lam, lam_exact)
        np.testing.assert_allclose(x_new, x_exact, rtol=1e-10, atol=0)


def _doc_problem():
    cfg = W.cantilever_2d(8, 4, 0.5)
    return ip.Problem(fe.Grid(8, 4), fe.element_stiffness(2), cfg["fixed"], cfg["f"], cfg["V"], 1.0)


def _check_doc_fixed_point(run):
    """At the converged DOC iterate the update leaves every element strictly inside the bounds
    unchanged, so E_i^q = lambda there (q = 1/2), with lambda the bisection's own value; and by
    convexity of the VTS problem (Sec. 2) the compliance equals the IP optimum's."""
    prob = _doc_problem()
    x, info = run(prob)
    x1, u, c, lam = oc.oc_step(prob, x, xlow=1e-10, q=0.5)
    E = fe.element_energy(prob.grid, prob.K0, u)
    inside = (x > 1e-3) & (x < 1.0 - 1e-3)
    assert inside.sum() >= 10
    np.testing.assert_allclose(np.sqrt(E[inside]), lam, rtol=1e-6)
    _, ipinfo = ip.ip_run(prob)
    assert abs(info["compliance"][-1] - ipinfo["compliance"]) <= 1e-6 * ipinfo["compliance"]


def _doc_run(prob):
    return oc.oc_run(prob, variant="doc", q=0.5, tau_oc=0.0, max_feval=300, xlow=1e-10)


def test_doc_step_closed_form():
    _check_doc_step(oc.bisect_lambda)


def test_doc_fixed_point_and_ip_optimum():
    _check_doc_fixed_point(_doc_run)


# planted mistakes in the damped update, each built from the oracle's own bisection
_bisect = oc.bisect_lambda


def _doc_exponent_outside(x, E, V, xbar, xlow, lam_hi=1e4, lam_lo=0.0, tau=1e-11, q=1.0):
    """x (E / lambda)^q: the same iterates, a different lambda (lambda^q of the right one)."""
    x_new, mu, steps = _bisect(x, E ** q, V, xbar, xlow, lam_hi, lam_lo, tau, q=1.0)
    return x_new, mu ** (1.0 / q), steps


def _doc_inverse_exponent(x, E, V, xbar, xlow, lam_hi=1e4, lam_lo=0.0, tau=1e-11, q=1.0):
    return _bisect(x, E, V, xbar, xlow, lam_hi, lam_lo, tau, q=1.0 / q)


def _doc_exponent_dropped(x, E, V, xbar, xlow, lam_hi=1e4, lam_lo=0.0, tau=1e-11, q=1.0):
    return _bisect(x, E, V, xbar, xlow, lam_hi, lam_lo, tau, q=1.0)


_DOC_MUTANTS = [_doc_exponent_outside, _doc_inverse_exponent, _doc_exponent_dropped]


@pytest.mark.parametrize("mutant", _DOC_MUTANTS)
def test_doc_step_pin_rejects_planted_mistakes(mutant):
    with pytest.raises(AssertionError):
        _check_doc_step(mutant)


@pytest.mark.parametrize("mutant", _DOC_MUTANTS)
def test_doc_fixed_point_pin_rejects_planted_mistakes(mutant, monkeypatch):
    """The mistake planted in the oracle's bisection, used by its OC step and its DOC run."""
    monkeypatch.setattr(oc, "bisect_lambda", mutant)
    with np.errstate(all="ignore"), pytest.raises(AssertionError):
        _check_doc_fixed_point(_doc_run)


# --------------------------------------------------------------------------------------------
# Newton stopping rule, Sec. 3.4:  ||Res1|| / ||f|| + ||tilde Res3|| / (||phi|| + ||psi||).
#
# Independent route for tilde Res3.  With Res3 = -1/2 u^T K_i u - lambda - phi + psi,
# Res4 = s - phi x and Res5 = r - psi (xbar - x), the reduced residual
#   tilde Res3 = Res3 - X^{-1} Res4 + (Xbar - X)^{-1} Res5
# simplifies to -1/2 u^T K_i u - lambda - s / x_i + r / (xbar - x_i): phi and psi cancel.
# --------------------------------------------------------------------------------------------

def _two_element_problem():
    cfg = W.cantilever_2d(2, 1, 0.5)
    return ip.Problem(fe.Grid(2, 1), fe.element_stiffness(2), cfg["fixed"], cfg["f"], cfg["V"], 1.0)


def _energies_by_assembly(prob, u):
    """u^T K_i u with K_i = K(e_i) assembled by the (separately pinned) assembly routine."""
    out = np.empty(prob.m)
    for i in range(prob.m):
        e = np.zeros(prob.m)
        e[i] = 1.0
        out[i] = float(u @ (fe.assemble(prob.grid, prob.K0, e) @ u))
    return out


def _check_newton_criterion(crit):
    prob = _two_element_problem()
    xbar = prob.xbar
    # (A) u = 0: Res1 = f, the energies vanish; hand-computed value
    x = np.array([0.25, 0.5])
    phi, psi = np.array([1.0, 2.0]), np.array([3.0, 4.0])
    s, r, lam = 0.1, 0.2, 0.3
    z = [np.zeros(prob.grid.n_dofs), lam, x, phi, psi]
    # tilde Res3 = (-0.3 - 0.1/0.25 + 0.2/0.75, -0.3 - 0.1/0.5 + 0.2/0.5) = (-13/30, -1/10)
    expect = 1.0 + math.sqrt(178.0) / 30.0 / (math.sqrt(5.0) + 5.0)
    got = crit(prob, z, s, r)
    assert abs(got - expect) <= 1e-14 * expect, (got, expect)
    # (B) a non-optimal u with non-zero energies, s != phi x and r != psi (xbar - x)
    rng = np.random.default_rng(5)
    u = np.zeros(prob.grid.n_dofs)
    u[prob.free] = rng.standard_normal(prob.free.size)
    x = np.array([0.35, 0.7])
    phi, psi = np.array([0.9, 0.2]), np.array([0.4, 1.3])
    s, r, lam = 0.05, 0.02, -0.6
    K = fe.assemble(prob.grid, prob.K0, x)
    res1 = (prob.f - K @ u)[prob.free]
    E = _energies_by_assembly(prob, u)
    rt3 = -0.5 * E - lam - s / x + r / (xbar - x)
    expect = (np.linalg.norm(res1) / np.linalg.norm(prob.f[prob.free])
              + np.linalg.norm(rt3) / (np.linalg.norm(phi) + np.linalg.norm(psi)))
    got = crit(prob, [u, lam, x, phi, psi], s, r)
    assert abs(got - expect) <= 1e-12 * expect, (got, expect)


def test_newton_criterion_hand_values():
    _check_newton_criterion(ip.newton_criterion)


def _terms(prob, z, s, r):
    u, lam, x, phi, psi = z
    return ip.kkt_residuals(prob, prob.K0, u, lam, x, phi, psi, s, r)


def _newton_res3_not_reduced(prob, z, s, r):
    res1, _, f3, _, _, _, _, _ = _terms(prob, z, s, r)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f)
            + np.linalg.norm(f3) / (np.linalg.norm(z[3]) + np.linalg.norm(z[4])))


def _newton_max_norm(prob, z, s, r):
    res1, _, _, _, _, rt3, _, _ = _terms(prob, z, s, r)
    return (np.max(np.abs(res1)) / np.max(np.abs(prob.f))
            + np.max(np.abs(rt3)) / (np.max(np.abs(z[3])) + np.max(np.abs(z[4]))))


def _newton_norm_of_sum(prob, z, s, r):
    res1, _, _, _, _, rt3, _, _ = _terms(prob, z, s, r)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f)
            + np.linalg.norm(rt3) / np.linalg.norm(z[3] + z[4]))


def _newton_res1_dropped(prob, z, s, r):
    _, _, _, _, _, rt3, _, _ = _terms(prob, z, s, r)
    return np.linalg.norm(rt3) / (np.linalg.norm(z[3]) + np.linalg.norm(z[4]))


def _newton_sign_slip(prob, z, s, r):
    """tilde Res3 with + X^{-1} Res4 (a sign slip in the elimination of d_phi)."""
    u, lam, x, phi, psi = z
    res1, _, f3, res4, res5, _, _, _ = _terms(prob, z, s, r)
    rt3 = f3 + res4 / x + res5 / (prob.xbar - x)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f)
            + np.linalg.norm(rt3) / (np.linalg.norm(phi) + np.linalg.norm(psi)))


@pytest.mark.parametrize("mutant", [_newton_res3_not_reduced, _newton_max_norm,
                                    _newton_norm_of_sum, _newton_res1_dropped, _newton_sign_slip])
def test_newton_criterion_pin_rejects_planted_mistakes(mutant):
    with pytest.raises(AssertionError):
        _check_newton_criterion(mutant)


# --------------------------------------------------------------------------------------------
# Scaled KKT residual of the Remark in Sec. 3.4 (reading: each complementarity term scaled by
# its own factors):
#   ||Res1||/||f|| + ||tilde Res3||/(||phi||+||psi||) + phi^T x/(||phi|| ||x||)
#   + psi^T (xbar - x)/(||psi|| ||xbar - x||).
# A point is built where KKT1 holds (u = K(x)^{-1} f) and tilde Res3 = 0 (lambda and r solved
# from the two element equations); then each KKT row is perturbed alone.
# --------------------------------------------------------------------------------------------

def _kkt_point():
    prob = _two_element_problem()
    x = np.array([0.3, 0.4])                 # ||x|| = 1/2, xbar - x = (0.7, 0.6)
    u = prob.solve_u(x)
    E = _energies_by_assembly(prob, u)
    s = 0.1
    # -1/2 E_i - lambda - s/x_i + r/(xbar - x_i) = 0 for i = 1, 2: linear in (lambda, r)
    A = np.array([[-1.0, 1.0 / (1.0 - x[0])], [-1.0, 1.0 / (1.0 - x[1])]])
    lam, r = np.linalg.solve(A, 0.5 * E + s / x)
    phi = np.array([0.8, 0.6])               # phi^T x / (||phi|| ||x||) = 0.48 / 0.5 = 0.96
    psi = np.array([0.6, 0.8])               # psi^T (xbar - x) = 0.9, ||psi|| = 1
    return prob, [u, float(lam), x, phi, psi], s, float(r)


def _check_kkt_criterion(crit):
    prob, z, s, r = _kkt_point()
    u, lam, x, phi, psi = z
    xu = prob.xbar - x
    base3, base4 = 0.96, 0.9 / math.sqrt(0.85)
    den = np.linalg.norm(phi) + np.linalg.norm(psi)      # = 2
    # P0: KKT1 and the reduced row 3 hold; only the two complementarity terms remain
    got = crit(prob, z, s, r)
    assert abs(got - (base3 + base4)) <= 1e-12, got
    # P1: lambda moved (row KKT3 only): tilde Res3 = -delta e
    d = 1e-3
    got = crit(prob, [u, lam + d, x, phi, psi], s, r)
    assert abs(got - (base3 + base4 + math.sqrt(2.0) * d / den)) <= 1e-12, got
    # P2: the load moved on one free DOF (row KKT1 only): Res1 = delta e_j
    f2 = prob.f.copy()
    j = prob.free[0]
    f2[j] += d
    prob2 = ip.Problem(prob.grid, prob.K0, prob.fixed, f2, prob.V, prob.xbar)
    got = crit(prob2, z, s, r)
    assert abs(got - (base3 + base4 + d / np.linalg.norm(f2))) <= 1e-12, got
    # P3: s moved (the perturbed complementarity of phi): tilde Res3 = -delta / x
    got = crit(prob, z, s + d, r)
    assert abs(got - (base3 + base4 + d * np.linalg.norm(1.0 / x) / den)) <= 1e-12, got
    # P4: r moved: tilde Res3 = +delta / (xbar - x)
    got = crit(prob, z, s, r + d)
    assert abs(got - (base3 + base4 + d * np.linalg.norm(1.0 / xu) / den)) <= 1e-12, got
    # P5: phi turned parallel to x (its complementarity term only; scale does not matter)
    got = crit(prob, [u, lam, x, 3.0 * np.array([0.6, 0.8]), psi], s, r)
    assert abs(got - (1.0 + base4)) <= 1e-12, got
    # P6: psi turned parallel to xbar - x
    got = crit(prob, [u, lam, x, phi, 2.0 * xu], s, r)
    assert abs(got - (base3 + 1.0)) <= 1e-12, got


def test_kkt_criterion_terms_one_row_at_a_time():
    _check_kkt_criterion(ip.kkt_criterion)


def _kkt_printed_denominator(prob, z, s, r):
    """The last term with the printed ||phi|| ||x|| denominator."""
    u, lam, x, phi, psi = z
    res1, _, _, _, _, rt3, _, _ = _terms(prob, z, s, r)
    nphi, npsi = np.linalg.norm(phi), np.linalg.norm(psi)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f) + np.linalg.norm(rt3) / (nphi + npsi)
            + float(phi @ x) / (nphi * np.linalg.norm(x))
            + float(psi @ (prob.xbar - x)) / (nphi * np.linalg.norm(x)))


def _kkt_term_dropped(prob, z, s, r):
    u, lam, x, phi, psi = z
    res1, _, _, _, _, rt3, _, _ = _terms(prob, z, s, r)
    nphi, npsi = np.linalg.norm(phi), np.linalg.norm(psi)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f) + np.linalg.norm(rt3) / (nphi + npsi)
            + float(psi @ (prob.xbar - x)) / (npsi * np.linalg.norm(prob.xbar - x)))


def _kkt_res3_not_reduced(prob, z, s, r):
    u, lam, x, phi, psi = z
    res1, _, f3, _, _, _, _, _ = _terms(prob, z, s, r)
    nphi, npsi = np.linalg.norm(phi), np.linalg.norm(psi)
    xu = prob.xbar - x
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f) + np.linalg.norm(f3) / (nphi + npsi)
            + float(phi @ x) / (nphi * np.linalg.norm(x))
            + float(psi @ xu) / (npsi * np.linalg.norm(xu)))


def _kkt_unscaled_products(prob, z, s, r):
    u, lam, x, phi, psi = z
    res1, _, _, _, _, rt3, _, _ = _terms(prob, z, s, r)
    nphi, npsi = np.linalg.norm(phi), np.linalg.norm(psi)
    return (np.linalg.norm(res1) / np.linalg.norm(prob.f) + np.linalg.norm(rt3) / (nphi + npsi)
            + float(phi @ x) + float(psi @ (prob.xbar - x)))


@pytest.mark.parametrize("mutant", [_kkt_printed_denominator, _kkt_term_dropped,
                                    _kkt_res3_not_reduced, _kkt_unscaled_products])
def test_kkt_criterion_pin_rejects_planted_mistakes(mutant):
    with pytest.raises(AssertionError):
        _check_kkt_criterion(mutant)
