"""Interior-point and OC trajectories on the GPU against the oracle, step by step (C1-shaped
cantilever, Example 2 shape 425: 64 x 32, 3 levels), with the linear systems solved to a parity
tolerance; checkpoint/resume; the paper's barrier schedule."""
import numpy as np
import pytest

from oracle import fe, ip as oip, oc as ooc
from paper_1606_06201_gb300 import workloads as W

from gpu_helpers import dev, host, topo_lib, torch_cuda

pytestmark = pytest.mark.gpu


def _problem(nx, ny, volfrac=0.5):
    cfg = W.cantilever_2d(nx, ny, volfrac)
    prob = oip.Problem(fe.Grid(nx, ny), fe.element_stiffness(2), cfg["fixed"], cfg["f"], cfg["V"],
                       cfg["xbar"])
    return cfg, prob


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("shape,levels", [((16, 8), 2), ((64, 32), 3)])
def test_ip_trajectory_fp64_matches_oracle(shape, levels):
    torch = torch_cuda()
    topo = topo_lib()
    cfg, prob = _problem(*shape)
    _, oinfo = oip.ip_run(prob, record=True)
    traj = oinfo["traj"]
    # late IP systems are ill-conditioned (D -> 0 on intermediate elements): allow long solves
    solver = topo.IP(*shape, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"],
                     xbar=cfg["xbar"], levels=levels, max_iter=5000)
    opts = topo.ip_options(cg_tol=1e-12, cg_tol_init=1e-13)
    solver.init(opts)
    worst_x = worst_u = 0.0
    for k, st in enumerate(traj):
        info = solver.step(opts)
        u, x, phi, psi, scal, _ = solver.state()
        worst_x = max(worst_x, _rel(host(x), st["x"]))
        worst_u = max(worst_u, _rel(host(u), st["u"]))
        assert abs(scal[0] - st["lam"]) <= 1e-9 * max(1.0, abs(st["lam"])), k
        assert abs(info.crit - st["crit"]) <= 1e-8, k  # normalised terms: absolute
        assert info.ip_iters == sum(1 for t in traj[:k + 1] if t["crit"] <= 0.1), k
    assert info.done == 1 and info.newton == oinfo["newton"] and info.ip_iters == oinfo["ip"] == 12
    assert worst_x <= 1e-10 and worst_u <= 1e-10, (worst_x, worst_u)
    c = float(cfg["f"] @ host(solver.state()[0]))
    assert abs(c - oinfo["compliance"]) <= 1e-10 * abs(oinfo["compliance"])


def test_ip_mixed_run_matches_oracle():
    torch = torch_cuda()
    topo = topo_lib()
    cfg, prob = _problem(64, 32)
    z, oinfo = oip.ip_run(prob)
    solver = topo.IP(64, 32, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"],
                     xbar=cfg["xbar"], levels=3, precision=topo.MIXED, max_iter=5000)
    info = solver.run(topo.ip_options(cg_tol=1e-10))
    u, x, phi, psi, scal, _ = solver.state()
    assert info.done == 1 and info.ip_iters == 12
    assert _rel(host(x), z[2]) <= 1e-6
    c = float(cfg["f"] @ host(u))
    assert abs(c - oinfo["compliance"]) <= 1e-6 * abs(oinfo["compliance"])
    # the volume row is solved to the CG tolerance: sum x = V up to that accuracy
    assert abs(float(host(x).sum()) - cfg["V"]) <= 1e-8 * cfg["V"]


def test_ip_checkpoint_resume_is_bitwise():
    """Resuming from a snapshot (iterate, scalars and the augmented solver's power-iteration
    vectors) reproduces the uninterrupted run bit for bit."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg, _ = _problem(32, 16)
    opts = topo.ip_options(cg_tol=1e-10)
    a = topo.IP(32, 16, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0, levels=3)
    a.init(opts)
    for _ in range(5):
        a.step(opts)
    snap = [t.clone() if hasattr(t, "clone") else t.copy() for t in a.state()]
    assert snap[5].numel() > 1 and float(snap[5][-1]) == 1.0  # warm vectors from the last build
    for _ in range(4):
        a.step(opts)
    ref = [host(t) if hasattr(t, "cpu") else t for t in a.state()]
    b = topo.IP(32, 16, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0, levels=3)
    b.init(opts)
    b.set_state(*snap)
    for _ in range(4):
        b.step(opts)
    got = [host(t) if hasattr(t, "cpu") else t for t in b.state()]
    for g_, r_ in zip(got, ref):
        assert np.array_equal(g_, r_)


@pytest.mark.parametrize("precision", [0, 1])
def test_ip_fused_coarse_sweeps_give_identical_bits(precision):
    """The first two sweeps of each coarse level of Z in one kernel, with the lambda row reduced in
    the same pass, run the arithmetic of the separate sweeps: nine Newton steps agree bit for bit
    with fusion on and off."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg, _ = _problem(64, 32)
    opts = topo.ip_options(cg_tol=1e-8)
    out = []
    for fused in (False, True):
        a = topo.IP(64, 32, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0,
                    levels=4, precision=precision)
        a.set_vcycle_fusion(fused)
        a.init(opts)
        for _ in range(9):
            a.step(opts)
        out.append([host(t) if hasattr(t, "cpu") else t for t in a.state()])
        a.close()
    for g_, r_ in zip(out[0], out[1]):
        np.testing.assert_array_equal(g_, r_)


def test_inexact_newton_settings_of_tab_ip():
    """Sec. 8.1 (tab:IP) on the square cantilever of Example 1 with 6 refinements (64 x 64): Z
    systems solved to 1e-10 ("exact"), to a fixed 1e-2, and to 1e-2 halved at every barrier
    reduction.  As in the paper at tau_IP = 1e-8: all three need the same 12 major iterations and
    about the same Newton steps; the fixed tolerance needs the fewest CG iterations, the
    decreasing one more, the exact one most; the solutions agree (x_min of the same order)."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg = W.cantilever_2d(64, 64, 0.5)
    f = dev(torch, cfg["f"])
    res = {}
    for name, tol, fac in (("exact", 1e-10, 1.0), ("fixed", 1e-2, 1.0), ("decreasing", 1e-2, 0.5)):
        ip = topo.IP(64, 64, fixed=cfg["fixed"], f=f, V=cfg["V"], xbar=1.0, levels=4,
                     precision=topo.MIXED)
        info = ip.run(topo.ip_options(cg_tol=tol, cg_tol_factor=fac, max_newton=500))
        u, x = ip.state()[:2]
        res[name] = (info, float(cfg["f"] @ host(u)), host(x))
        ip.close()
    ex, fx, dc = res["exact"][0], res["fixed"][0], res["decreasing"][0]
    assert ex.done and fx.done and dc.done
    assert ex.ip_iters == fx.ip_iters == dc.ip_iters == 12
    assert fx.newton <= ex.newton + 5 and dc.newton <= ex.newton + 2
    assert fx.cg_iters < dc.cg_iters < ex.cg_iters
    c_ex = res["exact"][1]
    assert abs(res["fixed"][1] - c_ex) <= 1e-4 * c_ex
    assert abs(res["decreasing"][1] - c_ex) <= 1e-6 * c_ex
    x_ex = res["exact"][2]
    assert np.max(np.abs(res["fixed"][2] - x_ex)) <= 0.05
    assert np.max(np.abs(res["decreasing"][2] - x_ex)) <= 1e-3
    for name in ("fixed", "decreasing"):
        assert 0.5 * x_ex.min() <= res[name][2].min() <= 2.0 * x_ex.min()


def test_ip_rejects_bad_tolerance_options():
    torch = torch_cuda()
    topo = topo_lib()
    cfg, _ = _problem(16, 8)
    ip = topo.IP(16, 8, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0, levels=2)
    for kw in (dict(cg_tol_factor=0.0), dict(cg_tol_factor=1.5), dict(cg_tol=0.0)):
        with pytest.raises(topo.TopoError) as e:
            ip.init(topo.ip_options(**kw))
        assert e.value.status == topo.E_INVALID_ARG
    ip.close()


def test_ip_kkt_stop_rule_matches_oracle():
    """The scaled-KKT-residual stop (Remark in Sec. 3.4, tau_kkt = 1e-4): the GPU IP (FP64)
    stops at the oracle's Newton step with the oracle's x."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg, prob = _problem(32, 16)
    z, oinfo = oip.ip_run(prob, stop_rule="kkt", tau_kkt=1e-4)
    ip_ = topo.IP(32, 16, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0,
                  levels=3, max_iter=5000)
    info = ip_.run(topo.ip_options(cg_tol=1e-12, cg_tol_init=1e-13, stop_rule="kkt",
                                   tau_kkt=1e-4))
    assert info.done == 1 and info.newton == oinfo["newton"] and info.kkt <= 1e-4
    assert _rel(host(ip_.state()[1]), z[2]) <= 1e-8
    ip_.close()


def test_ip_example3_corner_supported_matches_oracle():
    """Example 3's setting (lower corners fixed, load at the lower edge's middle node) on a 32 x 8
    grid, FP64: the same Newton steps and barrier reductions as the oracle, x to 1e-8."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg = W.corner_supported_2d(32, 8, 0.5)
    prob = oip.Problem(fe.Grid(32, 8), fe.element_stiffness(2), cfg["fixed"], cfg["f"], cfg["V"],
                       cfg["xbar"])
    z, oinfo = oip.ip_run(prob)
    ip_ = topo.IP(32, 8, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0,
                  levels=3, max_iter=5000)
    info = ip_.run(topo.ip_options(cg_tol=1e-12, cg_tol_init=1e-13))
    assert info.done == 1 and info.newton == oinfo["newton"] and info.ip_iters == oinfo["ip"]
    x = host(ip_.state()[1])
    assert _rel(x, z[2]) <= 1e-8
    xr = x.reshape(8, 32)
    assert np.max(np.abs(xr - xr[:, ::-1])) <= 1e-8
    ip_.close()


def test_ip_rejects_infeasible_volume():
    torch = torch_cuda()
    topo = topo_lib()
    cfg, _ = _problem(16, 8)
    with pytest.raises(topo.TopoError) as e:
        topo.IP(16, 8, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=200.0, xbar=1.0, levels=2)
    assert e.value.status == topo.E_INFEASIBLE


@pytest.mark.parametrize("variant", ["aoc", "oc", "doc"])
def test_oc_trajectory_matches_oracle(variant):
    torch = torch_cuda()
    topo = topo_lib()
    cfg, prob = _problem(64, 32)
    feval = 20
    _, oinfo = ooc.oc_run(prob, variant=variant, tau_oc=0.0, max_feval=feval, xlow=1e-6,
                          record=True)
    vmap = {"aoc": topo.OC_AOC, "oc": topo.OC_PLAIN, "doc": topo.OC_DOC}
    solver = topo.OC(64, 32, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0,
                     levels=3)
    solver.init()
    opts = topo.oc_options(variant=vmap[variant], tau_oc=0.0, max_feval=feval, cg_tol0=1e-13,
                           adaptive_tol=False)
    # plain OC zig-zags between two clusters of points (Sec. 4.1) and amplifies rounding: 1e-9
    tol = 1e-9 if variant == "oc" else 1e-10
    comps = []
    for st in oinfo["traj"]:
        info = solver.step(opts)
        comps.append(info.compliance)
        assert abs(info.compliance - st["c"]) <= tol * abs(st["c"])
        assert abs(info.lam - st["lam"]) <= 10 * tol * st["lam"]
    assert _rel(host(solver.x()), oinfo["x"]) <= tol
    assert len(comps) == len(oinfo["traj"])


def test_oc_run_stops_on_compliance_change():
    torch = torch_cuda()
    topo = topo_lib()
    cfg, prob = _problem(32, 16)
    solver = topo.OC(32, 16, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0,
                     levels=3)
    solver.init()
    info = solver.run(topo.oc_options(tau_oc=1e-5, cg_tol0=1e-10, adaptive_tol=False))
    assert abs(info.compliance - info.compliance_prev) <= 1e-5
    x = host(solver.x())
    assert abs(x.sum() - cfg["V"]) <= 1e-6 * cfg["V"] and x.min() >= 1e-6 and x.max() <= 1.0
    _, oinfo = ooc.oc_run(prob, variant="aoc", tau_oc=1e-5, xlow=1e-6)
    assert info.iters == oinfo["iters"]


def test_ip_512x256_scalars_stay_consistent():
    """Example-2 shape 428 (512 x 256, 6 levels): large enough that every fixed-grid reduction runs
    its full grid.  After a few Newton steps the barrier parameters are exact powers of 0.2, lambda
    is finite and the volume constraint holds to the solve tolerance."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg = W.cantilever_2d(512, 256, 0.4)
    for prec in (topo.FP64, topo.MIXED):
        ip = topo.IP(512, 256, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0,
                     levels=6, precision=prec, max_iter=1000)
        opts = topo.ip_options(cg_tol=1e-8)
        ip.init(opts)
        for _ in range(4):
            info = ip.step(opts)
            u, x, phi, psi, scal, _ = ip.state()
            assert scal[1] == 0.2 ** info.ip_iters and scal[2] == 0.2 ** info.ip_iters
            assert np.isfinite(scal[0]) and abs(scal[0]) < 10.0
            xh = host(x)
            assert xh.min() > 0.0 and xh.max() < 1.0
            assert info.alpha > 0.5, info.alpha
        assert abs(xh.sum() - cfg["V"]) <= 1e-6 * cfg["V"]
        ip.close()


@pytest.mark.parametrize("variant", ["aoc", "oc"])
def test_oc_adaptive_cg_tolerance_matches_oracle(variant):
    """Sec. 6.2: linear systems solved by MGCG to tau, tau starting at 0.1 and multiplied by 0.1
    after an iteration whose compliance exceeds the previous one's, warm starts from the previous
    u.  The oracle runs the same rule with its reference MGCG (the same hierarchy depth, smoother
    and stopping test), so the GPU (FP64) takes the same tolerance at every iteration, the same
    CG iteration counts and the same compliances."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg, prob = _problem(64, 32)
    feval = 40
    sol = ooc.MGCGSolve(prob, levels=3, nu1=2, nu2=2, omega=0.6, tau=0.1)
    _, oinfo = ooc.oc_run(prob, variant=variant, tau_oc=0.0, max_feval=feval, solve=sol,
                          adaptive_tol=True)
    taus = oinfo["tau"]
    assert any(taus[k] < taus[k - 1] for k in range(1, len(taus)))  # the rule fired
    comp = oinfo["compliance"]
    # every decision c_k > c_{k-1} has a margin far above the solves' rounding (equal values come
    # from solves that took no CG iteration and left u unchanged, on both sides)
    assert all(comp[k] == comp[k - 1] or abs(comp[k] - comp[k - 1]) > 1e-9 * comp[k]
               for k in range(1, len(comp)))
    vmap = {"aoc": topo.OC_AOC, "oc": topo.OC_PLAIN}
    solver = topo.OC(64, 32, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0,
                     levels=3, omega=0.6)
    solver.init()
    opts = topo.oc_options(variant=vmap[variant], tau_oc=0.0, max_feval=feval, cg_tol0=0.1,
                           adaptive_tol=True)
    info = solver.run(opts)
    assert info.iters == oinfo["iters"] and info.feval == oinfo["feval"]
    assert info.cg_iters == sol.iterations
    assert abs(info.compliance - comp[-1]) <= 1e-10 * comp[-1]
    assert info.cg_tol == pytest.approx(sol.tau, rel=1e-12)
    solver.close()
    # step by step: the tolerance in force and the compliance of every iteration
    solver = topo.OC(64, 32, fixed=cfg["fixed"], f=dev(torch, cfg["f"]), V=cfg["V"], xbar=1.0,
                     levels=3, omega=0.6)
    solver.init()
    for k in range(oinfo["iters"]):
        info = solver.step(opts)
        assert abs(info.compliance - comp[k]) <= 1e-10 * comp[k], k
        if k + 1 < len(taus):
            assert info.cg_tol == pytest.approx(taus[k + 1], rel=1e-12), k
    solver.close()
