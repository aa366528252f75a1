"""Boundary calls beyond the solve: the caller's element matrix K0 (Eq. (to) takes K_i as data),
the workspace query before creation, and checkpoint/resume of OC runs (Sec. 4)."""
import numpy as np
import pytest

from oracle import fe
from oracle.linsolve import SPDSolver
from paper_1606_06201_gb300 import workloads as W

from gpu_helpers import dev, host, rel_err, topo_lib, torch_cuda

pytestmark = pytest.mark.gpu

# an orthotropic plane-stress material with an xx-xy coupling: K0 has no butterfly structure
D_ANISO = np.array([[1.3, 0.35, 0.12], [0.35, 0.8, 0.05], [0.12, 0.05, 0.42]])


def _exact(nx, ny, nz, K0, x, fixed, f):
    grid = fe.Grid(nx, ny, nz)
    free = fe.free_dofs(fixed.astype(bool))
    K = fe.assemble(grid, K0, x)[free][:, free].tocsr()
    u = np.zeros(grid.n_dofs)
    u[free] = SPDSolver(K, grid, free).solve(f[free])
    return u


@pytest.mark.parametrize("kind", ["scaled", "anisotropic", "scaled3d"])
@pytest.mark.parametrize("precision", [0, 1])
def test_caller_K0_solves_its_own_problem(kind, precision):
    """K0 given by the caller: a scaled isotropic matrix keeps the specialised finest-level kernels
    (their coefficients are derived from K0 itself), an anisotropic one falls back to the generic
    kernels; both solve K(x) u = f with that K0 (oracle: banded Cholesky with the same K0)."""
    torch = torch_cuda()
    topo = topo_lib()
    if kind == "scaled3d":
        nx, ny, nz, levels = 8, 4, 4, 2
        K0 = 2.5 * fe.element_stiffness(3)
    else:
        nx, ny, nz, levels = 64, 32, 0, 3
        K0 = 2.5 * fe.element_stiffness(2) if kind == "scaled" else fe.element_stiffness(2, D=D_ANISO)
    fixed = W.clamp_xmin(nx, ny, nz)
    x = np.random.default_rng(3).uniform(1e-2, 1.0, nx * ny * max(nz, 1))
    f = W.normal_load(fixed, 4)
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, precision=precision, K0=K0,
                    max_iter=2000)
    s.set_density(dev(torch, x))
    tol = 1e-12 if precision == 0 else 1e-9
    u, info = s.solve(dev(torch, f), tol=tol)
    exact = _exact(nx, ny, nz, K0, x, fixed, f)
    assert rel_err(host(u), exact) <= (1e-9 if precision == 0 else 1e-6)
    # the operator itself against the oracle's K(x) with the caller's K0
    v = W.random_vector(fixed.size, 5, fixed)
    Kv = host(s.apply_K(dev(torch, v)))
    ref = fe.assemble(fe.Grid(nx, ny, nz), K0, x) @ v
    ref[fixed.astype(bool)] = 0.0
    assert np.max(np.abs(Kv - ref)) <= 1e-13 * np.max(np.abs(ref))
    s.close()


@pytest.mark.parametrize("kw", [dict(nx=64, ny=32, levels=3),
                                dict(nx=64, ny=32, levels=3, precision=1),
                                dict(nx=256, ny=128, levels=6, precision=1, nrhs=3),
                                dict(nx=64, ny=32, levels=4, smoother=1),
                                dict(nx=64, ny=32, levels=4, precision=1, omega_auto=True),
                                dict(nx=64, ny=32, levels=3, precision=1, flexible=1),
                                dict(nx=64, ny=32, levels=3, generic_kernels=True),
                                dict(nx=16, ny=8, nz=8, levels=3, precision=1, nrhs=2),
                                dict(nx=16, ny=8, nz=8, levels=2)])
def test_workspace_query_equals_allocation(kw):
    torch_cuda()
    topo = topo_lib()
    nz = kw.get("nz", 0)
    fixed = W.clamp_xmin(kw["nx"], kw["ny"], nz)
    planned = topo.workspace_bytes(fixed=fixed, **kw)
    s = topo.Solver(fixed=fixed, **kw)
    assert s.device_bytes == planned
    s.close()


@pytest.mark.parametrize("variant,precision", [("aoc", 0), ("doc", 1), ("aoc_adaptive", 1)])
def test_oc_checkpoint_resume_is_bitwise(variant, precision):
    """A run resumed from a snapshot (x, u, the tolerance and compliance history, the counts)
    repeats the uninterrupted run bit for bit, also under the adaptive tolerance of Sec. 6.2."""
    torch = torch_cuda()
    topo = topo_lib()
    cfg = W.cantilever_2d(64, 32, 0.5)
    f = dev(torch, cfg["f"])
    vmap = {"aoc": topo.OC_AOC, "doc": topo.OC_DOC, "aoc_adaptive": topo.OC_AOC}
    opts = topo.oc_options(variant=vmap[variant], tau_oc=0.0, cg_tol0=0.1 if "adaptive" in variant
                           else 1e-8, adaptive_tol="adaptive" in variant)

    def make():
        o = topo.OC(64, 32, fixed=cfg["fixed"], f=f, V=cfg["V"], xbar=1.0, levels=3,
                    precision=precision)
        o.init()
        return o

    a = make()
    for _ in range(4):
        a.step(opts)
    snap = a.state()
    snap = (snap[0].clone(), snap[1].clone(), snap[2].copy(), snap[3].clone())
    ref_infos = [a.step(opts) for _ in range(5)]
    ref = a.state()
    b = make()
    b.set_state(*snap)
    infos = [b.step(opts) for _ in range(5)]
    got = b.state()
    np.testing.assert_array_equal(host(got[0]), host(ref[0]))
    np.testing.assert_array_equal(host(got[1]), host(ref[1]))
    np.testing.assert_array_equal(got[2], ref[2])
    for i, j in zip(infos, ref_infos):
        assert (i.compliance, i.lam, i.cg_tol, i.cg_iters, i.feval) == \
            (j.compliance, j.lam, j.cg_tol, j.cg_iters, j.feval)
    with pytest.raises(topo.TopoError):
        bad = snap[2].copy()
        bad[0] = -5.0
        b.set_state(snap[0], snap[1], bad)
    a.close()
    b.close()


def test_per_solve_records(tmp_path):
    """topo_set_record_file: one JSON line per solve with the solve's own counts."""
    import json
    torch = torch_cuda()
    topo = topo_lib()
    fixed = W.clamp_xmin(64, 32)
    s = topo.Solver(64, 32, fixed=fixed, levels=3, precision=topo.MIXED)
    s.set_density(dev(torch, np.random.default_rng(1).uniform(1e-2, 1, 64 * 32)))
    path = tmp_path / "solves.jsonl"
    s.set_record_file(path)
    infos = [s.solve(dev(torch, W.normal_load(fixed, k)), tol=tol)[1]
             for k, tol in ((1, 1e-8), (2, 1e-10))]
    s.set_record_file(None)
    s.solve(dev(torch, W.normal_load(fixed, 3)), tol=1e-8)
    recs = [json.loads(line) for line in open(path)]
    assert len(recs) == 2
    for r, info, tol in zip(recs, infos, (1e-8, 1e-10)):
        assert r["iterations"] == info.iterations and r["rel_residual"] == info.rel_residual
        assert r["tol"] == tol and r["precision"] == "mixed" and r["system"] == "K"
        assert r["free_dofs"] == int(np.count_nonzero(fixed == 0)) and r["status"] == 0
    s.close()
