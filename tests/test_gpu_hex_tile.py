"""The tile form of the 3D finest-level kernels (element forces through shared memory, one launch)
against the node-parallel and buffered forms on grids that span several tiles, z chunks and a
ragged edge in every direction, with several right-hand sides:

* the V-cycle operator with the element rows of K0 (TOPO_HEX_SWEEP=dense) has the arithmetic of
  the node-parallel kernel (TOPO_HEX_SWEEP=node): V-cycle outputs agree bit for bit, whole solves
  to rounding (the tile forms fuse r~^T y~ and beta into the last smoothing sweep);
* the Walsh-Hadamard V-cycle operator (the default), and the dense one on the tensor cores
  (TOPO_HEX_SWEEP=tc, 3 x TF32), are the same operator with other roundings: the solves reach the
  node-parallel solutions and the exact solution of the oracle's sparse matrix;
* the tile outer operator (TOPO_HEX_OUTER=tile) forms the buffered kernels' q; its p^T q sums in
  another order, so solves agree with the buffered form (the default) to rounding, with the same
  iteration counts.
"""
import numpy as np
import pytest

from paper_1606_06201_gb300 import workloads as W

from oracle.linsolve import SPDSolver
from gpu_helpers import dev, host, oracle_K_free, rel_err, topo_lib, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [((16, 8, 8, 3), 1), ((48, 40, 24, 4), 3), ((136, 24, 16, 3), 2), ((8, 72, 12, 3), 1)]


def _x(nx, ny, nz, seed):
    return np.random.default_rng(seed).uniform(1e-3, 1.0, nx * ny * nz)


def _solve(monkeypatch, env, shape, nrhs, precision, tol=1e-10, vcycle_input=None):
    torch = torch_cuda()
    topo = topo_lib()
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    nx, ny, nz, levels = shape
    fixed = W.clamp_xmin(nx, ny, nz)
    x = dev(torch, _x(nx, ny, nz, 61))
    F = np.stack([W.normal_load(fixed, 62 + k) for k in range(nrhs)])
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, precision=precision, nrhs=nrhs)
    s.set_density(x)
    U, info = s.solve(dev(torch, F if nrhs > 1 else F[0]), tol=tol)
    out = [host(U), info.iterations]
    if vcycle_input is not None:  # (one vector per right-hand side of the solver)
        A = np.stack([vcycle_input * (1.0 + 0.5 * k) for k in range(nrhs)])
        assert A.size == s.n * nrhs
        out.append(host(s.apply_vcycle(dev(torch, A))))
    s.close()
    for k in env:
        monkeypatch.delenv(k)
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,nrhs", SHAPES)
def test_dense_tile_sweep_gives_the_node_parallel_bits(shape, nrhs, precision, monkeypatch):
    nx, ny, nz, _ = shape
    fixed = W.clamp_xmin(nx, ny, nz)
    a = W.random_vector(fixed.size, 63, fixed)
    U0, it0, M0 = _solve(monkeypatch, {"TOPO_HEX_SWEEP": "node"}, shape, nrhs, precision,
                         vcycle_input=a)
    U1, it1, M1 = _solve(monkeypatch, {"TOPO_HEX_SWEEP": "dense"}, shape, nrhs, precision,
                         vcycle_input=a)
    np.testing.assert_array_equal(M0, M1)
    # (whole solves to rounding: the tile forms fuse r~^T y~ and beta into the last sweep, which
    # sums the dot product in another order than the separate kernel)
    assert abs(it0 - it1) <= 1
    assert rel_err(U1, U0) <= (1e-12 if precision == 0 else 1e-8)


@pytest.mark.parametrize("form", ["wht", "tc"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,nrhs", SHAPES)
def test_walsh_hadamard_tile_sweep_agrees_with_the_node_parallel_operator(shape, nrhs, precision,
                                                                          form, monkeypatch):
    """(form tc: the dense element product on the tensor cores, 3 x TF32, in the FP32 V-cycle;
    the FP64 V-cycle keeps FMA chains.)"""
    tol = 1e-11 if precision == 0 else 1e-10
    U, it = _solve(monkeypatch, {"TOPO_HEX_SWEEP": form}, shape, nrhs, precision, tol=tol)
    Un, itn = _solve(monkeypatch, {"TOPO_HEX_SWEEP": "node"}, shape, nrhs, precision, tol=tol)
    assert abs(it - itn) <= 1
    assert rel_err(U, Un) <= 1e-8


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,nrhs", [((16, 8, 8, 3), 1), ((24, 16, 8, 3), 3)])
def test_walsh_hadamard_tile_sweep_solves_the_system(shape, nrhs, precision, monkeypatch):
    nx, ny, nz, _ = shape
    tol = 1e-11 if precision == 0 else 1e-9
    U, _ = _solve(monkeypatch, {}, shape, nrhs, precision, tol=tol)
    fixed = W.clamp_xmin(nx, ny, nz)
    K, free, grid = oracle_K_free(nx, ny, nz, _x(nx, ny, nz, 61), fixed.astype(bool))
    solver = SPDSolver(K, grid, free)
    U = U.reshape(nrhs, -1)
    for r in range(nrhs):
        f = W.normal_load(fixed, 62 + r)
        exact = np.zeros(fixed.size)
        exact[free] = solver.solve(f[free])
        assert rel_err(U[r], exact) <= (1e-9 if precision == 0 else 1e-7), r


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,nrhs", SHAPES)
def test_tile_outer_operator_matches_the_buffered_form(shape, nrhs, precision, monkeypatch):
    U0, it0 = _solve(monkeypatch, {"TOPO_HEX_SWEEP": "node"}, shape, nrhs, precision)
    U1, it1 = _solve(monkeypatch, {"TOPO_HEX_OUTER": "tile", "TOPO_HEX_SWEEP": "node"}, shape,
                     nrhs, precision)
    assert it0 == it1
    assert rel_err(U1, U0) <= 1e-12
