"""The FP32 finest-level sweeps with two node columns per lane against the one-column kernels
(TOPO_Q1_NARROW=1): the same per-node arithmetic in the same order, so the mixed-precision
V-cycle outputs (first two sweeps from zero, residual and restriction, prolongation with the first
post-sweep, the plain sweeps of the unfused path) agree bit for bit on grids whose widths are not
multiples of the warp tile, with several right-hand sides and masks.  Whole solves agree to
rounding: the fused r~^T y~ of the last sweep sums its terms in another order."""
import numpy as np
import pytest

from paper_1606_06201_gb300 import workloads as W

from gpu_helpers import dev, host, rel_err, topo_lib, torch_cuda

pytestmark = pytest.mark.gpu


def _x(nx, ny, seed):
    return np.random.default_rng(seed).uniform(1e-3, 1.0, nx * ny)


def _mask(kind, nx, ny):
    if kind == "clamp":
        return W.clamp_xmin(nx, ny)
    return W.corner_supported_2d(nx, ny, 0.5)["fixed"]


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("shape,nrhs,mask", [((2048, 1024, 9), 1, "clamp"),
                                             ((200, 48, 4), 2, "clamp"),
                                             ((124, 64, 3), 1, "corner"),
                                             ((122, 28, 2), 2, "clamp"),
                                             ((60, 30, 2), 3, "corner"),
                                             ((12, 6, 2), 1, "clamp"),
                                             ((250, 4, 2), 1, "clamp")])
def test_wide_sweeps_match_one_column_sweeps(shape, nrhs, mask, fused, monkeypatch):
    torch = torch_cuda()
    topo = topo_lib()
    nx, ny, levels = shape
    fixed = _mask(mask, nx, ny)
    x = dev(torch, _x(nx, ny, 5))
    R = np.stack([W.random_vector(fixed.size, 80 + k, fixed) for k in range(nrhs)])
    F = np.stack([W.normal_load(fixed, 90 + k) for k in range(nrhs)])
    out = []
    for narrow in ("1", "0"):
        monkeypatch.setenv("TOPO_Q1_NARROW", narrow)
        s = topo.Solver(nx, ny, fixed=fixed, levels=levels, precision=topo.MIXED, nrhs=nrhs,
                        max_iter=500)
        s.set_vcycle_fusion(fused)
        s.set_density(x)
        y = host(s.apply_vcycle(dev(torch, R)))
        u, info = s.solve(dev(torch, F), tol=1e-9)
        out.append((y, host(u), info.iterations))
        s.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert abs(out[0][2] - out[1][2]) <= 1
    assert rel_err(out[1][1], out[0][1]) <= 1e-8
