"""Workloads run against both builds of the library by test_gpu_bounds_check.py: ragged 2D
grids (mixed with the wide and fused finest-level kernels, FP64), a batched 3D grid with the tile
sweeps and both outer-operator forms, the IP method and AOC on a small cantilever.  Also run as a
script: ``python bounds_check_cases.py OUT.npz`` (the binding loads the library that
TOPO_LIBRARY names) writes the results and the index-check report."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1606_06201_gb300 import workloads as W  # noqa: E402


def _x(n, seed):
    return np.random.default_rng(seed).uniform(1e-3, 1.0, n)


def run_cases(topo, torch):
    out = {}

    def dev(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")

    for name, (nx, ny, levels, prec, nrhs) in {
            "mixed_200x48": (200, 48, 4, topo.MIXED, 2),
            "mixed_122x28": (122, 28, 2, topo.MIXED, 1),
            "fp64_64x32": (64, 32, 3, topo.FP64, 1)}.items():
        fixed = W.clamp_xmin(nx, ny)
        F = np.stack([W.normal_load(fixed, 90 + k) for k in range(nrhs)])
        s = topo.Solver(nx, ny, fixed=fixed, levels=levels, precision=prec, nrhs=nrhs)
        s.set_density(dev(_x(nx * ny, 91)))
        U, info = s.solve(dev(F if nrhs > 1 else F[0]), tol=1e-10)
        out[name] = U.cpu().numpy()
        out[name + "_it"] = np.array([info.iterations, info.status])
        out[name + "_mg"] = s.apply_vcycle(dev(F if nrhs > 1 else F[0])).cpu().numpy()
        s.close()
    cfg = W.random_field_3d(24, 16, 16, n_rhs=3)
    for outer in ("buffered", "tile"):
        os.environ["TOPO_HEX_OUTER"] = outer
        s = topo.Solver(24, 16, 16, fixed=cfg["fixed"], levels=3, precision=topo.MIXED, nrhs=3)
        s.set_density(dev(cfg["x"]))
        U, info = s.solve(dev(cfg["f"]), tol=1e-10)
        out["hex_" + outer] = U.cpu().numpy()
        out["hex_" + outer + "_it"] = np.array([info.iterations, info.status])
        s.close()
    os.environ.pop("TOPO_HEX_OUTER", None)
    c = W.cantilever_2d(64, 32, 0.4)
    ip = topo.IP(64, 32, fixed=c["fixed"], f=dev(c["f"]), V=c["V"], xbar=1.0, levels=3,
                 precision=topo.MIXED)
    opts = topo.ip_options(cg_tol=1e-8)
    ip.init(opts)
    for _ in range(5):
        ip.step(opts)
    out["ip_x"] = ip.state()[1].cpu().numpy()
    ip.close()
    oc = topo.OC(64, 32, fixed=c["fixed"], f=dev(c["f"]), V=c["V"], xbar=1.0, levels=3,
                 precision=topo.MIXED)
    oc.init()
    oopts = topo.oc_options(variant=topo.OC_AOC, max_feval=10)
    for _ in range(4):
        oc.step(oopts)
    out["oc_x"] = oc.x().cpu().numpy()
    oc.close()
    return out


if __name__ == "__main__":
    import torch

    from paper_1606_06201_gb300 import topo

    assert topo.bounds_check_enabled(), "TOPO_LIBRARY does not name the index-checked build"
    res = run_cases(topo, torch)
    count, index, size, file, line = topo.bounds_report()
    res["report"] = np.array([count, index, size, line])
    # one check that fails by construction, in a kernel that addresses no buffer
    topo.bounds_selftest(5, 3)
    res["selftest"] = np.array(topo.bounds_report(reset=True)[:3] + (topo.bounds_report()[0],))
    np.savez(sys.argv[1], **res)
