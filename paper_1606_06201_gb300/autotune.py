"""Smoother autotuner for the MGCG solver.

For one grid, boundary mask, precision and batch size it times complete solves (hierarchy build +
PCG to the requested tolerance) over a small grid of damped-Jacobi parameters (omega, nu1 = nu2)
and keeps the fastest setting that converges.  Results are cached per
(dim, nx, ny, nz, levels, precision, nrhs) in memory and, if a path is given, in a JSON file.
The timing uses CUDA events on the current stream; all work runs in the CUDA library.
"""
import json
import os

import torch

from . import topo

_CACHE = {}


def _key(nx, ny, nz, levels, precision, nrhs):
    return "%d:%dx%dx%d:L%d:P%d:R%d" % (3 if nz else 2, nx, ny, nz, levels, precision, nrhs)


def autotune(nx, ny, nz, fixed, x, f, levels, precision=topo.MIXED, nrhs=1, tol=1e-8,
             omegas=None, sweeps=(1, 2, 3), reps=2, cache_path=None):
    """Return {"omega", "nu", "ms", "iterations"} of the fastest converging setting.

    x: density tensor (device, FP64); f: right-hand sides (device, FP64, nrhs x n).
    """
    key = _key(nx, ny, nz, levels, precision, nrhs)
    if key in _CACHE:
        return _CACHE[key]
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            disk = json.load(fh)
        if key in disk:
            _CACHE[key] = disk[key]
            return disk[key]
    if omegas is None:
        omegas = (0.4, 0.5, 0.6, 0.7) if not nz else (0.3, 0.4, 0.5, 0.6)
    best = None
    for omega in omegas:
        for nu in sweeps:
            s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, precision=precision,
                            nu1=nu, nu2=nu, omega=omega, nrhs=nrhs)
            u = torch.zeros_like(f)
            s.set_density(x)
            _, info = s.solve(f, u, tol=tol, allow_not_converged=True)  # warm-up and capture
            if info.status != topo.OK:
                s.close()
                continue
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                s.set_density(x)
                _, info = s.solve(f, u, tol=tol)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            s.close()
            if best is None or ms < best["ms"]:
                best = {"omega": omega, "nu": nu, "ms": ms, "iterations": info.iterations}
    if best is None:
        raise RuntimeError("autotune: no smoother setting converged")
    _CACHE[key] = best
    if cache_path:
        disk = {}
        if os.path.exists(cache_path):
            with open(cache_path) as fh:
                disk = json.load(fh)
        disk[key] = best
        with open(cache_path, "w") as fh:
            json.dump(disk, fh, indent=1)
    return best
