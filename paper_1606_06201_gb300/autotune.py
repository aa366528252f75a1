"""Smoother and tile autotuner for the MGCG solver.

For one grid, boundary mask, precision and batch size it times complete solves (hierarchy build +
PCG to the requested tolerance) over
  * damped Jacobi with omega in a small set and nu1 = nu2 in ``sweeps``,
  * the Chebyshev smoother (topo_solver_desc.smoother = 1) of each degree in ``cheb_degrees``,
  * for 2D grids, the strip height of the finest-level warp sweeps in ``rows`` (0 = automatic)
    with the fastest smoother,
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


def _time(nx, ny, nz, fixed, x, f, levels, precision, nrhs, tol, reps, smoother, omega, nu,
          rows):
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, precision=precision, nu1=nu, nu2=nu,
                    omega=omega, nrhs=nrhs, smoother=smoother)
    try:
        if rows:
            s.set_sweep_rows(rows)
        u = torch.zeros_like(f)
        s.set_density(x)
        _, info = s.solve(f, u, tol=tol, allow_not_converged=True)  # warm-up and capture
        if info.status != topo.OK:
            return None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            s.set_density(x)
            _, info = s.solve(f, u, tol=tol)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, info.iterations
    except topo.TopoError:
        return None
    finally:
        s.close()


def autotune(nx, ny, nz, fixed, x, f, levels, precision=topo.MIXED, nrhs=1, tol=1e-8,
             omegas=None, sweeps=(1, 2, 3), cheb_degrees=(1, 2, 3), rows=(0, 4, 8, 16), reps=2,
             cache_path=None):
    """Return {"smoother", "omega", "nu", "rows", "ms", "iterations", "tried"} of the fastest
    converging setting ("nu" is the Chebyshev degree for the Chebyshev smoother).

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
    cands = [("jacobi", 0, om, nu) for om in omegas for nu in sweeps]
    cands += [("chebyshev", 1, 0.6 if not nz else 0.5, deg) for deg in cheb_degrees]
    best, tried = None, 0
    for name, smoother, omega, nu in cands:
        r = _time(nx, ny, nz, fixed, x, f, levels, precision, nrhs, tol, reps, smoother, omega,
                  nu, 0)
        tried += 1
        if r is not None and (best is None or r[0] < best["ms"]):
            best = {"smoother": name, "omega": omega, "nu": nu, "rows": 0, "ms": r[0],
                    "iterations": r[1]}
    if best is None:
        raise RuntimeError("autotune: no smoother setting converged")
    if not nz and precision == topo.MIXED:  # the tile of the finest-level FP32 sweeps
        smoother = 1 if best["smoother"] == "chebyshev" else 0
        for rw in rows:
            if rw == 0:
                continue
            r = _time(nx, ny, nz, fixed, x, f, levels, precision, nrhs, tol, reps, smoother,
                      best["omega"], best["nu"], rw)
            tried += 1
            if r is not None and r[0] < best["ms"]:
                best.update(rows=rw, ms=r[0], iterations=r[1])
    best["tried"] = tried
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


def solver_for(tuned, nx, ny, nz, fixed, levels, precision=topo.MIXED, nrhs=1, max_iter=1000):
    """A Solver configured with an autotune() result."""
    s = topo.Solver(nx, ny, nz, fixed=fixed, levels=levels, precision=precision,
                    nu1=tuned["nu"], nu2=tuned["nu"], omega=tuned["omega"], nrhs=nrhs,
                    max_iter=max_iter, smoother=1 if tuned["smoother"] == "chebyshev" else 0)
    if tuned.get("rows"):
        s.set_sweep_rows(tuned["rows"])
    return s
