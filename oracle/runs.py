"""Oracle runs of whole IP and OC optimisations (Sec. 3, Sec. 4), shaped for the parity tests and
the bench's error-against-oracle fields (test infrastructure, like the rest of this package: it
imports the oracle and the seeded input generators only, no torch, so that it can run in a
spawned CPU process beside a GPU process).

Each function returns plain Python/numpy data small enough to pass between processes: the
per-step scalars of the whole run, and the iterates at the requested steps only.
"""
import os
import time

import numpy as np

from paper_1606_06201_gb300 import workloads as W

from . import fe, ip, oc


def spawn_pool(processes=2, threads=None):
    """A spawn-context process pool for oracle runs beside a GPU process.  The host's cores are
    split between the workers (BLAS and OpenMP threads set before they start): workers that each
    take every core spin against one another and run tens of times slower.  ``threads`` fixes the
    BLAS threads of each worker instead (1: the factorisations do not depend on how many cores the
    host has)."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    share = int(threads) if threads else max(1, _cores() // processes)
    for k in keys:
        os.environ[k] = str(share)
    try:
        pool = mp.get_context("spawn").Pool(processes)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, share


def cantilever_problem(nx, ny, volfrac):
    cfg = W.cantilever_2d(nx, ny, volfrac)
    return cfg, ip.Problem(fe.Grid(nx, ny), fe.element_stiffness(2), cfg["fixed"], cfg["f"],
                           cfg["V"], cfg["xbar"])


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def ip_run(nx, ny, volfrac, keep_steps=(), max_newton=500):
    """The Sec. 3 algorithm with exact Newton solves.  Returns the step count, barrier count,
    compliance, wall time, per-step lambda and Newton criterion, and (x, u) after each Newton
    step listed in keep_steps (1-based) and at the end."""
    _, prob = cantilever_problem(nx, ny, volfrac)
    t0 = time.perf_counter()
    z, info = ip.ip_run(prob, record=True, max_newton=max_newton)
    wall = time.perf_counter() - t0
    traj = info["traj"]
    kept = {k: (traj[k - 1]["x"], traj[k - 1]["u"]) for k in keep_steps if k <= len(traj)}
    return dict(newton=info["newton"], ip=info["ip"], compliance=info["compliance"],
                wall_s=wall, cores=_cores(), lam=[t["lam"] for t in traj],
                crit=[t["crit"] for t in traj], kept=kept, x=z[2], u=z[0])


def aoc_run(nx, ny, volfrac, max_feval, keep_iters=(), xlow=1e-6):
    """Algorithm AOC with exact solves for max_feval linear solves.  Returns per-iteration
    compliance and lambda (of the iteration's first solve), (x, u) at the listed iterations
    (1-based: the iterate the iteration starts from and its solve), the final x, and the wall
    time."""
    _, prob = cantilever_problem(nx, ny, volfrac)
    t0 = time.perf_counter()
    x, info = oc.oc_run(prob, variant="aoc", tau_oc=0.0, max_feval=max_feval, xlow=xlow,
                        record=True)
    wall = time.perf_counter() - t0
    traj = info["traj"]
    kept = {k: (traj[k - 1]["x"], traj[k - 1]["u"]) for k in keep_iters if k <= len(traj)}
    return dict(feval=info["feval"], iters=info["iters"], wall_s=wall, cores=_cores(),
                compliance=[t["c"] for t in traj], lam=[t["lam"] for t in traj], kept=kept, x=x)
