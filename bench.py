"""Benchmark: standalone MGCG solve K(x) u = f to a relative residual of 1e-8 on a 2048 x 1024 Q1
plane-stress grid (4.2M DOFs, 9 levels), densities 10^U(-3,0) smoothed by a 5x5 box filter, load
N(0,1) on the free DOFs, left edge clamped.  One step = Galerkin hierarchy build + PCG solve
(Algorithm MG / Algorithm PCG), inputs resident in HBM.  Metric: free DOFs x CG iterations / s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The headline is the mixed-precision solver (FP32 V-cycle, FP64 CG); the plain FP64 solver is
reported beside it.  ``--impl reference`` times the CPU oracle (plain scipy MGCG) on a bounded
sample of the same recipe.  Under torchrun every rank solves its own copy (replicas: the method
has no exchange step on one grid) and rank 0 prints one JSON line.
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1606_06201_gb300 import workloads as W  # noqa: E402

NX, NY, LEVELS, TOL = 2048, 1024, 9, 1e-8
# the oracle's IP / AOC runs that give the errors against the oracle are collected at most this
# long after the bench starts (on a GB300 host the 512 x 256 runs take about a minute each)
ORACLE_DEADLINE_S = 420.0
T_START = time.perf_counter()
METRIC = "MGCG DOF·iterations/s at 1e-8 rel. residual (mixed: FP32 V-cycle, FP64 CG)"
UNIT = "DOF·it/s"
WORKLOAD = "mgcg_2d_q1_2048x1024_9lev_logunif_box5_normal_load"
# Derived issue peaks (not measured; MEASURED_PEAKS.json has the copy bandwidth and cuBLAS bf16
# only): SMs x lanes x clock, with the SM count read from the device at run time
# (cudaDeviceProp.multiProcessorCount: 152 on GB300) and the maximum SM clock of MEASURED_PEAKS.json
# (2070 MHz).  FP64: 2 instructions per SM and clock (an add, multiply or fused multiply-add each
# take one issue slot; a probe on this part measured 0.60e12 FP64 FMA/s); FP32: 128 lanes per SM,
# one operation per lane and clock (an FMA counts as one).
SM_COUNT_DEFAULT, SM_MHZ_DEFAULT = 152, 2070.0


def derived_peaks(sm_count, sm_mhz):
    """(FP64, FP32) issue rates in T operations/s from unit counts and clock."""
    return sm_count * 2 * sm_mhz * 1e6 / 1e12, sm_count * 128 * sm_mhz * 1e6 / 1e12


FP64_PEAK_TOPS, FP32_PEAK_TOPS = derived_peaks(SM_COUNT_DEFAULT, SM_MHZ_DEFAULT)
# FP64 operations of the FP64 butterfly operator kernel: 37 per element (two 4-point butterflies
# per displacement component: 15 adds; 8 products; 14 multiply-adds for the scalings and the inverse
# butterflies) + 6 node-assembly adds + 2 FMA of the fused p^T q per node.
OPS_PER_ELEM, OPS_PER_NODE = 37.0, 8.0
# FP32 operations of the same operator in float pairs: per element 29 pair additions (8 FP32
# operations each: TwoSum and the low parts, no renormalisation) and 12 pair products (4: product,
# FMA error term, two cross FMAs, no renormalisation), plus the 2 pair additions of the carried
# node sums; per output node 4 pair additions of the node sums, 2 renormalised products (7) + 2
# renormalised additions (11) of p^T q, and 2 FP32 multiplies of each of the two input splits.
DF_OPS_PER_ELEM = 29 * 8 + 12 * 4 + 2 * 8
DF_OPS_PER_NODE = 4 * 8 + 2 * 7 + 2 * 11 + 4
# DRAM bytes of one launch of the FP64 operator on this workload from an ncu capture; None until
# the operator as built now (37-operation element product) has been captured.
OPERATOR_DRAM_BYTES = None
# The same for the float-pair operator (ncu capture of k_q1_sweep_df on this workload:
# 54.73 MB read + 2.70 MB write).
DF_OPERATOR_DRAM_BYTES = 57426944.0


def _measured_hbm_gbs():
    """Measured copy bandwidth of this GPU model (MEASURED_PEAKS.json), else 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def _measured_sm_max_mhz():
    """Maximum SM clock recorded with the measured peaks, else 2070 MHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return SM_MHZ_DEFAULT


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(v, ws, device):
    """The largest of every rank's v (a time: the job ends with its slowest replica); v itself on
    one rank.  device: where the process group's backend reduces (cuda for NCCL, cpu for gloo)."""
    if ws == 1:
        return v
    import torch
    t = torch.tensor([float(v)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def oracle_mgcg_sample(nx, ny, levels, seconds=None, reps=1):
    """Time the CPU oracle's MGCG (scipy sparse, Algorithm PCG + Algorithm MG) on the same recipe."""
    from oracle import fe, mg
    cfg = W.random_field_2d(nx, ny)
    grid = fe.Grid(nx, ny)
    fixed = cfg["fixed"].astype(bool)
    free = fe.free_dofs(fixed)
    total_t, total_work, runs = 0.0, 0.0, 0
    while True:
        t0 = time.perf_counter()
        K = fe.assemble(grid, fe.element_stiffness(2), cfg["x"])[free][:, free].tocsr()
        levs = mg.hierarchy(grid, fixed, K, levels)
        _, it, _ = mg.pcg(K, cfg["f"][free], lambda r: mg.vcycle(levs, r, 2, 2, 0.6), tol=TOL)
        total_t += time.perf_counter() - t0
        total_work += free.size * it
        runs += 1
        if (seconds is None and runs >= reps) or (seconds is not None and total_t >= seconds):
            break
    return total_work / total_t, total_t, runs, free.size, it


def reference_arm(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    nx, ny, lev = 512, 256, 7
    for _ in range(args.warmup):
        oracle_mgcg_sample(nx, ny, lev)
    t0 = time.perf_counter()
    work = 0.0
    for _ in range(args.steps):
        v, t, _, nfree, it = oracle_mgcg_sample(nx, ny, lev)
        work += nfree * it
    el = time.perf_counter() - t0
    value = work / el
    sample = "oracle MGCG (scipy sparse, FP64) on the same recipe at 512x256 (263,168 free DOFs, 7 levels), " \
             "hierarchy build + PCG to 1e-8 per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "512x256"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ip", action="store_true", help="skip the 512x256 IP/OC wall-time runs")
    ap.add_argument("--outer-fp64", action="store_true",
                    help="mixed solver with the FP64 outer operator instead of float pairs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="--only batched3d: damped Jacobi omega=0.6, nu=1 without the autotuner")
    ap.add_argument("--only", choices=["mixed", "fp64", "batched3d", "ip", "simp", "oc_accuracy"],
                    default=None,
                    help="run one solver configuration only (for profiler launch lists); no JSON "
                         "line.  oc_accuracy: the Sec. 8.2-8.3 accuracy study (one JSON line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    ws, rank = _dist()
    # the CPU baseline first, on an idle host (the oracle processes below share its cores)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not args.only:
        v, t, runs, nf, it = oracle_mgcg_sample(1024, 512, 8, seconds=10.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "oracle MGCG (scipy sparse, FP64, single thread) on the same recipe at "
                         "1024x512 (%d free DOFs, 8 levels), %d run(s), %.1f s" % (nf, runs, t)}
    # the oracle's IP and AOC runs of the Example-2-shaped workloads (64 x 32 and 512 x 256), for
    # the errors against the oracle beside the GPU runs: started now, in two spawned CPU
    # processes that share the host's cores, and collected after the GPU work
    oracle_jobs, oracle_pool = {}, None
    if rank == 0 and not args.no_ip and not args.only:
        from oracle import runs as oruns
        oracle_pool, _ = oruns.spawn_pool(2)
        oracle_jobs = {
            "c1": (oracle_pool.apply_async(oruns.ip_run, (64, 32, 0.5)),
                   oracle_pool.apply_async(oruns.aoc_run, (64, 32, 0.5, 50))),
            "c2": (oracle_pool.apply_async(oruns.ip_run, (512, 256, 0.4)),
                   oracle_pool.apply_async(oruns.aoc_run, (512, 256, 0.4, 50)))}
        oracle_pool.close()

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1606_06201_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_1606_06201_gb300 import topo

    cfg = W.random_field_2d(NX, NY)
    nfree = int(np.count_nonzero(cfg["fixed"] == 0))
    x_d = torch.as_tensor(cfg["x"], device=dev)
    f_d = torch.as_tensor(cfg["f"], device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def run(precision, steps, warmup, profile_mask=0, host_io=False):
        s = topo.Solver(NX, NY, fixed=cfg["fixed"], levels=LEVELS, precision=precision)
        if args.outer_fp64:
            s.set_outer_precision(0)
        u_d = torch.zeros_like(f_d)
        if host_io:
            x_h = torch.as_tensor(cfg["x"]).contiguous().pin_memory()
            f_h = torch.as_tensor(cfg["f"]).contiguous().pin_memory()
            u_h = torch.empty_like(f_h).pin_memory()

        def step():
            if host_io:  # the C-ABI call with host buffers: copies inside the call
                info = s.solve_host(x_h, f_h, u_h, tol=TOL)
            else:
                s.set_density(x_d)
                _, info = s.solve(f_d, u_d, tol=TOL)
            return info

        for _ in range(warmup):
            step()
        profile = profile_mask != 0
        if profile:
            s.set_profiling_mask(profile_mask)
            step()  # capture the instrumented graph outside the timed region
            s.set_profiling_mask(profile_mask)  # and restart the counters
        barrier()
        l0 = s.launch_count
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = 0
        res = 0.0
        solve_ms = 0.0
        e0.record()
        for _ in range(steps):
            info = step()
            iters += info.iterations
            res = max(res, info.rel_residual)
            solve_ms += info.wall_ms
        e1.record()
        barrier()
        ms = e0.elapsed_time(e1)
        launches = s.launch_count - l0
        prof = s.profile() if profile else None
        kinds = [s.profile_kernel(k) for k in range(len(topo.Solver.PROFILE_KINDS))] if profile else None
        s.close()
        return dict(ms=ms, iters=iters, res=res, launches=launches, prof=prof, kinds=kinds,
                    solve_ms=solve_ms)

    def batched_3d_run(steps=3, warmup=3, tune=True):
        """128x64x64 hex grid (1.6M DOFs, 5 levels), 8 unit point loads on the x = max face as one
        batched mixed solve per step (hierarchy build + PCG to 1e-8 for all 8) with the
        autotuner's smoother (damped Jacobi omega x nu, Chebyshev degree); DOF*iterations summed
        over the load cases."""
        from paper_1606_06201_gb300 import autotune
        c4 = W.random_field_3d(128, 64, 64, n_rhs=8)
        nfree4 = int(np.count_nonzero(c4["fixed"] == 0))
        x4 = torch.as_tensor(c4["x"], device=dev)
        f4 = torch.as_tensor(c4["f"], device=dev)
        t_tune = time.perf_counter()
        if tune:
            tuned = autotune.autotune(128, 64, 64, c4["fixed"], x4, f4, 5, precision=topo.MIXED,
                                      nrhs=8, tol=TOL, sweeps=(1, 2, 3), cheb_degrees=(1, 2, 3),
                                      reps=1)
        else:  # (--no-autotune: the setting the autotuner picks on this workload, for profiling)
            tuned = {"smoother": "jacobi", "omega": 0.6, "nu": 1, "rows": 0, "tried": 0}
        t_tune = time.perf_counter() - t_tune
        s4 = autotune.solver_for(tuned, 128, 64, 64, c4["fixed"], 5, precision=topo.MIXED, nrhs=8)
        u4 = torch.zeros_like(f4)
        for _ in range(warmup):
            s4.set_density(x4)
            s4.solve(f4, u4, tol=TOL)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = 0
        e0.record()
        for _ in range(steps):
            s4.set_density(x4)
            _, info4 = s4.solve(f4, u4, tol=TOL)
            iters += info4.iterations
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s4.close()
        return {"workload": "3d_hex_128x64x64_5lev_8_point_loads_batched", "free_dofs": nfree4,
                "nrhs": 8, "steps": steps, "ms_per_step": ms / steps,
                "iterations_per_solve": iters / steps,
                "value": 8 * nfree4 * iters / (ms * 1e-3), "unit": UNIT,
                "smoother": ("%s omega=%g nu1=nu2=%d (autotuned over %d settings in %.1f s, "
                             "outside the timed steps)" % (tuned["smoother"], tuned["omega"],
                                                          tuned["nu"], tuned["tried"], t_tune)),
                "precision": "FP32 V-cycle, FP64 CG recurrences and dots, outer operator in "
                             "float pairs (~48-bit)"}

    def err_vs_oracle(x, u, c, o):
        """Errors of a GPU run against the oracle's (exact solves): x in the max norm relative to
        max|x|, u in the 2-norm relative, compliance relative."""
        return {"x_max_rel": float(np.max(np.abs(x - o["x"])) / np.max(np.abs(o["x"]))),
                "u_rel": float(np.linalg.norm(u - o["u"]) / np.linalg.norm(o["u"])),
                "compliance_rel": float(abs(c - o["compliance"]) / abs(o["compliance"]))}

    def ip_oc_runs(nx, ny, volfrac, levels, jobs, with_inexact):
        """Example-2-shaped cantilever (V = volfrac m): IP (to tau_IP) and AOC (50 linear solves),
        FP64 and mixed, linear solves to 1e-8; each with its error against the oracle's run of
        the same problem (exact solves, Cholesky), whose wall time and cores are reported."""
        out = {}
        c2 = W.cantilever_2d(nx, ny, volfrac)
        f2 = torch.as_tensor(c2["f"], device=dev)
        gpu = {}
        for name, prec in (("fp64", topo.FP64), ("mixed", topo.MIXED)):
            ip = topo.IP(nx, ny, fixed=c2["fixed"], f=f2, V=c2["V"], xbar=1.0, levels=levels,
                         precision=prec, max_iter=1000)
            info = ip.run(topo.ip_options(cg_tol=1e-8, max_newton=50))
            u, x = ip.state()[:2]
            out["ip_" + name] = {"wall_s": info.wall_ms * 1e-3, "newton": info.newton,
                                 "ip_iters": info.ip_iters, "cg_iters": info.cg_iters,
                                 "feval": info.feval, "compliance": float(f2 @ u), "done": info.done}
            gpu["ip_" + name] = (x.cpu().numpy(), u.cpu().numpy(), float(f2 @ u))
            if prec == topo.MIXED:
                x_exact = x
            ip.close()
            oc = topo.OC(nx, ny, fixed=c2["fixed"], f=f2, V=c2["V"], xbar=1.0, levels=levels,
                         precision=prec)
            oc.init()
            oinfo = oc.run(topo.oc_options(max_feval=50, tau_oc=0.0, cg_tol0=1e-8,
                                           adaptive_tol=False))
            out["aoc_" + name] = {"wall_s": oinfo.wall_ms * 1e-3, "feval": oinfo.feval,
                                  "iters": oinfo.iters, "cg_iters": oinfo.cg_iters,
                                  "compliance": oinfo.compliance}
            gpu["aoc_" + name] = oc.x().cpu().numpy()
            oc.close()
        if with_inexact:
            # Sec. 8.1 settings (tab:IP): every PCG stopped at 1e-2 ("CG tol fixed"), or at 1e-2
            # halved at every barrier reduction ("CG tol decreasing"); mixed precision, to tau_IP
            x_ref = x_exact
            for name, fac in (("fixed", 1.0), ("decreasing", 0.5)):
                ip = topo.IP(nx, ny, fixed=c2["fixed"], f=f2, V=c2["V"], xbar=1.0, levels=levels,
                             precision=topo.MIXED, max_iter=1000)
                info = ip.run(topo.ip_options(cg_tol=1e-2, cg_tol_factor=fac, max_newton=500))
                u, x = ip.state()[:2]
                out["ip_mixed_tau_cg_1e-2_" + name] = {
                    "wall_s": info.wall_ms * 1e-3, "newton": info.newton, "ip_iters": info.ip_iters,
                    "cg_iters": info.cg_iters, "feval": info.feval,
                    "cg_iters_per_system": info.cg_iters / max(info.feval, 1),
                    "compliance": float(f2 @ u), "x_min": float(x.min()),
                    "max_abs_x_diff_vs_cg_tol_1e-8": float((x - x_ref).abs().max()),
                    "done": info.done}
                ip.close()
        # the oracle's runs (started before the GPU work, in spawned CPU processes)
        try:
            o_ip = jobs[0].get(timeout=max(1.0, ORACLE_DEADLINE_S - (time.perf_counter() - T_START)))
            o_oc = jobs[1].get(timeout=max(1.0, ORACLE_DEADLINE_S - (time.perf_counter() - T_START)))
        except Exception as exc:  # reported, not fatal for the GPU numbers
            out["oracle"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            return out
        for name in ("fp64", "mixed"):
            x, u, c = gpu["ip_" + name]
            out["ip_" + name]["err_vs_oracle"] = err_vs_oracle(x, u, c, o_ip)
            xo = gpu["aoc_" + name]
            out["aoc_" + name]["err_vs_oracle"] = {
                "x_max_rel": float(np.max(np.abs(xo - o_oc["x"])) / np.max(np.abs(o_oc["x"]))),
                "compliance_rel": float(abs(out["aoc_" + name]["compliance"] - o_oc["compliance"][-1])
                                        / abs(o_oc["compliance"][-1]))}
        out["oracle"] = {"kind": "oracle (scipy sparse assembly, banded Cholesky: exact solves)",
                         "cores": o_ip["cores"], "ip_wall_s": o_ip["wall_s"],
                         "ip_newton": o_ip["newton"], "ip_compliance": o_ip["compliance"],
                         "aoc_wall_s": o_oc["wall_s"], "aoc_feval": o_oc["feval"],
                         "aoc_compliance": o_oc["compliance"][-1]}
        return out

    def oc_accuracy_study(n_inf=5000):
        """Sec. 8.2-8.3 (tab:exact1, tab:exact2) on Example 1's problem 226 (the 64 x 64 square,
        left edge clamped, unit load at the right-edge midpoint, V = 0.5 m, xbar = 1): AOC runs
        stopped by Eq. (OCstop) at tau_OC = 1e-5, 1e-7, 1e-9 and after n_inf iterations (the
        paper's "-inf"), for the lower bounds 1e-7 and 1e-17; the pairwise 2-norm and max-norm
        differences of their x; and the IP at tau_IP = 1e-8 ... 1e-14 against the "-inf" OC
        solution with lower bound 1e-17.  FP64, linear solves to 1e-12 (the paper uses a direct
        solver here)."""
        cfg = W.cantilever_2d(64, 64, 0.5)
        f1 = torch.as_tensor(cfg["f"], device=dev)
        sols, meta = {}, {}
        for xlow in (1e-7, 1e-17):
            for tau in (1e-5, 1e-7, 1e-9, None):
                oc = topo.OC(64, 64, fixed=cfg["fixed"], f=f1, V=cfg["V"], xbar=1.0, levels=5,
                             precision=topo.FP64, max_iter=2000)
                oc.init()
                opts = topo.oc_options(variant=topo.OC_AOC, xlow=xlow,
                                       tau_oc=tau if tau else 0.0,
                                       max_feval=2 * n_inf,
                                       cg_tol0=1e-12, adaptive_tol=False)
                try:
                    info = oc.run(opts)
                    key = "%g/%s" % (xlow, "-inf" if tau is None else "%g" % tau)
                    sols[key] = oc.x().cpu().numpy()
                    meta[key] = {"iters": info.iters, "feval": info.feval, "cg_iters": info.cg_iters,
                                 "compliance": info.compliance, "wall_s": info.wall_ms * 1e-3,
                                 "status": info.status}
                except topo.TopoError as exc:
                    meta["%g/%s" % (xlow, tau)] = {"error": str(exc)}
                oc.close()
        keys = list(sols)
        pair = {a: {b: [float(np.linalg.norm(sols[a] - sols[b])),
                        float(np.max(np.abs(sols[a] - sols[b])))] for b in keys} for a in keys}
        ipres = {}
        ref = sols.get("1e-17/-inf")
        for tau_ip in (1e-8, 1e-10, 1e-12, 1e-14):
            ip = topo.IP(64, 64, fixed=cfg["fixed"], f=f1, V=cfg["V"], xbar=1.0, levels=5,
                         precision=topo.FP64, max_iter=5000)
            try:
                info = ip.run(topo.ip_options(tau_ip=tau_ip, cg_tol=1e-12, max_newton=500))
                x = ip.state()[1].cpu().numpy()
                ipres["%g" % tau_ip] = {"newton": info.newton, "ip_iters": info.ip_iters,
                                        "done": info.done}
                if ref is not None:
                    ipres["%g" % tau_ip].update(err_2=float(np.linalg.norm(x - ref)),
                                                err_max=float(np.max(np.abs(x - ref))))
            except topo.TopoError as exc:
                ipres["%g" % tau_ip] = {"error": str(exc)}
            ip.close()
        return {"study": "Sec. 8.2 tab:exact1 / Sec. 8.3 tab:exact2 on problem 226 (64 x 64)",
                "oc_runs": meta, "oc_pairwise_2norm_maxnorm": pair, "ip_vs_oc_inf": ipres}

    def simp_example4_runs():
        """Sec. 9.1 Example 4 shape 427: the Example 2 beam on 256 x 128 (5 levels), xbar = 3,
        SIMP p = 3 with the Manhattan density filter r_min = 2, V = 0.4 m, mixed precision, CG
        capped at 1000 iterations (Sec. 8.1).  The paper's tau_CG = 1e-2 and a tight 1e-6, each
        bounded to 250 Newton steps; Newton steps per barrier value as in tab:202."""
        out = {}
        c4 = W.cantilever_2d(256, 128, 0.4)
        f4 = torch.as_tensor(c4["f"], device=dev)
        for tol in (1e-2, 1e-6):
            ip = topo.IP(256, 128, fixed=c4["fixed"], f=f4, V=c4["V"], xbar=3.0, levels=5,
                         precision=topo.MIXED, max_iter=1000, simp=(3.0, 2.0))
            opts = topo.ip_options(cg_tol=tol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ip.init(opts)
            per_barrier, last, info = [0], 0, None
            for _ in range(250):
                info = ip.step(opts)
                per_barrier[-1] += 1
                if info.ip_iters > last:
                    last = info.ip_iters
                    per_barrier.append(0)
                if info.done:
                    break
            wall = time.perf_counter() - t0
            u, x = ip.state()[:2]
            out["tau_cg_%g" % tol] = {
                "wall_s": wall, "newton": info.newton, "ip_iters": info.ip_iters,
                "done": info.done, "feval": info.feval, "cg_iters": info.cg_iters,
                "cg_iters_per_system": info.cg_iters / max(info.feval, 1),
                "newton_per_barrier": per_barrier[:12],
                "compliance": float(f4 @ u), "volume_rel_err": float((x.sum() - c4["V"]) / c4["V"])}
            ip.close()
        return out

    if args.only == "ip":  # profiling aid: the mixed IP run on 512x256, steps = Newton budget
        c2 = W.cantilever_2d(512, 256, 0.4)
        f2 = torch.as_tensor(c2["f"], device=dev)
        ip = topo.IP(512, 256, fixed=c2["fixed"], f=f2, V=c2["V"], xbar=1.0, levels=6,
                     precision=topo.MIXED, max_iter=1000)
        info = ip.run(topo.ip_options(cg_tol=1e-8, max_newton=args.steps))
        print("only=ip wall_ms=%.3f newton=%d cg_iters=%d" % (info.wall_ms, info.newton,
                                                              info.cg_iters))
        ip.close()
        return 0
    if args.only == "simp":  # profiling aid: Example 4 shape 427 (SIMP), steps = Newton budget
        c4 = W.cantilever_2d(256, 128, 0.4)
        f4 = torch.as_tensor(c4["f"], device=dev)
        ip = topo.IP(256, 128, fixed=c4["fixed"], f=f4, V=c4["V"], xbar=3.0, levels=5,
                     precision=topo.MIXED, max_iter=1000, simp=(3.0, 2.0))
        info = ip.run(topo.ip_options(cg_tol=1e-6, max_newton=args.steps))
        print("only=simp wall_ms=%.3f newton=%d cg_iters=%d" % (info.wall_ms, info.newton,
                                                                info.cg_iters))
        ip.close()
        return 0
    if args.only == "oc_accuracy":
        print(json.dumps(oc_accuracy_study()), flush=True)
        return 0
    if args.only == "batched3d":
        r = batched_3d_run(args.steps, args.warmup, tune=not args.no_autotune)
        print("only=batched3d ms_per_step=%.3f iterations=%.1f" % (r["ms_per_step"],
                                                                  r["iterations_per_solve"]))
        return 0
    if args.only:
        r = run(topo.MIXED if args.only == "mixed" else topo.FP64, args.steps, args.warmup)
        print("only=%s ms_per_step=%.3f iterations=%d launches=%d" % (
            args.only, r["ms"] / args.steps, r["iters"], r["launches"]), flush=True)
        return 0
    # warm-up + timed steps: mixed (headline), FP64, end-to-end, then the outer operators' live
    # launch times in runs of their own
    with ClockSampler(dev.index) as clk:
        # headline and FP64 without event nodes: an event pair around the outer operator in every
        # CG iteration made the 2048 x 1024 mixed step 4.2% longer (4.72 against 4.53 ms)
        mixed = run(topo.MIXED, args.steps, args.warmup)
        fp64 = run(topo.FP64, args.steps, args.warmup)
        e2e = run(topo.MIXED, args.steps, args.warmup, host_io=True)
        # the same solves with event pairs around the outer operator (its live launch time)
        mixed_oprun = run(topo.MIXED, max(1, min(args.steps, 10)), args.warmup, profile_mask=1)
        fp64_oprun = run(topo.FP64, max(1, min(args.steps, 5)), args.warmup, profile_mask=1)
        # separate run with every kind profiled, for the per-kernel and per-part times (its own
        # step time is longer by the extra event nodes and is not reported)
        kinds_run = run(topo.MIXED, max(1, min(args.steps, 5)), 3,
                        profile_mask=(1 << len(topo.Solver.PROFILE_KINDS)) - 1)

    def gather_max(v):
        return max_over_ranks(v, ws, dev)

    ms_mixed = gather_max(mixed["ms"])
    ms_fp64 = gather_max(fp64["ms"])
    ms_e2e = gather_max(e2e["ms"])
    value = ws * nfree * mixed["iters"] / (ms_mixed * 1e-3)
    line = None
    if rank == 0:
        m, n = NX * NY, cfg["f"].size
        nodes = (NX + 1) * (NY + 1)
        op_ms, op_cnt = mixed_oprun["prof"]
        op_avg_ms = op_ms / op_cnt if op_cnt else float("nan")
        # the method's bytes of one K(x) p (Sec. 8(d): p and q at 16 B per node each, x at 8 B per
        # element as a float pair, the fixed-DOF mask at 1 B per DOF)
        alg_bytes = 8.0 * m + 16.0 * n + 1.0 * n
        hbm_peak = _measured_hbm_gbs()
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = _measured_sm_max_mhz()
        fp64_peak, fp32_peak = derived_peaks(sm_count, sm_mhz)
        peak_src = ("derived, not measured: %d SMs (cudaDeviceProp.multiProcessorCount) x %s x "
                    "%.0f MHz (maximum SM clock)")
        if args.outer_fp64:
            ops_per_launch = OPS_PER_ELEM * m + OPS_PER_NODE * nodes
            kname = "k_q1_sweep<double,0,1> (outer FP64 operator q = K(x) p, fused p^T q)"
            issue = {"bound": "alu", "achieved": ops_per_launch / (op_avg_ms * 1e-3) / 1e12,
                     "peak": fp64_peak, "unit": "T FP64-op/s",
                     "peak_source": peak_src % (sm_count, "2 FP64 issue slots", sm_mhz),
                     "algorithmic_ops_per_launch": ops_per_launch}
            traffic = OPERATOR_DRAM_BYTES
        else:
            ops_per_launch = DF_OPS_PER_ELEM * m + DF_OPS_PER_NODE * nodes
            kname = "k_q1_sweep_df (outer operator q = K(x) p in float pairs, fused p^T q)"
            issue = {"bound": "alu", "achieved": ops_per_launch / (op_avg_ms * 1e-3) / 1e12,
                     "peak": fp32_peak, "unit": "T FP32-op/s",
                     "peak_source": peak_src % (sm_count, "128 FP32 lanes", sm_mhz),
                     "algorithmic_ops_per_launch": ops_per_launch,
                     "note": "operations of the pair arithmetic as written (296 FP32 ops per "
                             "element + 72 per node), against the derived FP32 issue rate"}
            traffic = DF_OPERATOR_DRAM_BYTES
        issue["frac"] = issue["achieved"] / issue["peak"]
        achieved = alg_bytes / (op_avg_ms * 1e-3) / 1e9
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
                "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": alg_bytes,
                "bytes_model": "8 B per element (x) + 16 B per DOF (p, q) + 1 B per DOF (mask)",
                "avg_launch_ms": op_avg_ms, "launches_timed": op_cnt,
                "launch_timing": "CUDA event pairs around every launch on the solver's stream, in "
                                 "a run of the same solve separate from the headline's timed "
                                 "region (the event nodes lengthen the step by about 4%)",
                "issue_view": issue}
        f_ms, f_cnt = fp64_oprun["prof"]
        fp64_op = None
        if f_cnt:
            f_avg = f_ms / f_cnt
            f_ops = OPS_PER_ELEM * m + OPS_PER_NODE * nodes
            fp64_op = {"kernel": "k_q1_sweep<double,0,1> (FP64 solver's outer operator)",
                       "bound": "alu", "achieved": f_ops / (f_avg * 1e-3) / 1e12,
                       "peak": fp64_peak, "unit": "T FP64-op/s",
                       "frac": f_ops / (f_avg * 1e-3) / 1e12 / fp64_peak,
                       "peak_source": peak_src % (sm_count, "2 FP64 issue slots", sm_mhz),
                       "traffic": OPERATOR_DRAM_BYTES, "avg_launch_ms": f_avg,
                       "launches_timed": f_cnt,
                       "hbm_view": {"achieved": alg_bytes / (f_avg * 1e-3) / 1e9,
                                    "peak": hbm_peak, "unit": "GB/s",
                                    "frac": alg_bytes / (f_avg * 1e-3) / 1e9 / hbm_peak}}
        # HBM-bound kernels of the FP32 V-cycle on the finest level, timed live like the operator:
        # algorithmic bytes per launch (FP32 vectors of n DOFs, FP32 densities of m elements, the
        # byte mask) / average launch time, against the measured copy bandwidth.
        nc = ((NX // 2) + 1) * ((NY // 2) + 1) * 2
        hbm_bytes = {
            "fine_smoothing_sweep": ("k_q1w<float,4,0>: first two Jacobi sweeps from zero, "
                                     "z = omega D^-1 b formed on the fly, diag from x",
                                     4.0 * m + 9.0 * n),
            "fine_residual": (("k_q1w_resrestrict<float>: b_c = P^T (b - K(x) z) in one pass, the "
                               "residual not stored", 4.0 * m + 9.0 * n + 5.0 * nc)
                              if kinds_run["kinds"] and not kinds_run["kinds"][3][1] else
                              ("k_q1w<float,1,0>: r = b - K(x) z", 4.0 * m + 13.0 * n)),
            "fine_restriction": ("k_restrict<2,float>: b_c = P^T r", 4.0 * n + 5.0 * nc),
            "fine_prolongation": ("k_q1w<float,5,0>: v = z + P z_c formed on the fly, then "
                                  "one Jacobi sweep", 4.0 * m + 13.0 * n + 4.0 * nc),
        }
        hbm_kernels = []
        for k, key in enumerate(topo.Solver.PROFILE_KINDS):
            if key not in hbm_bytes or not kinds_run["kinds"]:
                continue
            kms, kcnt = kinds_run["kinds"][k]
            if not kcnt:
                continue
            desc, nbytes = hbm_bytes[key]
            avg = kms / kcnt
            gbs = nbytes / (avg * 1e-3) / 1e9
            hbm_kernels.append({"kernel": desc, "bound": "hbm", "bytes_per_launch": nbytes,
                                "avg_launch_us": avg * 1e3, "achieved": gbs, "peak": hbm_peak,
                                "unit": "GB/s", "frac": gbs / hbm_peak, "launches_timed": kcnt})
        breakdown = None
        if kinds_run["kinds"]:
            avg = {key: (ms * 1e3 / cnt if cnt else None)
                   for key, (ms, cnt) in zip(topo.Solver.PROFILE_KINDS, kinds_run["kinds"])}
            step_us = ms_mixed * 1e3 / args.steps
            breakdown = {"outer_operator": avg["outer_operator"], "vcycle": avg["vcycle"],
                         "vcycle_finest_level": (avg["vcycle"] - avg["vcycle_levels_ge1"])
                         if avg["vcycle"] and avg["vcycle_levels_ge1"] else None,
                         "vcycle_first_coarse_level": (avg["vcycle_levels_ge1"] - avg["vcycle_levels_ge2"])
                         if avg["vcycle_levels_ge1"] and avg["vcycle_levels_ge2"] else None,
                         "vcycle_levels_ge2": avg["vcycle_levels_ge2"],
                         # per coarse level (levels >= j minus levels >= j + 1); the fused deep
                         # part counts as one span from its first level down
                         "vcycle_per_level": {
                             "level_%d" % j: (avg["vcycle_levels_ge%d" % j]
                                              - (avg["vcycle_levels_ge%d" % (j + 1)] or 0.0))
                             for j in range(2, 6) if avg["vcycle_levels_ge%d" % j]},
                         "vcycle_levels_ge6": avg["vcycle_levels_ge6"],
                         "unit": "us per CG iteration (live CUDA events, mixed solver, separate fully "
                                 "profiled run)",
                         "step_us": step_us}
        bi = 8 * (m + n)
        bo = 8 * n
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle + f64 CG" + (" (f64 outer operator)" if args.outer_fp64 else
                                                 " (outer operator in f32 pairs, ~48-bit)"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "levels": LEVELS, "tol": TOL,
                       "free_dofs": nfree, "smoother": "damped Jacobi omega=0.6 nu1=nu2=2",
                       "step": "hierarchy build + PCG solve", "parallelism": "replicas" if ws > 1 else "1 GPU",
                       "l2": "working set > L2 (vectors 33.6 MB each, ~0.5 GB resident)"},
            "iterations_per_solve": mixed["iters"] / args.steps, "final_rel_residual": mixed["res"],
            # the step split into the PCG solve (its own device events) and the rest (hierarchy
            # build and host gaps); the DOF*iterations rate over the solve alone beside it
            "build_ms_per_step": (mixed["ms"] - mixed["solve_ms"]) / args.steps,
            "solve_ms_per_step": mixed["solve_ms"] / args.steps,
            "value_solve_only": ws * nfree * mixed["iters"] / (mixed["solve_ms"] * 1e-3),
            "fp64": {"value": ws * nfree * fp64["iters"] / (ms_fp64 * 1e-3), "unit": UNIT,
                     "ms_per_step": ms_fp64 / args.steps, "iterations_per_solve": fp64["iters"] / args.steps,
                     "build_ms_per_step": (fp64["ms"] - fp64["solve_ms"]) / args.steps,
                     "operator_roofline": fp64_op},
            "roofline": roof,
            "hbm_kernels": hbm_kernels,
            "iteration_breakdown": breakdown,
            "cpu_baseline": cpu,
            "e2e": {"value": ws * nfree * e2e["iters"] / (ms_e2e * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
            "gpu_launches": mixed["launches"],
            "clocks": clk.summary(),
        }
        if not args.no_ip:
            try:
                line["batched_3d_128x64x64"] = batched_3d_run()
            except topo.TopoError as exc:
                line["batched_3d_128x64x64"] = {"error": str(exc)}
            try:
                line["ip_oc_64x32"] = ip_oc_runs(64, 32, 0.5, 3, oracle_jobs["c1"], False)
            except topo.TopoError as exc:  # reported, not fatal for the headline measurement
                line["ip_oc_64x32"] = {"error": str(exc)}
            try:
                line["ip_oc_512x256"] = ip_oc_runs(512, 256, 0.4, 6, oracle_jobs["c2"], True)
            except topo.TopoError as exc:
                line["ip_oc_512x256"] = {"error": str(exc)}
            try:
                line["simp_example4_256x128"] = simp_example4_runs()
            except topo.TopoError as exc:
                line["simp_example4_256x128"] = {"error": str(exc)}
        print(json.dumps(line), flush=True)
    if oracle_pool is not None:
        oracle_pool.terminate()
        oracle_pool.join()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
