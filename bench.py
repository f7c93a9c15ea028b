"""Benchmark: mixed-precision perturbed DIRK steps of the 3D heat equation on B300.

One step = one pass of the whole stage loop (stage right-hand sides, FP64
operator, low-precision block-Jacobi CG solve, FP64 explicit correction and
true residual, FP64 update) over the workload below.

Default workload (heat256): kappa = 1 on the 256^3 interior grid, u0 = unit
sine mode + 32 seeded random low modes (amplitudes N(0, 0.1^2)), the
two-stage L-stable SDIRK split for mixed precision (implicit stages in low
precision, explicit history and the update in FP64), dt = 1e-3, FP32
storage/arithmetic CG with x-line block-Jacobi (8), tol_rel 1e-6; FP64
correction and update.  The plain FP64 DIRK step of the same problem is
timed beside it; both errors against the exact solution are reported (they
agree to 1e-4 relative: matched error).  --workload heat256-4s3pB runs
Grant's method 4s3pB instead, heat256-f16 FP16 storage.

Metric: DOF*steps/s = n^3 * steps / seconds (device time, CUDA events on the
library's stream), inputs resident in HBM, working set (> 1.5 GB) larger than
L2.  Usage:
    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica on its own GPU (the
single problem does not shard): value = total DOF*steps over all ranks / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "DOF*steps/s"
# tol: solver tolerance of the mixed path; tol64: of the plain FP64 path.  Each
# is the loosest tolerance (of 1e-2, 3e-3, 1e-3, 3e-4, 1e-4, 1e-5) whose error
# against the exact solution after 23 steps stays within 1.05x that of an
# exact solve (profiles/heat256_tolerance_sweep.md); 1e-3 is also the
# tolerance of the paper's accuracy study (Sec. 5.4).
WORKLOADS = {
    "heat256": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-3, tol64=3e-4, storage="f32"),
    "heat256-tight": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-6, tol64=1e-6, storage="f32"),
    "heat256-4s3pB": dict(n=256, kappa=1.0, tableau="4s3pB", dt=1e-3, bs=8, tol=1e-6, tol64=1e-6, storage="f32"),
    "heat256-f16": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-3, tol64=3e-4, storage="f16"),
    "heat128": dict(n=128, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-3, tol64=1e-4, storage="f32"),
    # the fast-diagonalization preconditioner (tensor-core mode products) in place of block-Jacobi
    "heat256-fdm": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-3, tol64=3e-4, storage="f32",
                        precond="fdm"),
}
MATCH = 1.05  # matched error: within 5 % of the exact solve's error
# FP64-pipe instructions per DOF of the heat FP64 kernels (counted from the
# source: heat_apply_f64 = 5 DADD neighbour sum + 2 DFMA for d x + o nb + f,
# one DFMA for ||g||^2, and one DMNMX for ||g||_inf with FP16 storage only)
# and the FP64 peak in lane-operations per second: the nominal 1.25 TFLOP/s
# of the part is 2 FP64 FMA lanes per SM per clock, x 148 SMs x 2.032 GHz
# (maximum SM clock).
FP64_ALU = {"op_apply_f64": 8, "correct_f64": 7}
FP64_ALU_MAXNORM = {"f16": 1}  # the max-norm DMNMX, by storage
FP64_PEAK_GINSTR = 2 * 148 * 2.032
HBM_FALLBACK_GBS = 6400.0


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def ncu_traffic(kernel, workload):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None
    when there is none or the kernel sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)[workload]
        h = hashlib.sha256()
        for name in d.get("sources", ("rk_heat.cuh", "rk_tiled.cuh")):
            with open(os.path.join(ROOT, "paper_2412_16638_b300", "csrc", name), "rb") as f:
                h.update(f.read())
        sha = h.hexdigest()[:16]
        if d.get("kernel_src_sha256_16") != sha:
            return None
        return float(d[kernel]["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.lines, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def closed_form(n, kappa, dt, steps, tab, modes):
    """Exact fully discrete solution sum_m a_m R(dt lambda_m)^steps phi_m and the
    continuous solution sum_m a_m exp(lambda^c_m t) phi_m (written out here
    from the sine-mode eigenvalues; not the library, not the oracle)."""
    A = np.array(tab[0]) + np.array(tab[1])
    b = np.array(tab[2])
    q = len(b)
    h = 1.0 / (n + 1)
    disc = np.zeros(n ** 3)
    cont = np.zeros(n ** 3)
    for a, kx, ky, kz in modes:
        lam = -4.0 * kappa / h ** 2 * sum(math.sin(k * math.pi * h / 2) ** 2 for k in (kx, ky, kz))
        z = dt * lam
        R = 1.0 + z * (b @ np.linalg.solve(np.eye(q) - z * A, np.ones(q)))
        phi = synth.sine_mode(n, kx, ky, kz)
        disc += a * R ** steps * phi
        cont += a * math.exp(-math.pi ** 2 * kappa * (kx * kx + ky * ky + kz * kz) * dt * steps) * phi
    return disc, cont


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_step_seconds(cfg, iters_per_step):
    """Oracle (float64 numpy, one thread) cost of one step of the workload.

    Bounded sample: after the oracle's setup (excluded, as for the GPU), one
    step is run with every stage solve capped at 1 CG iteration and once with
    2; the difference gives the cost per iteration and the remainder the
    per-step cost outside the iterations; the step time is extrapolated to
    `iters_per_step` iterations.  Returns (seconds per step, sample text)."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:  # numpy's element-wise kernels are single-threaded anyway
        import contextlib

        def threadpool_limits(_):
            return contextlib.nullcontext()

    from oracle import dirk, operators, tableau

    with threadpool_limits(1):
        n = cfg["n"]
        op = operators.HeatOperator(n, cfg["kappa"])
        tab = tableau.get(cfg["tableau"])
        u0 = synth.heat_modes(seed=0).evaluate(n)
        solver = dirk.Solver("cg", bs=cfg["bs"], tol_rel=cfg["tol"], max_iter=1, precond=cfg.get("precond", "bj"))
        shifts = sorted({cfg["dt"] * a for a in np.diag(tab[1]) if a != 0.0})
        for s in shifts:  # preconditioner setup, untimed
            solver.solve(op, s, np.zeros(n ** 3))
        nsolves = int(np.count_nonzero(np.diag(tab[1])))
        times = {}
        for cap in (1, 2):
            solver.max_iter = cap
            t0 = time.perf_counter()
            dirk.rk_step(u0, cfg["dt"], tab, op, solver)
            times[cap] = time.perf_counter() - t0
    per_iter = max((times[2] - times[1]) / nsolves, 1e-9)
    fixed = max(times[1] - nsolves * per_iter, 0.0)
    sample = ("oracle float64 numpy, 1 thread: one %d^3 step with each of the %d stage solves capped at 1 and "
              "at 2 CG iterations (%.1f s, %.1f s); per-iteration %.3f s and per-step %.2f s extrapolated to %.1f "
              "iterations per step" % (n, nsolves, times[1], times[2], per_iter, fixed, iters_per_step))
    return fixed + iters_per_step * per_iter, sample


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    ipath = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(ipath) as f:
            iters = float(json.load(f)[args.workload]["iters_per_step"])
    except Exception:
        iters = 60.0
    t_step, sample = oracle_step_seconds(cfg, iters)
    N = cfg["n"] ** 3
    value = N / t_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF*steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, cfg),
        "cpu_baseline": {"value": value, "unit": "DOF*steps/s", "cores": 1, "kind": "oracle",
                         "sample": sample + " (iterations per step from profiles/traffic.json)"},
        "e2e": {"value": value, "unit": "DOF*steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(name, cfg):
    return {"workload": name, "grid": "%d^3" % cfg["n"], "dof": cfg["n"] ** 3, "kappa": cfg["kappa"],
            "tableau": cfg["tableau"], "dt": cfg["dt"], "krylov": "cg", "bj_block": cfg["bs"],
            "precond": cfg.get("precond", "bj"), "precond_fp64": "bj",
            "initial_guess": "previous step's stage solution" if cfg.get("warm") else "zero",
            "tol_rel": cfg["tol"], "tol_rel_fp64": cfg["tol64"], "storage": cfg["storage"], "arith": "f32",
            "solution": "f32", "high_precision": "f64",
            "u0": "sine mode + 32 random modes (seed 0)", "l2": "working set > L2 (no flush needed)"}


def run_batch(args):
    """Batched workload: 512 independent heat problems (n uniform in 16..64,
    kappa log-uniform in [0.1, 10], amplitude * sine mode), SDIRK2, dt 1e-3,
    FP32 solves / FP64 corrections, --batch-steps steps in persistent
    graph-captured launches.  Value = sum n^3 * steps / device seconds."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_16638_b300 as rk

    torch.cuda.set_device(0)
    probs = synth.batch_problems(512, seed=0)
    tab = rk.tableaux.get("sdirk2")
    dt = 1e-3
    ps = [rk.Problem(rk.problem_desc(n=pr.n, kappa=pr.kappa),
                     rk.solver_desc(bj_block=8, tol_rel=1e-6, storage="f32", max_iter=2000, correct=1),
                     tableau=tab, u0=pr.amplitude * synth.sine_mode(pr.n)) for pr in probs]
    handles = [p.h for p in ps]
    rk.rk_integrate_batch(handles, dt, 1)  # warm-up (autotune)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = rk.rk_integrate_batch(handles, dt, args.batch_steps)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    dof = sum(pr.n ** 3 for pr in probs)
    line = {"metric": METRIC, "workload": "batch512", "value": dof * args.batch_steps / secs,
            "unit": "DOF*steps/s", "problems": 512, "total_dof": dof, "steps": args.batch_steps,
            "seconds": secs, "iters_per_solve": st.iters_total / max(st.solves, 1),
            "true_res_max": st.true_res, "config": {"tableau": "sdirk2", "dt": dt, "storage": "f32",
                                                    "bj_block": 8, "tol_rel": 1e-6, "n": "uniform 16..64",
                                                    "kappa": "log-uniform [0.1, 10]"}}
    for p in ps:
        p.close()
    print(json.dumps(line))
    return 0


def run_advdiff(args):
    """Advection-diffusion workload (variable kappa, CSR, GMRES(30) + block-
    Jacobi 8, DIRK3, dt 5e-4, tol 1e-8): the mixed step (FP32 GMRES, FP64
    corrections) against the plain FP64 step on the same problem, both timed
    with CUDA events over --steps steps after --warmup; errors against an FP64
    run solved to 1e-12 (no closed form for variable kappa)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_16638_b300 as rk

    torch.cuda.set_device(0)
    n, dt, vel = args.advdiff, 5e-4, (1.0, 0.5, 0.25)
    N = n ** 3
    kap = synth.kappa_field(n, seed=0)
    u0 = synth.gaussian_bump(n)
    tab = rk.tableaux.get("dirk3")
    stream = torch.cuda.current_stream()

    def make(storage, tol, correct, basis=None):
        kw = {} if basis is None else {"basis": basis}
        return rk.Problem(rk.problem_desc(op=rk.RK_OP_ADVDIFF_CSR, n=n, kappa_field=kap, vel=vel),
                          rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=tol,
                                         storage=storage, correct=correct, max_iter=3000, **kw),
                          tableau=tab, u0=u0, stream=stream.cuda_stream)

    def timed(p, prof=False):
        rk.rk_integrate(p.h, dt, args.warmup)
        if prof:
            rk.rk_profile(p.h, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = rk.rk_integrate(p.h, dt, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        out = (e0.elapsed_time(e1) / 1e3, st)
        if prof:
            out += rk.rk_profile_read(p.h)
        return out

    with make("f64", 1e-12, 0) as q:
        rk.rk_integrate(q.h, dt, args.warmup + args.steps)
        ref = q.state()
    variants = {"mixed_f32": ("f32", 1e-8, 1, None), "fp64_plain": ("f64", 1e-8, 0, None)}
    if args.advdiff_basis:
        variants["mixed_f32_basis_" + args.advdiff_basis] = ("f32", 1e-8, 1, args.advdiff_basis)
    res = {}
    peak, peak_kind = measured_peaks()
    for name, (storage, tol, corr, basis) in variants.items():
        with make(storage, tol, corr, basis) as p:
            secs, st, prof, launches = timed(p, prof=True)
            u = p.state()
        kern = {k: {"launches": v["launches"], "avg_us": round(1e3 * v["ms_total"] / max(v["launches"], 1), 2),
                    "GBps": round(v["bytes_total"] / max(v["ms_total"], 1e-9) / 1e6, 1),
                    "share": round(v["ms_total"] / sum(x["ms_total"] for x in prof.values()), 4)}
                for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms_total"])}
        dom, d = max(prof.items(), key=lambda kv: kv[1]["ms_total"])
        achieved = d["bytes_total"] / (d["ms_total"] / 1e3) / 1e9
        res[name] = {"value": N * args.steps / secs, "ms_per_step": 1e3 * secs / args.steps,
                     "iters_per_solve": st.iters_total / max(st.solves, 1), "err_vs_fp64_tight": rel(u, ref),
                     "gpu_launches": launches,
                     "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                                  "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind},
                     "kernels": kern}
    line = {"metric": METRIC, "workload": "advdiff%d" % n, "unit": "DOF*steps/s", "steps": args.steps,
            "warmup": args.warmup, "data": "synthetic",
            "config": {"grid": "%d^3" % n, "kappa": "exp(Gaussian field, sigma 0.5, l 0.1), seed 0",
                       "vel": vel, "tableau": "dirk3", "dt": dt, "krylov": "gmres(30)", "bj_block": 8,
                       "tol_rel": 1e-8, "u0": "Gaussian bump"},
            "variants": res,
            "speedup_vs_fp64": res["mixed_f32"]["value"] / res["fp64_plain"]["value"]}
    print(json.dumps(line))
    return 0


def run_paper_sweep(args):
    """Error at T = 0.1 against the analytic solution for the paper's two test
    problems (Sec. 5.2) over tau = 1/10 .. 1/1280 (Fig. CombinedErrors), FP32
    mixed precision (perturbed step, FP64 corrections) vs plain FP64.  Heat
    (Sec. 5.2.1): u_t = Lap u + g, g the sine mode, u(0) = 0,
    u_a = g (1 - e^{-3 pi^2 t}) / (3 pi^2); FP32 CG with the fast-diagonalization
    preconditioner at tol 1e-3 and 1e-6, FP64 CG with block-Jacobi at tol 1e-3
    and 1e-10 (the paper's FP64 solver is exact in one iteration).  Advection
    (Sec. 5.2.2): periodic, beta = (1,1,1), the Gaussian bump, exact solution
    the bump translated by beta t; GMRES(30) + block-Jacobi at tol 1e-3 in both
    precisions, for tau <= 1/80 (block-Jacobi GMRES stalls beyond: the paper
    preconditions advection with the complex fast diagonalization)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_16638_b300 as rk

    torch.cuda.set_device(0)
    T = 0.1
    taus = [1.0 / m for m in (10, 20, 40, 80, 160, 320, 640, 1280)]
    out = {}
    for problem in args.paper_sweep.split(","):
        heat = problem == "heat"
        n = args.paper_n or (256 if heat else 200)
        methods = ["midpoint1", "4s3pB", "4s3pC"] + ([] if heat else ["4s3pA"])
        variants = ([("f32", 1e-3), ("f32", 1e-6), ("f64", 1e-3), ("f64", 1e-10)] if heat
                    else [("f32", 1e-3), ("f64", 1e-3)])
        if heat:
            g = synth.sine_mode(n)
            exact = g * (1.0 - math.exp(-3.0 * math.pi ** 2 * T)) / (3.0 * math.pi ** 2)
            u0 = np.zeros(n ** 3)
            desc = rk.problem_desc(n=n, kappa=1.0, source=g)
        else:
            beta = (1.0, 1.0, 1.0)
            x, y, z = synth.periodic_coords(n)
            d2 = sum(((c - 0.5 - T * b + 0.5) % 1.0 - 0.5) ** 2 for c, b in zip((x, y, z), beta))
            exact = np.exp(-100.0 * d2).ravel()
            u0 = synth.gaussian_bump_periodic(n)
            desc = rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=n, vel=beta)
        rows = []
        for name in methods:
            tab = rk.tableaux.get(name)
            for tau in (taus if heat else [t for t in taus if t <= 1.0 / 80]):
                steps = int(round(T / tau))
                row = {"method": name, "tau": tau, "steps": steps}
                for prec, tol in variants:
                    key = "%s_tol%g" % (prec, tol)
                    if heat:
                        sol = rk.solver_desc(tol_rel=tol, storage=prec, max_iter=3000, correct=1 if prec == "f32" else 0,
                                             precond="fdm" if prec == "f32" else "bj", bj_block=8)
                    else:
                        sol = rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=tol,
                                             storage=prec, max_iter=1000, correct=1 if prec == "f32" else 0)
                    with rk.Problem(desc, sol, tableau=tab, u0=u0) as p:
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        try:
                            st = rk.rk_integrate(p.h, tau, steps, allow_not_converged=True)
                            u = p.state()
                            err = rel(u, exact) if np.all(np.isfinite(u)) else float("inf")
                            row[key] = {"err": err, "iters_per_solve": st.iters_total / max(st.solves, 1),
                                        "not_converged": st.not_converged,
                                        "ms_per_step": 1e3 * (time.perf_counter() - t0) / steps}
                        except rk.RKError as e:
                            row[key] = {"err": None, "status": e.status}
                rows.append(row)
        out[problem] = {"n": n, "rows": rows}
    print(json.dumps({"paper_sweep": out, "T": T, "data": "synthetic",
                      "note": "errors are relative L2 against the analytic solution at T"}))
    return 0


def run_serve(args):
    """Serving workload: Poisson arrivals (200 jobs/s) of --serve jobs, n in
    {32, 64, 96, 128, 192}, tableau in {midpoint + 1 correction, SDIRK2,
    DIRK3}, storage in {FP32, FP16}, 10..200 steps, kappa log-uniform in
    [0.1, 10], dt 1e-3, 120 GB budget.  Reports p50/p99 latency (submit to
    finish), aggregate DOF*steps/s over the makespan."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_16638_b300 as rk

    torch.cuda.set_device(0)
    jobs = synth.serve_jobs(args.serve, seed=0)
    srv = rk.rk_server_create(120 << 30, args.serve_slots)
    prepared = []
    for jb in jobs:
        d = rk.problem_desc(n=jb.n, kappa=jb.kappa)
        sol = rk.solver_desc(bj_block=8, tol_rel=1e-6 if jb.storage == "f32" else 1e-3, storage=jb.storage,
                             max_iter=2000, correct=1)
        prepared.append((jb, d, sol, rk.tableaux.get(jb.tableau), jb.amplitude * synth.sine_mode(jb.n)))
    t0 = time.perf_counter()
    ids = []
    for jb, d, sol, tab, u0 in prepared:
        delay = jb.arrival - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(rk.rk_submit_job(srv, d, sol, *tab, u0, 1e-3, jb.steps))
    lats, service, failed = [], [], {}
    work = 0
    for jid, (jb, *_rest) in zip(ids, prepared):
        try:
            st, lat = rk.rk_wait_job(srv, jid, None, allow_not_converged=True)
            lats.append(lat)
            service.append(st.seconds)
            work += jb.n ** 3 * jb.steps
        except rk.RKError as e:
            # a job that diverged (non-finite state) is reported, not timed
            key = "%s/%s/n%d: status %d" % (jb.tableau, jb.storage, jb.n, e.status)
            failed[key] = failed.get(key, 0) + 1
    makespan = time.perf_counter() - t0
    rk.rk_server_destroy(srv)
    line = {"metric": METRIC, "workload": "serve", "jobs": len(jobs), "value": work / makespan,
            "unit": "DOF*steps/s", "makespan_s": makespan,
            "latency_p50_s": float(np.percentile(lats, 50)), "latency_p99_s": float(np.percentile(lats, 99)),
            "service_p50_s": float(np.percentile(service, 50)), "service_p99_s": float(np.percentile(service, 99)),
            "completed": len(lats), "failed": failed,
            "config": {"arrival_rate_per_s": 200, "slots": args.serve_slots, "budget_bytes": 120 << 30,
                       "sizes": [32, 64, 96, 128, 192], "tableaux": ["midpoint1", "sdirk2", "dirk3"],
                       "storage": ["f32", "f16"], "steps": "uniform 10..200", "dt": 1e-3}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heat256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-fdm", action="store_true",
                    help="skip the fast-diagonalization variant of a block-Jacobi workload")
    ap.add_argument("--bs", type=int, default=0, help="override the block-Jacobi block size")
    ap.add_argument("--tol", type=float, default=0.0, help="override the solver tolerance")
    ap.add_argument("--tol64", type=float, default=0.0, help="override the plain FP64 solver tolerance")
    ap.add_argument("--warm", action="store_true",
                    help="start every stage solve (mixed and FP64) from the previous step's solution")
    ap.add_argument("--batch", action="store_true", help="run the 512-problem batched workload instead")
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--serve", type=int, default=0, help="run the serving workload with this many jobs instead")
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--paper-sweep", default="", help="heat,advection: error vs tau at T = 0.1 (Sec. 5.2)")
    ap.add_argument("--paper-n", type=int, default=0, help="grid of the paper sweep (256 heat, 200 advection)")
    ap.add_argument("--advdiff", type=int, default=0, help="run the advection-diffusion GMRES workload at this n")
    ap.add_argument("--advdiff-basis", default="", help="also run the mixed step with this GMRES basis dtype")
    args = ap.parse_args()
    if args.paper_sweep:
        return run_paper_sweep(args)
    if args.advdiff:
        return run_advdiff(args)
    if args.batch:
        return run_batch(args)
    if args.serve:
        return run_serve(args)
    cfg = dict(WORKLOADS[args.workload])
    if args.bs:
        cfg["bs"] = args.bs
    if args.tol:
        cfg["tol"] = args.tol
    if args.tol64:
        cfg["tol64"] = args.tol64
    if args.warm:
        cfg["warm"] = True
    if args.impl == "reference":
        return run_reference(args, cfg)

    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_16638_b300 as rk

    n, dt = cfg["n"], cfg["dt"]
    N = n ** 3
    modes = synth.heat_modes(seed=0).modes
    u0 = synth.ModeSum(modes).evaluate(n)
    tab = rk.tableaux.get(cfg["tableau"])
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    def make(storage, tol, correct, precond="bj"):
        return rk.Problem(rk.problem_desc(n=n, kappa=cfg["kappa"]),
                          rk.solver_desc(bj_block=cfg["bs"], tol_rel=tol, storage=storage, correct=correct,
                                         max_iter=2000, precond=precond, warm_start=cfg.get("warm", False)),
                          tableau=tab, u0=u0, stream=sptr)

    # ---------------- mixed-precision path, device-resident inputs
    p = make(cfg["storage"], cfg["tol"], 1, cfg.get("precond", "bj"))
    rk.rk_integrate(p.h, dt, args.warmup)
    rk.rk_profile(p.h, True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = rk.rk_integrate(p.h, dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    prof, launches = rk.rk_profile_read(p.h)
    rk.rk_profile(p.h, False)
    secs = e0.elapsed_time(e1) / 1e3
    if dist is not None:
        t = torch.tensor([secs], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    value = world * N * args.steps / secs
    iters_per_step = st.iters_total / args.steps
    u = p.state()
    disc, cont = closed_form(n, cfg["kappa"], dt, args.warmup + args.steps, tab, modes)
    err_disc, err_cont = rel(u, disc), rel(u, cont)

    # ---------------- end to end through the public API: host state in/out every step
    hin = torch.from_numpy(u0.copy()).pin_memory()
    hout = torch.empty(N, dtype=torch.float64).pin_memory()
    k_e2e = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        rk.rk_set_state(p.h, hin)
        rk.rk_step(p.h, dt)
        rk.rk_get_state(p.h, hout)
    torch.cuda.synchronize()
    barrier()
    e2e_secs = time.perf_counter() - t0
    e2e_value = world * N * k_e2e / e2e_secs
    p.close()

    # ---------------- roofline of the dominant HBM-bound kernel; the FP64
    # stencil kernels are bound by the FP64 pipe and reported apart
    peak, peak_kind = measured_peaks()
    dom = max(((k, v) for k, v in prof.items() if k not in FP64_ALU), key=lambda kv: kv[1]["ms_total"])
    dname, d = dom
    achieved = d["bytes_total"] / (d["ms_total"] / 1e3) / 1e9
    kernels = {k: {"launches": v["launches"], "noop_launches": v["noop_launches"],
                   "ms_total": round(v["ms_total"], 3),
                   "avg_us": round(1e3 * v["ms_total"] / max(v["launches"], 1), 2),
                   "GBps": round(v["bytes_total"] / max(v["ms_total"], 1e-9) / 1e6, 1),
                   "share": round(v["ms_total"] / sum(x["ms_total"] for x in prof.values()), 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms_total"])}
    traffic = ncu_traffic(dname, args.workload)
    roofline = {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "traffic": traffic,
                "bytes_per_launch": d["bytes_total"] / max(d["launches"], 1),
                "avg_launch_us": 1e3 * d["ms_total"] / max(d["launches"], 1)}
    fp64_alu = None
    if "op_apply_f64" in prof:
        a = prof["op_apply_f64"]
        ipd = FP64_ALU["op_apply_f64"] + FP64_ALU_MAXNORM.get(cfg["storage"], 0)
        rate = ipd * N * a["launches"] / (a["ms_total"] / 1e3) / 1e9
        fp64_alu = {"bound": "alu", "kernel": "op_apply_f64", "fp64_instr_per_dof": ipd,
                    "achieved": round(rate, 1), "peak": FP64_PEAK_GINSTR, "unit": "G FP64 instr/s",
                    "frac": round(rate / FP64_PEAK_GINSTR, 4),
                    "share": round(a["ms_total"] / sum(x["ms_total"] for x in prof.values()), 4)}

    # ---------------- plain FP64 DIRK step of the same problem
    fp64 = None
    if not args.no_fp64:
        q = make("f64", cfg["tol64"], 0)
        rk.rk_integrate(q.h, dt, args.warmup)
        k64 = args.steps
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64 = rk.rk_integrate(q.h, dt, k64)
        f1.record(stream)
        torch.cuda.synchronize()
        sec64 = f0.elapsed_time(f1) / 1e3
        u64 = q.state()
        q.close()
        d64, c64 = closed_form(n, cfg["kappa"], dt, args.warmup + k64, tab, modes)
        fp64 = {"value": N * k64 / sec64, "ms_per_step": 1e3 * sec64 / k64, "steps": k64,
                "iters_per_step": s64.iters_total / k64, "tol_rel": cfg["tol64"], "err_vs_discrete": rel(u64, d64),
                "err_vs_continuous": rel(u64, c64)}

    # ---------------- the same workload with the fast-diagonalization preconditioner
    fdm_line = None
    if cfg.get("precond", "bj") == "bj" and cfg["storage"] != "f64" and n <= 256 and not args.no_fdm:
        f = make(cfg["storage"], cfg["tol"], 1, "fdm")
        rk.rk_integrate(f.h, dt, args.warmup)
        rk.rk_profile(f.h, True)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        sf = rk.rk_integrate(f.h, dt, args.steps)
        g1.record(stream)
        torch.cuda.synchronize()
        fprof, flaunch = rk.rk_profile_read(f.h)
        secf = g0.elapsed_time(g1) / 1e3
        uf = f.state()
        f.close()
        fk = {k: v for k, v in fprof.items() if k.startswith("fdm_pass")}
        fms = sum(v["ms_total"] for v in fk.values())
        fbytes = sum(v["bytes_total"] for v in fk.values())
        fn = sum(v["launches"] for v in fk.values())
        fdm_line = {"value": world * N * args.steps / secf, "ms_per_step": 1e3 * secf / args.steps,
                    "iters_per_step": sf.iters_total / args.steps, "tol_rel": cfg["tol"],
                    "err_vs_discrete": rel(uf, disc), "err_vs_continuous": rel(uf, cont),
                    "matched_ratio": rel(uf, cont) / rel(disc, cont), "gpu_launches": flaunch,
                    "fdm_pass": {"launches": fn, "avg_us": 1e3 * fms / max(fn, 1),
                                 "GBps": fbytes / max(fms, 1e-9) / 1e6,
                                 "frac_hbm": fbytes / max(fms, 1e-9) / 1e6 / peak},
                    "share_fdm_pass": fms / sum(v["ms_total"] for v in fprof.values())}

    # ---------------- matched error: both paths within MATCH x the error of an
    # exact solve (the fully discrete solution) against the exact solution
    e_exact = rel(disc, cont)
    matched = {"exact_solve_err": e_exact, "mixed_ratio": err_cont / e_exact,
               "fp64_ratio": (fp64["err_vs_continuous"] / e_exact) if fp64 else None, "bound": MATCH}
    matched["ok"] = bool(matched["mixed_ratio"] <= MATCH and (fp64 is None or matched["fp64_ratio"] <= MATCH))

    # ---------------- oracle on the host cores
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        t_step, sample = oracle_step_seconds(cfg, iters_per_step)
        cpu = {"value": N / t_step, "unit": "DOF*steps/s", "cores": 1, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF*steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args.workload, cfg), parallelism="replicas" if world > 1 else "single"),
            "e2e": {"value": e2e_value, "unit": "DOF*steps/s", "h2d_bytes_per_step": 8 * N,
                    "d2h_bytes_per_step": 8 * N, "steps": k_e2e},
            "gpu_launches": launches,
            "roofline": roofline,
            "fp64_alu": fp64_alu,
            "cpu_baseline": cpu,
            "clocks": clk,
            "iters_per_step": iters_per_step,
            "true_res_max": st.true_res,
            "err_vs_discrete": err_disc,
            "err_vs_continuous": err_cont,
            "matched_error": matched,
            "fp64_plain": fp64,
            "speedup_vs_fp64": (value / world / fp64["value"]) if fp64 else None,
            "fdm": (dict(fdm_line, speedup_vs_fp64=(fdm_line["value"] / world / fp64["value"]) if fp64 else None)
                    if fdm_line else None),
            "kernels": kernels,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
