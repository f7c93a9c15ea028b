"""Benchmark: mixed-precision perturbed DIRK steps of the 3D heat equation on B300.

One step = one pass of the whole stage loop (stage right-hand sides, FP64
operator, low-precision block-Jacobi CG solve, FP64 explicit correction and
true residual, FP64 update) over the workload below.

Headline workload (heat256): kappa = 1 on the 256^3 interior grid, u0 = unit
sine mode + 32 seeded random low modes (amplitudes N(0, 0.1^2)), the
two-stage L-stable SDIRK split for mixed precision (implicit stages in low
precision, explicit history and the update in FP64), dt = 1e-3, FP32
storage/arithmetic CG with x-line block-Jacobi (8) at the loosest tolerance
whose result stays within 1e-6 of the exact fully discrete solution at
T = 0.1 (100 steps) and whose error against the exact solution matches that of
an exact solve (within 5 %).  The plain FP64 DIRK step of the same problem is
timed beside it at its own loosest matched tolerance.  The line carries
`parity_ok` (both conditions, checked at T = 0.1) and, as further keys of the
same run: the step at tol 1e-3, FP16 and BF16 storage at 256^3, the 128^3
(L2-resident) grid, the fast-diagonalization preconditioner, 512 batched
problems, the 192^3 advection-diffusion GMRES pair, the paper's periodic
advection problem at 200^3 (complex fast diagonalization) and a slice of the
serving workload.

Metric: DOF*steps/s = n^3 * steps / seconds (device time, CUDA events on the
library's stream), inputs resident in HBM; the 256^3 working set (about
1.3 GB) is larger than L2, so no flush is needed.  Usage:
    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica on its own GPU (the
single problem does not shard): value = total DOF*steps over all ranks / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import platform
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
T_END = 0.1  # the paper's final time (Sec. 5.3); 100 steps of dt = 1e-3
# tol: solver tolerance of the mixed path; tol64: of the plain FP64 path.  The
# heat256 values are the loosest tolerances (on the half-decade grid 1e-2,
# 3e-3, 1e-3, 3e-4, 1e-4, ...) that meet the conditions of the module
# docstring at T = 0.1; tol 1e-3 is also the tolerance of the paper's accuracy
# study (Sec. 5.4) and is reported as a secondary key.
WORKLOADS = {
    "heat256": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-4, tol64=3e-4, storage="f32"),
    "heat256-tight": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-6, tol64=1e-6, storage="f32"),
    "heat256-4s3pB": dict(n=256, kappa=1.0, tableau="4s3pB", dt=1e-3, bs=8, tol=1e-6, tol64=1e-6, storage="f32"),
    "heat256-f16": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-3, tol64=3e-4, storage="f16"),
    "heat256-bf16": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-3, tol64=3e-4, storage="bf16"),
    "heat128": dict(n=128, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-4, tol64=3e-4, storage="f32"),
    # the fast-diagonalization preconditioner (tensor-core mode products) in place of block-Jacobi
    "heat256-fdm": dict(n=256, kappa=1.0, tableau="sdirk2", dt=1e-3, bs=8, tol=1e-3, tol64=3e-4, storage="f32",
                        precond="fdm"),
}


def max_over_ranks(dist, seconds, device="cuda"):
    """Largest `seconds` over all ranks (the slowest replica sets the job's
    time); `dist` None means a single process."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(world, dof, steps, seconds):
    """Whole-job throughput of `world` independent replicas, each stepping
    `dof` unknowns `steps` times, finished within `seconds` (max over ranks)."""
    return world * dof * steps / seconds


MATCH = 1.05  # matched error: within 5 % of the exact solve's error
PARITY = {"f64": 1e-10, "f32": 1e-6, "f16": 5e-3, "bf16": 5e-3}  # bound against the exact discrete solution
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
CPU_N = 128  # grid of the oracle's timed sample (whole converged steps)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from one ncu capture, valid while the kernel's sources are
# those the counters were taken on (first 16 hex digits of the sha256 of the
# listed files, concatenated).  Capture (after the same command exited 0):
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none -k regex:cg_tiled_b -s 60 -c 3
#       python bench.py --no-extras --no-cpu --no-fp64 --steps 2 --warmup 1
# (three launches: 282.8, 280.0, 279.9 MB; cold L2 between launches).
TRAFFIC = {"cg_sweep_b": {"bytes": 280.9e6, "sources": ["paper_2412_16638_b300/csrc/rk_tiled.cuh",
                                                        "paper_2412_16638_b300/csrc/rk_heat.cuh"],
                          "sha256_16": "fc2f9ac65e387c4b"}}


def measured_traffic(kernel):
    """The captured DRAM bytes per launch of `kernel`, or None when there is no
    capture or the kernel's sources changed since it was taken."""
    import hashlib
    t = TRAFFIC.get(kernel)
    if t is None:
        return None
    h = hashlib.sha256()
    try:
        for f in t["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return t["bytes"] if h.hexdigest()[:16] == t["sha256_16"] else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


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


_CLOSED = {}


def closed_form(n, kappa, dt, steps, tab, modes):
    """Exact fully discrete solution sum_m a_m R(dt lambda_m)^steps phi_m and the
    continuous solution sum_m a_m exp(lambda^c_m t) phi_m (written out here
    from the sine-mode eigenvalues; not the library, not the oracle).  Cached:
    several paths of one run are checked at the same step counts."""
    key = (n, kappa, dt, steps, tuple(np.ravel(tab[0])), tuple(np.ravel(tab[1])), tuple(tab[2]),
           tuple(tuple(m) for m in modes))
    if key not in _CLOSED:
        _CLOSED[key] = _closed_form(n, kappa, dt, steps, tab, modes)
    return _CLOSED[key]


def _closed_form(n, kappa, dt, steps, tab, modes):
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


def cpu_info():
    model = platform.processor() or ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model}


# ------------------------------------------------------------------ oracle timing
def _oracle_setup(cfg, n):
    from oracle import dirk, operators, tableau
    op = operators.HeatOperator(n, cfg["kappa"])
    tab = tableau.get(cfg["tableau"])
    u0 = synth.heat_modes(seed=0).evaluate(n)
    solver = dirk.Solver("cg", bs=cfg["bs"], tol_rel=cfg["tol"], max_iter=2000, precond=cfg.get("precond", "bj"))
    return dirk, op, tab, u0, solver


def _one_thread():
    """Limit BLAS/OpenMP pools to one thread (threadpoolctl when installed;
    numpy's element-wise kernels, the oracle's main cost, are single-threaded
    anyway)."""
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(1)
    except ImportError:
        import contextlib
        return contextlib.nullcontext()


def _oracle_replica(args):
    """One oracle process (1 thread): `warm` untimed steps, a barrier, then
    `steps` timed steps.  Returns (t_start, t_end, CG iterations)."""
    cfg, n, warm, steps, barrier = args
    with _one_thread():
        dirk, op, tab, u, solver = _oracle_setup(cfg, n)
        for _ in range(warm):
            u = dirk.rk_step(u, cfg["dt"], tab, op, solver)
        if barrier is not None:
            barrier.wait()
        stats = []
        t0 = time.monotonic()
        for _ in range(steps):
            u = dirk.rk_step(u, cfg["dt"], tab, op, solver, stats=stats)
        t1 = time.monotonic()
    return t0, t1, sum(s[0] for s in stats), all(s[1] for s in stats)


def _replica_count(n):
    """Oracle processes for the all-cores figure: one per core, as many as the
    host memory holds (about 1 GB each at 128^3)."""
    avail = None
    try:
        import psutil
        avail = psutil.virtual_memory().available
    except Exception:
        pass
    per = 1.0e9 * (n / 128.0) ** 3
    cap = int(avail // per) if avail else 8
    return max(1, min(os.cpu_count() or 1, cap, 64))


def oracle_all_cores(cfg, n, warm, steps):
    """P one-thread oracle processes (spawned, so that no CUDA state is
    inherited) stepping P copies of the problem at once after a common
    barrier: aggregate DOF*steps/s of the host = P n^3 steps / (last end -
    first start)."""
    P = _replica_count(n)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"  # inherited by the spawned processes: one thread each
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(P)
        with ctx.Pool(P) as pool:
            res = pool.map(_oracle_replica, [(cfg, n, warm, steps, barrier)] * P)
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    return {"value": P * n ** 3 * steps / (t1 - t0), "processes": P, "seconds": t1 - t0,
            "iters_per_step": res[0][2] / steps, "converged": all(r[3] for r in res)}


def oracle_one_thread(cfg, n, steps, best_of=3):
    """Best of `best_of` single whole oracle steps (1 thread), after one untimed
    step that also builds the preconditioners."""
    with _one_thread():
        dirk, op, tab, u, solver = _oracle_setup(cfg, n)
        u = dirk.rk_step(u, cfg["dt"], tab, op, solver)
        times, iters, conv = [], [], True
        for _ in range(best_of):
            stats = []
            t0 = time.perf_counter()
            for _ in range(steps):
                u = dirk.rk_step(u, cfg["dt"], tab, op, solver, stats=stats)
            times.append(time.perf_counter() - t0)
            iters.append(sum(s[0] for s in stats) / steps)
            conv = conv and all(s[1] for s in stats)
    best = min(times)
    return {"value": n ** 3 * steps / best, "seconds_per_step": best / steps, "all_seconds": times,
            "iters_per_step": iters[int(np.argmin(times))], "converged": conv}


def cpu_baseline(cfg):
    """The oracle (float64 numpy, as it stands) on the host cores: whole
    converged steps of the same problem at 128^3 (the 256^3 step takes about
    half a minute per step on one core), one thread (best of 3) and all cores
    (one process per core, one step each)."""
    n = CPU_N
    one = oracle_one_thread(cfg, n, 1, best_of=3)
    allc = oracle_all_cores(cfg, n, warm=1, steps=1)
    info = cpu_info()
    return {"value": allc["value"], "unit": "DOF*steps/s", "cores": allc["processes"], "kind": "oracle",
            "sample": ("oracle float64 numpy at %d^3 (same tableau, tolerance, block size and seeded data as the "
                       "GPU workload; whole converged steps, %.1f CG iterations per step): all cores = %d "
                       "one-thread processes each stepping its own copy once after a barrier (%.1f s); one thread "
                       "= best of 3 single steps; DOF*steps/s per grid point, not rescaled to 256^3"
                       % (n, one["iters_per_step"], allc["processes"], allc["seconds"])),
            "one_thread": {"value": one["value"], "seconds_per_step": one["seconds_per_step"],
                           "all_seconds": one["all_seconds"]},
            "all_cores": allc, "host": info, "grid": "%d^3" % n}


def run_reference(args, cfg):
    """The reference arm: the float64 oracle itself on the host cores, one
    one-thread process per core, each stepping its own copy of the workload's
    problem at 128^3 (W untimed steps, a barrier, K timed steps)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = CPU_N
    allc = oracle_all_cores(cfg, n, warm=args.warmup, steps=args.steps)
    value = allc["value"]
    sample = ("oracle float64 numpy at %d^3, %d one-thread processes (one per core, memory permitting), each "
              "%d untimed + %d timed whole converged steps of the %s problem (%.1f CG iterations per step); "
              "value = processes * %d^3 * steps / wall time of the timed region"
              % (n, allc["processes"], args.warmup, args.steps, args.workload, allc["iters_per_step"], n))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF*steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * allc["seconds"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args.workload, cfg), oracle_grid="%d^3" % n),
        "cpu_baseline": {"value": value, "unit": "DOF*steps/s", "cores": allc["processes"], "kind": "oracle",
                         "sample": sample, "host": cpu_info()},
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


# ------------------------------------------------------------------ GPU runs
class Ctx:
    """Library handle, stream and the workload's seeded data."""

    def __init__(self, rk, torch, stream):
        self.rk, self.torch, self.stream = rk, torch, stream
        self.modes = synth.heat_modes(seed=0).modes
        self._u0 = {}

    def u0(self, n):
        if n not in self._u0:
            self._u0[n] = synth.ModeSum(self.modes).evaluate(n)
        return self._u0[n]


def heat_problem(c, cfg, storage, tol, correct, precond="bj"):
    rk = c.rk
    return rk.Problem(rk.problem_desc(n=cfg["n"], kappa=cfg["kappa"]),
                      rk.solver_desc(bj_block=cfg["bs"], tol_rel=tol, storage=storage, correct=correct,
                                     max_iter=2000, precond=precond, warm_start=cfg.get("warm", False)),
                      tableau=rk.tableaux.get(cfg["tableau"]), u0=c.u0(cfg["n"]), stream=c.stream.cuda_stream)


def kernel_table(prof):
    tot = sum(x["ms_total"] for x in prof.values()) or 1e-9
    return {k: {"launches": v["launches"], "noop_launches": v["noop_launches"], "ms_total": round(v["ms_total"], 3),
                "avg_us": round(1e3 * v["ms_total"] / max(v["launches"], 1), 2),
                "GBps": round(v["bytes_total"] / max(v["ms_total"], 1e-9) / 1e6, 1),
                "share": round(v["ms_total"] / tot, 4)}
            for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms_total"])}


def roofline_of(prof, peak, peak_kind):
    """HBM roofline of the dominant HBM-bound kernel: its algorithmic bytes per
    launch over its average CUDA-event duration (the FP64 stencil kernels are
    bound by the FP64 pipe and reported apart)."""
    cands = [(k, v) for k, v in prof.items() if k not in FP64_ALU and v["launches"] > 0]
    if not cands:
        return None
    dname, d = max(cands, key=lambda kv: kv[1]["ms_total"])
    achieved = d["bytes_total"] / (d["ms_total"] / 1e3) / 1e9
    return {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
            "bytes_per_launch": d["bytes_total"] / max(d["launches"], 1),
            "avg_launch_us": 1e3 * d["ms_total"] / max(d["launches"], 1)}


def timed_heat(c, cfg, storage, tol, correct, K, W, total=None, precond="bj", profile=False, clocks=None,
               barrier=None):
    """W untimed steps, K steps timed with CUDA events on the library's
    stream, then (if total) further steps up to `total`.  Errors against the
    closed forms after W + K steps and after `total` steps."""
    rk, torch = c.rk, c.torch
    p = heat_problem(c, cfg, storage, tol, correct, precond)
    rk.rk_integrate(p.h, cfg["dt"], W)
    if profile:
        rk.rk_profile(p.h, True)
    if clocks is not None:
        clocks.start()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(c.stream)
    st = rk.rk_integrate(p.h, cfg["dt"], K)
    e1.record(c.stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    out = {"clocks": clocks.stop() if clocks is not None else None}
    if profile:
        out["prof"], out["launches"] = rk.rk_profile_read(p.h)
        rk.rk_profile(p.h, False)
    secs = e0.elapsed_time(e1) / 1e3
    tab = rk.tableaux.get(cfg["tableau"])
    n = cfg["n"]
    u = p.state()
    disc, cont = closed_form(n, cfg["kappa"], cfg["dt"], W + K, tab, c.modes)
    out.update({"seconds": secs, "value": n ** 3 * K / secs, "ms_per_step": 1e3 * secs / K,
                "iters_per_step": st.iters_total / K, "true_res_max": st.true_res, "not_converged": st.not_converged,
                "steps_checked": W + K, "err_vs_discrete": rel(u, disc), "err_vs_continuous": rel(u, cont),
                "exact_solve_err": rel(disc, cont), "tol_rel": tol, "storage": storage})
    if total and total > W + K:
        rk.rk_integrate(p.h, cfg["dt"], total - W - K)
        uT = p.state()
        dT, cT = closed_form(n, cfg["kappa"], cfg["dt"], total, tab, c.modes)
        out.update({"steps_T": total, "err_vs_discrete_T": rel(uT, dT), "err_vs_continuous_T": rel(uT, cT),
                    "exact_solve_err_T": rel(dT, cT)})
    out["_problem"] = p
    return out


def summary(r, keys=("value", "ms_per_step", "iters_per_step", "tol_rel", "storage", "err_vs_discrete",
                     "err_vs_continuous", "steps_checked", "err_vs_discrete_T", "err_vs_continuous_T", "steps_T")):
    return {k: r[k] for k in keys if k in r}


def run_batch_key(c, steps):
    """512 independent heat problems (n uniform in 16..64, kappa log-uniform in
    [0.1, 10], amplitude * sine mode), SDIRK2, dt 1e-3, FP32 solves / FP64
    corrections, tol 1e-6, `steps` steps in persistent graph-captured launches,
    timed with CUDA events.  Value = sum n^3 * steps / seconds."""
    rk, torch = c.rk, c.torch
    probs = synth.batch_problems(512, seed=0)
    tab = rk.tableaux.get("sdirk2")
    dt = 1e-3
    ps = [rk.Problem(rk.problem_desc(n=pr.n, kappa=pr.kappa),
                     rk.solver_desc(bj_block=8, tol_rel=1e-6, storage="f32", max_iter=2000, correct=1),
                     tableau=tab, u0=pr.amplitude * synth.sine_mode(pr.n), stream=c.stream.cuda_stream)
          for pr in probs]
    handles = [p.h for p in ps]
    rk.rk_integrate_batch(handles, dt, 3)  # warm-up (the launch-shape autotuner times its candidates here)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(c.stream)
    st = rk.rk_integrate_batch(handles, dt, steps)
    e1.record(c.stream)
    torch.cuda.synchronize()
    host_secs = time.perf_counter() - t0
    secs = e0.elapsed_time(e1) / 1e3
    peak, peak_kind = measured_peaks()
    achieved = st.bytes / secs / 1e9
    dof = sum(pr.n ** 3 for pr in probs)
    # parity against the closed form on a few problems (amplitude * R^N * phi)
    A = np.array(tab[0]) + np.array(tab[1])
    b = np.array(tab[2])
    errs = []
    for pr, p in list(zip(probs, ps))[:16]:
        h = 1.0 / (pr.n + 1)
        lam = -12.0 * pr.kappa / h ** 2 * math.sin(math.pi * h / 2) ** 2
        z = dt * lam
        R = 1.0 + z * (b @ np.linalg.solve(np.eye(2) - z * A, np.ones(2)))
        errs.append(rel(p.state(), pr.amplitude * R ** (steps + 3) * synth.sine_mode(pr.n)))
    for p in ps:
        p.close()
    return {"value": dof * steps / secs, "unit": METRIC, "problems": 512, "total_dof": dof, "steps": steps,
            "seconds": secs, "host_seconds": host_secs, "ms_per_step": 1e3 * secs / steps,
            "iters_per_solve": st.iters_total / max(st.solves, 1),
            "true_res_max": st.true_res, "max_err_vs_discrete_16": max(errs),
            "roofline": {"bound": "hbm", "kernel": "whole batched step (work-list kernels)",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "bytes_per_step": st.bytes / steps},
            "config": {"tableau": "sdirk2", "dt": dt, "storage": "f32", "bj_block": 8, "tol_rel": 1e-6,
                       "n": "uniform 16..64", "kappa": "log-uniform [0.1, 10]",
                       "timer": "CUDA events on the problems' stream around the call"}}


def run_advdiff_key(c, n, steps, warmup, basis=None):
    """Advection-diffusion (variable kappa, CSR, GMRES(30) + block-Jacobi 8,
    DIRK3, dt 5e-4, tol 1e-8): the mixed step (FP32 GMRES, FP64 corrections)
    against the plain FP64 step on the same problem, both timed with CUDA
    events over `steps` steps after `warmup`; errors against an FP64 run
    solved to 1e-12 (no closed form for variable kappa)."""
    rk, torch = c.rk, c.torch
    dt, vel = 5e-4, (1.0, 0.5, 0.25)
    N = n ** 3
    kap = synth.kappa_field(n, seed=0)
    u0 = synth.gaussian_bump(n)
    tab = rk.tableaux.get("dirk3")
    stream = c.stream

    def make(storage, tol, correct, basis=None, tau=0.0):
        kw = {} if basis is None else {"basis": basis}
        return rk.Problem(rk.problem_desc(op=rk.RK_OP_ADVDIFF_CSR, n=n, kappa_field=kap, vel=vel),
                          rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=tol,
                                         storage=storage, correct=correct, max_iter=3000, bj_adapt_tau=tau, **kw),
                          tableau=tab, u0=u0, stream=stream.cuda_stream)

    with make("f64", 1e-12, 0) as q:
        rk.rk_integrate(q.h, dt, warmup + steps)
        ref = q.state()
    # adaptive-precision block-Jacobi (tau 1e-2: FP16 block inverses where kappa_1 <= 20)
    variants = {"mixed_f32": ("f32", 1e-8, 1, None, 0.0), "mixed_f32_adaptive_bj": ("f32", 1e-8, 1, None, 1e-2),
                "fp64_plain": ("f64", 1e-8, 0, None, 0.0)}
    if basis:
        variants["mixed_f32_basis_" + basis] = ("f32", 1e-8, 1, basis, 0.0)
    res = {}
    peak, peak_kind = measured_peaks()
    for name, (storage, tol, corr, bas, tau) in variants.items():
        with make(storage, tol, corr, bas, tau) as p:
            rk.rk_integrate(p.h, dt, warmup)
            rk.rk_profile(p.h, True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = rk.rk_integrate(p.h, dt, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            prof, launches = rk.rk_profile_read(p.h)
            secs = e0.elapsed_time(e1) / 1e3
            u = p.state()
            info = rk.rk_get_problem_info(p.h)
        res[name] = {"value": N * steps / secs, "ms_per_step": 1e3 * secs / steps,
                     "bj_half_blocks": info.bj_half_blocks, "bj_blocks": info.bj_blocks,
                     "iters_per_solve": st.iters_total / max(st.solves, 1), "err_vs_fp64_tight": rel(u, ref),
                     "gpu_launches": launches, "roofline": roofline_of(prof, peak, peak_kind),
                     "kernels": kernel_table(prof)}
    return {"unit": METRIC, "steps": steps, "warmup": warmup,
            "config": {"grid": "%d^3" % n, "kappa": "exp(Gaussian field, sigma 0.5, l 0.1), seed 0",
                       "vel": vel, "tableau": "dirk3", "dt": dt, "krylov": "gmres(30)", "bj_block": 8,
                       "tol_rel": 1e-8, "u0": "Gaussian bump"},
            "variants": res, "speedup_vs_fp64": res["mixed_f32"]["value"] / res["fp64_plain"]["value"],
            "speedup_vs_fp64_adaptive_bj": res["mixed_f32_adaptive_bj"]["value"] / res["fp64_plain"]["value"]}


# nominal FP32 FMA rate of the part: 128 FP32 lanes per SM x 148 SMs x 2.032 GHz
FP32_FMA_PEAK_T = 128 * 148 * 2.032e9 / 1e12


def cfdm_dft_ops(N):
    """FP32 lane operations (FADD, FMUL, FFMA) of the compile-time DFT of size
    N in csrc/rk_cfdm.cuh: size 2 four adds; an odd prime through the
    symmetric pairs (4H^2 + 10H, H = (N - 1) / 2); N = P Q (P the smallest
    factor) Q transforms of size P, a complex product (4 operations) for each
    twiddle that is not 1, -1 or +-i, and P transforms of size Q."""
    if N == 1:
        return 0
    if N == 2:
        return 4
    p = next((d for d in range(2, int(math.isqrt(N)) + 1) if N % d == 0), N)
    if p == N:
        h = (N - 1) // 2
        return 4 * h * h + 10 * h
    q = N // p
    tw = sum(1 for j2 in range(q) for k1 in range(p) if (j2 * k1) % N and 4 * ((j2 * k1) % N) % N)
    return q * cfdm_dft_ops(p) + 4 * tw + p * cfdm_dft_ops(q)


def cfdm_ct_ops(n):
    """FP32 operations per element of one compile-time pass at n = n1 n2:
    n2 transforms of size n1 with the n1 - 1 table twiddles each, then n1 of
    size n2, per line of n elements."""
    n1 = max(d for d in range(1, int(math.isqrt(n)) + 1) if n % d == 0)
    n2 = n // n1
    return (n2 * (cfdm_dft_ops(n1) + 4 * (n1 - 1)) + n1 * cfdm_dft_ops(n2)) / n


def run_periodic_key(c, n=200, steps=3, warmup=1, tau=0.1):
    """The paper's periodic advection problem (Sec. 5.2.2; beta = (1,1,1), the
    Gaussian bump, n = 200) at its largest time step tau = 1/10 with 4s3pB:
    FP32 GMRES(30) at tol 1e-3 preconditioned by the complex fast
    diagonalization, with FP64 corrections (mixed), against the plain FP64 step
    with the same preconditioner in FP64.  Timed with CUDA events; errors
    against the exact solution (the bump translated by beta t).  n = 200 runs
    the compile-time small transforms (about 29 FP32 operations per element
    and pass, `cfdm_ct_ops`), far from the FP32 rate, so the roofline of
    `cfdm_pass` is its HBM bytes; the FP32 operations are reported beside it."""
    rk, torch = c.rk, c.torch
    stream = c.stream
    beta = (1.0, 1.0, 1.0)
    tab = rk.tableaux.get("4s3pB")
    u0 = synth.gaussian_bump_periodic(n)
    x, y, z = synth.periodic_coords(n)
    t_end = (warmup + steps) * tau
    d2 = sum(((q - 0.5 - t_end * b + 0.5) % 1.0 - 0.5) ** 2 for q, b in zip((x, y, z), beta))
    exact = np.exp(-100.0 * d2).ravel()
    res = {}
    for name, storage, corr in (("mixed_f32", "f32", 1), ("fp64_plain", "f64", 0)):
        sol = rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=1e-3, storage=storage,
                             max_iter=1000, correct=corr, precond="fdm")
        with rk.Problem(rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=n, vel=beta), sol, tableau=tab, u0=u0,
                        stream=stream.cuda_stream) as p:
            rk.rk_integrate(p.h, tau, warmup)
            rk.rk_profile(p.h, True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = rk.rk_integrate(p.h, tau, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            prof, launches = rk.rk_profile_read(p.h)
            secs = e0.elapsed_time(e1) / 1e3
            u = p.state()
        r = {"value": n ** 3 * steps / secs, "ms_per_step": 1e3 * secs / steps,
             "iters_per_solve": st.iters_total / max(st.solves, 1), "err_vs_exact": rel(u, exact),
             "gpu_launches": launches, "kernels": kernel_table(prof)}
        cf = prof.get("cfdm_pass")
        if cf and cf["launches"] > 0:
            work = cf["launches"]  # passes that ran (skipped ones are counted apart)
            secs_cf = cf["ms_total"] / 1e3
            gbps = cf["bytes_total"] / secs_cf / 1e9
            ops = cfdm_ct_ops(n) * n ** 3 * work  # FP32 lane operations of the passes that ran
            hbm, hbm_kind = measured_peaks()
            r["cfdm_roofline"] = {"bound": "hbm", "achieved": round(gbps, 1), "unit": "GB/s", "peak": hbm,
                                  "peak_kind": hbm_kind, "frac": round(gbps / hbm, 4),
                                  "avg_us": round(1e3 * cf["ms_total"] / work, 1),
                                  "fp32_ops_per_element": round(cfdm_ct_ops(n), 2),
                                  "fp32_ops_T": round(ops / secs_cf / 1e12, 2),
                                  "fp32_frac": round(ops / secs_cf / 1e12 / FP32_FMA_PEAK_T, 4)} \
                if storage == "f32" else {"avg_us": round(1e3 * cf["ms_total"] / work, 1)}
        res[name] = r
    return {"unit": METRIC, "steps": steps, "warmup": warmup,
            "config": {"grid": "%d^3" % n, "problem": "periodic advection, beta (1,1,1), Gaussian bump",
                       "tableau": "4s3pB", "dt": tau, "krylov": "gmres(30)", "precond": "complex fdm",
                       "tol_rel": 1e-3},
            "variants": res, "speedup_vs_fp64": res["mixed_f32"]["value"] / res["fp64_plain"]["value"]}


def run_serve_key(c, njobs, slots=64, budget=120 << 30):
    """Serving: the first `njobs` jobs of the seeded stream (Poisson arrivals,
    200 jobs/s; n in {32, 64, 96, 128, 192}, tableau in {midpoint + 1
    correction, SDIRK2, DIRK3}, storage in {FP32, FP16}, 10..200 steps, kappa
    log-uniform in [0.1, 10], dt 1e-3), 120 GB budget.  Reports p50/p99
    latency (submit to finish) and aggregate DOF*steps/s over the makespan."""
    rk = c.rk
    jobs = synth.serve_jobs(njobs, seed=0)
    srv = rk.rk_server_create(budget, slots)
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
    lats, service, failed, resident = [], [], {}, []
    work = 0
    infos = []
    for jid, (jb, *_rest) in zip(ids, prepared):
        try:
            st, info = rk.rk_wait_job_info(srv, jid, None, allow_not_converged=True)
            lats.append(info.t_done - info.t_submit)
            service.append(info.t_done - info.t_admit)
            infos.append(info)
            work += jb.n ** 3 * jb.steps
        except rk.RKError as e:
            # a job that diverged (non-finite state) is reported, not timed
            key = "%s/%s/n%d: status %d" % (jb.tableau, jb.storage, jb.n, e.status)
            failed[key] = failed.get(key, 0) + 1
    makespan = time.perf_counter() - t0
    rk.rk_server_destroy(srv)
    # jobs stepped in the same tick (concurrently on the device), averaged over ticks
    if infos:
        last = max(f.last_tick for f in infos)
        counts = np.zeros(last + 1)
        for f in infos:
            counts[f.first_tick:f.last_tick + 1] += 1
        resident = {"mean_jobs_per_tick": float(counts.mean()), "max_jobs_per_tick": int(counts.max()),
                    "ticks": int(last + 1)}
    return {"value": work / makespan, "unit": METRIC, "jobs": len(jobs), "makespan_s": makespan,
            "latency_p50_s": float(np.percentile(lats, 50)) if lats else None,
            "latency_p99_s": float(np.percentile(lats, 99)) if lats else None,
            "service_p50_s": float(np.percentile(service, 50)) if service else None,
            "service_p99_s": float(np.percentile(service, 99)) if service else None,
            "completed": len(lats), "failed": failed, "co_residency": resident,
            "config": {"arrival_rate_per_s": 200, "slots": slots, "budget_bytes": budget,
                       "sizes": [32, 64, 96, 128, 192], "tableaux": ["midpoint1", "sdirk2", "dirk3"],
                       "storage": ["f32", "f16"], "steps": "uniform 10..200", "dt": 1e-3,
                       "jobs": "the first %d of the seeded 2000-job stream" % njobs}}


def run_fp32_floor(c, steps=10):
    """The FP32 floor of the perturbed step: errors against the exact fully
    discrete solution on the 256^3 mode sum (dt 1e-3, FP32 block-Jacobi CG at
    tol 1e-6) per tableau, without and with refinement against the FP64 true
    residual (tol_true 1e-9, k^eps then held in FP64); and the stiffest
    problems of the batched workload (dt ||L|| > 300, 5 steps of SDIRK2)."""
    rk = c.rk
    out = {"heat256": [], "stiff_batch": []}
    n, dt = 256, 1e-3
    for tab in ("sdirk2", "dirk3", "4s3pB", "4s3pC"):
        cfg = dict(WORKLOADS["heat256"], tableau=tab)
        row = {"tableau": tab, "steps": steps, "dt_norm_L": dt * 12.0 * (n + 1) ** 2}
        t = rk.tableaux.get(tab)
        disc, _ = closed_form(n, 1.0, dt, steps, t, c.modes)
        for label, kw in (("plain", {}), ("refined", {"max_refine": 4, "tol_true": 1e-9})):
            with rk.Problem(rk.problem_desc(n=n, kappa=1.0),
                            rk.solver_desc(bj_block=8, tol_rel=1e-6, storage="f32", correct=1, max_iter=2000, **kw),
                            tableau=t, u0=c.u0(n), stream=c.stream.cuda_stream) as p:
                st = rk.rk_integrate(p.h, dt, steps)
                row[label] = {"err_vs_discrete": rel(p.state(), disc), "true_res_max": st.true_res,
                              "refinements": st.refinements}
        out["heat256"].append(row)
    tab = rk.tableaux.get("sdirk2")
    A = np.array(tab[0]) + np.array(tab[1])
    b = np.array(tab[2])
    for pr in [q for q in synth.batch_problems(512, seed=0) if 1e-3 * 12 * q.kappa * (q.n + 1) ** 2 > 300][:6]:
        h = 1.0 / (pr.n + 1)
        z = 1e-3 * (-12.0 * pr.kappa / h ** 2 * math.sin(math.pi * h / 2) ** 2)
        R = 1.0 + z * (b @ np.linalg.solve(np.eye(2) - z * A, np.ones(2)))
        exact = pr.amplitude * R ** 5 * synth.sine_mode(pr.n)
        row = {"n": pr.n, "kappa": pr.kappa, "dt_norm_L": 1e-3 * 12 * pr.kappa * (pr.n + 1) ** 2}
        for label, kw in (("plain", {}), ("refined", {"max_refine": 4, "tol_true": 1e-10})):
            with rk.Problem(rk.problem_desc(n=pr.n, kappa=pr.kappa),
                            rk.solver_desc(bj_block=8, tol_rel=1e-6, storage="f32", correct=1, max_iter=2000, **kw),
                            tableau=tab, u0=pr.amplitude * synth.sine_mode(pr.n), stream=c.stream.cuda_stream) as p:
                rk.rk_integrate(p.h, 1e-3, 5)
                row[label] = rel(p.state(), exact)
        out["stiff_batch"].append(row)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heat256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline workload (no secondary tolerance, 16-bit, 128^3, FDM, batch, "
                         "advection-diffusion or serving keys)")
    ap.add_argument("--bs", type=int, default=0, help="override the block-Jacobi block size")
    ap.add_argument("--tol", type=float, default=0.0, help="override the solver tolerance")
    ap.add_argument("--tol64", type=float, default=0.0, help="override the plain FP64 solver tolerance")
    ap.add_argument("--warm", action="store_true",
                    help="start every stage solve (mixed and FP64) from the previous step's solution")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--batch", action="store_true", help="run only the 512-problem batched workload")
    ap.add_argument("--serve-jobs", type=int, default=60, help="jobs of the serving key in the default line")
    ap.add_argument("--serve", type=int, default=0, help="run only the serving workload with this many jobs")
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--paper-sweep", default="", help="heat,advection: error vs tau at T = 0.1 (Sec. 5.2)")
    ap.add_argument("--paper-n", type=int, default=0, help="grid of the paper sweep (256 heat, 200 advection)")
    ap.add_argument("--advdiff", type=int, default=0, help="run only the advection-diffusion workload at this n")
    ap.add_argument("--advdiff-basis", default="", help="also run the mixed step with this GMRES basis dtype")
    ap.add_argument("--advdiff-steps", type=int, default=6)
    ap.add_argument("--fp32-floor", action="store_true", help="run only the FP32-floor table (256^3, stiff batch)")
    ap.add_argument("--periodic", type=int, default=0,
                    help="run only the periodic advection key (complex fast diagonalization) at this n")
    args = ap.parse_args()
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

    c = Ctx(rk, torch, torch.cuda.current_stream())
    if args.paper_sweep:
        return run_paper_sweep(args, rk)
    if args.advdiff:
        print(json.dumps(dict(run_advdiff_key(c, args.advdiff, args.steps, args.warmup, args.advdiff_basis or None),
                              metric=METRIC, workload="advdiff%d" % args.advdiff, data="synthetic")))
        return 0
    if args.serve:
        print(json.dumps(dict(run_serve_key(c, args.serve, args.serve_slots), metric=METRIC, workload="serve")))
        return 0
    if args.batch:
        print(json.dumps(dict(run_batch_key(c, args.batch_steps), metric=METRIC, workload="batch512")))
        return 0
    if args.fp32_floor:
        print(json.dumps(run_fp32_floor(c)))
        return 0
    if args.periodic:
        print(json.dumps(dict(run_periodic_key(c, args.periodic), metric=METRIC,
                              workload="periodic%d" % args.periodic, data="synthetic")))
        return 0

    n, dt = cfg["n"], cfg["dt"]
    N = n ** 3
    K, W = args.steps, args.warmup
    total = max(int(round(T_END / dt)), W + K)
    peak, peak_kind = measured_peaks()

    # ---------------- headline: mixed-precision path, device-resident inputs
    clocks = ClockSampler(local)
    head = timed_heat(c, cfg, cfg["storage"], cfg["tol"], 1, K, W, total=total,
                      precond=cfg.get("precond", "bj"), profile=True, clocks=clocks, barrier=barrier)
    p = head.pop("_problem")
    secs = max_over_ranks(dist, head["seconds"])
    value = replicas_value(world, N, K, secs)

    # ---------------- end to end through the public API: host state in/out every step
    u0 = c.u0(n)
    hin = torch.from_numpy(u0.copy()).pin_memory()
    hout = torch.empty(N, dtype=torch.float64).pin_memory()
    k_e2e = max(1, min(K, 10))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        rk.rk_set_state(p.h, hin)
        rk.rk_step(p.h, dt)
        rk.rk_get_state(p.h, hout)
    torch.cuda.synchronize()
    barrier()
    e2e_secs = max_over_ranks(dist, time.perf_counter() - t0)
    e2e_value = replicas_value(world, N, k_e2e, e2e_secs)
    p.close()

    prof = head.pop("prof")
    launches = head.pop("launches")
    roofline = roofline_of(prof, peak, peak_kind)
    roofline["traffic"] = measured_traffic(roofline.get("kernel"))
    fp64_alu = None
    if "op_apply_f64" in prof:
        a = prof["op_apply_f64"]
        ipd = FP64_ALU["op_apply_f64"] + FP64_ALU_MAXNORM.get(cfg["storage"], 0)
        rate = ipd * N * a["launches"] / (a["ms_total"] / 1e3) / 1e9
        fp64_alu = {"bound": "alu", "kernel": "op_apply_f64", "fp64_instr_per_dof": ipd,
                    "achieved": round(rate, 1), "peak": FP64_PEAK_GINSTR, "unit": "G FP64 instr/s",
                    "frac": round(rate / FP64_PEAK_GINSTR, 4),
                    "share": round(a["ms_total"] / sum(x["ms_total"] for x in prof.values()), 4)}

    # ---------------- plain FP64 DIRK step of the same problem, same checks
    fp64 = None
    if not args.no_fp64:
        r64 = timed_heat(c, cfg, "f64", cfg["tol64"], 0, K, W, total=total)
        r64.pop("_problem").close()
        fp64 = summary(r64)

    # ---------------- parity and matched error at T = 0.1
    e_exact_T = head.get("exact_solve_err_T", head["exact_solve_err"])
    err_disc_T = head.get("err_vs_discrete_T", head["err_vs_discrete"])
    matched = {"T": total * dt, "exact_solve_err": e_exact_T,
               "mixed_ratio": head.get("err_vs_continuous_T", head["err_vs_continuous"]) / e_exact_T,
               "fp64_ratio": (fp64.get("err_vs_continuous_T", fp64["err_vs_continuous"]) / e_exact_T) if fp64 else None,
               "bound": MATCH}
    matched["ok"] = bool(matched["mixed_ratio"] <= MATCH and (fp64 is None or matched["fp64_ratio"] <= MATCH))
    bound = PARITY[cfg["storage"]]
    parity = {"err_vs_discrete_T": err_disc_T, "bound": bound, "T": total * dt,
              "err_vs_discrete_timed": head["err_vs_discrete"], "steps_timed_check": head["steps_checked"]}
    parity_ok = bool(err_disc_T <= bound and head["err_vs_discrete"] <= bound and matched["ok"])

    extras = {}
    if not args.no_extras and world == 1:
        def tol1e3():
            # the same step at the paper's accuracy-study tolerance 1e-3
            r = timed_heat(c, cfg, cfg["storage"], 1e-3, 1, K, W, total=total)
            r.pop("_problem").close()
            return dict(summary(r), parity_ok=bool(r["err_vs_discrete_T"] <= bound))

        def sixteen(st16):
            # 16-bit storage of the Krylov vectors at 256^3 (FP32 arithmetic, FP64 corrections)
            c16 = dict(WORKLOADS["heat256-" + st16])
            r = timed_heat(c, c16, st16, c16["tol"], 1, K, W, profile=True)
            r.pop("_problem").close()
            return dict(summary(r), roofline=roofline_of(r["prof"], peak, peak_kind),
                        parity_ok=bool(r["err_vs_discrete"] <= PARITY[st16]), bound=PARITY[st16])

        def heat128():
            # 128^3: the FP32 Krylov vectors (8.4 MB each) stay in the 126 MB L2
            c128 = dict(WORKLOADS["heat128"])
            r = timed_heat(c, c128, "f32", c128["tol"], 1, K, W, total=total, profile=True)
            r.pop("_problem").close()
            r64 = timed_heat(c, c128, "f64", c128["tol64"], 0, K, W)
            r64.pop("_problem").close()
            return dict(summary(r), roofline=roofline_of(r["prof"], peak, peak_kind),
                        parity_ok=bool(r["err_vs_discrete_T"] <= bound), note="L2-resident Krylov vectors",
                        fp64_plain=summary(r64), speedup_vs_fp64=r["value"] / r64["value"])

        def fdm():
            # fast-diagonalization preconditioner (tensor cores) on the headline problem
            r = timed_heat(c, cfg, cfg["storage"], 1e-3, 1, K, W, total=total, precond="fdm", profile=True)
            r.pop("_problem").close()
            fprof = r["prof"]
            fk = {k: v for k, v in fprof.items() if k.startswith("fdm_pass")}
            fms = sum(v["ms_total"] for v in fk.values())
            fbytes = sum(v["bytes_total"] for v in fk.values())
            fn = sum(v["launches"] for v in fk.values())
            return dict(summary(r), gpu_launches=r["launches"], parity_ok=bool(r["err_vs_discrete_T"] <= bound),
                        fdm_pass={"launches": fn, "avg_us": 1e3 * fms / max(fn, 1),
                                  "GBps": fbytes / max(fms, 1e-9) / 1e6,
                                  "frac_hbm": fbytes / max(fms, 1e-9) / 1e6 / peak},
                        share_fdm_pass=fms / sum(v["ms_total"] for v in fprof.values()),
                        kernels=kernel_table(fprof),
                        speedup_vs_fp64=(r["value"] / fp64["value"]) if fp64 else None)

        jobs = [("tol1e-3", tol1e3), ("heat256_f16", lambda: sixteen("f16")),
                ("heat256_bf16", lambda: sixteen("bf16")), ("heat128", heat128)]
        if cfg.get("precond", "bj") == "bj" and n <= 256:
            jobs.append(("fdm", fdm))
        jobs += [("batch512", lambda: run_batch_key(c, args.batch_steps)),
                 ("advdiff192", lambda: run_advdiff_key(c, 192, args.advdiff_steps, 2)),
                 ("periodic200", lambda: run_periodic_key(c, 200))]
        if args.serve_jobs > 0:
            jobs.append(("serve", lambda: run_serve_key(c, args.serve_jobs, args.serve_slots)))
        for key, fn in jobs:
            t0 = time.perf_counter()
            try:
                extras[key] = fn()
            except Exception as e:  # reported in the line; the other keys still run
                extras[key] = {"error": repr(e)}
            extras[key]["wall_s"] = round(time.perf_counter() - t0, 1)

    # ---------------- oracle on the host cores
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline(cfg)
        except Exception as e:  # the GPU line is still printed
            cpu = {"value": None, "unit": "DOF*steps/s", "kind": "oracle", "error": repr(e)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF*steps/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": 1e3 * secs / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args.workload, cfg), parallelism="replicas" if world > 1 else "single",
                           T_check=total * dt),
            "e2e": {"value": e2e_value, "unit": "DOF*steps/s", "h2d_bytes_per_step": 8 * N,
                    "d2h_bytes_per_step": 8 * N, "steps": k_e2e},
            "gpu_launches": launches,
            "roofline": roofline,
            "fp64_alu": fp64_alu,
            "cpu_baseline": cpu,
            "clocks": head["clocks"],
            "parity_ok": parity_ok,
            "parity": parity,
            "iters_per_step": head["iters_per_step"],
            "true_res_max": head["true_res_max"],
            "err_vs_discrete": head["err_vs_discrete"],
            "err_vs_continuous": head["err_vs_continuous"],
            "matched_error": matched,
            "fp64_plain": fp64,
            "speedup_vs_fp64": (value / world / fp64["value"]) if fp64 else None,
            "kernels": kernel_table(prof),
        }
        line.update(extras)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_paper_sweep(args, rk):
    """Error at T = 0.1 against the analytic solution for the paper's two test
    problems (Sec. 5.2) over tau = 1/10 .. 1/1280 (Fig. CombinedErrors), FP32
    mixed precision (perturbed step, FP64 corrections) vs plain FP64.  Heat
    (Sec. 5.2.1): u_t = Lap u + g, g the sine mode, u(0) = 0,
    u_a = g (1 - e^{-3 pi^2 t}) / (3 pi^2); FP32 CG with the fast-diagonalization
    preconditioner at tol 1e-3 and 1e-6, FP64 CG with block-Jacobi at tol 1e-3
    and 1e-10 (the paper's FP64 solver is exact in one iteration).  Advection
    (Sec. 5.2.2): periodic, beta = (1,1,1), the Gaussian bump, exact solution
    the bump translated by beta t; GMRES(30) at tol 1e-3 and 1e-6 in FP32 with
    the complex fast diagonalization at every tau, and in FP64 with it for
    tau >= 1/80 and with block-Jacobi below (the FP64 Fourier passes run on
    the FP64 pipe, about 30x slower, and block-Jacobi converges there).""" 
    import torch

    T = 0.1
    taus = [1.0 / m for m in (10, 20, 40, 80, 160, 320, 640, 1280)]
    out = {}
    for problem in args.paper_sweep.split(","):
        heat = problem == "heat"
        n = args.paper_n or (256 if heat else 200)
        methods = ["midpoint1", "4s3pB", "4s3pC"] + ([] if heat else ["4s3pA"])
        variants = ([("f32", 1e-3), ("f32", 1e-6), ("f64", 1e-3), ("f64", 1e-10)] if heat
                    else [("f32", 1e-3), ("f32", 1e-6), ("f64", 1e-3)])
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
            for tau in taus:
                steps = int(round(T / tau))
                row = {"method": name, "tau": tau, "steps": steps}
                for prec, tol in variants:
                    key = "%s_tol%g" % (prec, tol)
                    if heat:
                        sol = rk.solver_desc(tol_rel=tol, storage=prec, max_iter=3000, correct=1 if prec == "f32" else 0,
                                             precond="fdm" if prec == "f32" else "bj", bj_block=8)
                    else:
                        pre = "fdm" if (prec == "f32" or tau >= 1.0 / 80) else "bj"
                        sol = rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=tol,
                                             storage=prec, max_iter=1000, correct=1 if prec == "f32" else 0,
                                             precond=pre)
                    with rk.Problem(desc, sol, tableau=tab, u0=u0) as p:
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        try:
                            st = rk.rk_integrate(p.h, tau, steps, allow_not_converged=True)
                            u = p.state()
                            err = rel(u, exact) if np.all(np.isfinite(u)) else float("inf")
                            row[key] = {"err": err, "iters_per_solve": st.iters_total / max(st.solves, 1),
                                        "precond": "fdm" if sol.precond == rk.RK_PREC_FDM else "bj",
                                        "not_converged": st.not_converged,
                                        "ms_per_step": 1e3 * (time.perf_counter() - t0) / steps}
                        except rk.RKError as e:
                            row[key] = {"err": None, "status": e.status}
                rows.append(row)
        out[problem] = {"n": n, "rows": rows}
    print(json.dumps({"paper_sweep": out, "T": T, "data": "synthetic",
                      "note": "errors are relative L2 against the analytic solution at T"}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
