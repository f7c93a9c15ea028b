"""Serving with continuous batching: jobs admitted by HBM footprint, stepped
together, and each result the same alone and in the mix."""
import time

import numpy as np
import pytest

import synth
from closed_forms import rel_l2
from gpu_util import require_gpu
from oracle import dirk, operators, tableau

pytestmark = pytest.mark.gpu
BOUND = {"f32": 1e-6, "f16": 5e-3}


@pytest.fixture(scope="module")
def rk():
    return require_gpu()


def job_args(rk, n, kappa, tab, storage, seed):
    desc = rk.problem_desc(n=n, kappa=kappa)
    sol = rk.solver_desc(bj_block=8, tol_rel={"f32": 1e-7, "f16": 1e-3}[storage], storage=storage, max_iter=2000)
    u0 = synth.heat_modes(seed=seed, n_random=4).evaluate(n)
    return desc, sol, rk.tableaux.get(tab), u0


# (n, kappa, tableau, storage).  The midpoint jobs (|R(-inf)| = 1, no damping
# of solver noise) stay at dt*||L|| <= 20: their correction stage amplifies the
# rounding of k^eps by about (dt lambda)^2 / 2 per step (Sec. 2.1).
MIX = [(24, 1.0, "sdirk2", "f32"), (40, 0.5, "dirk3", "f32"), (96, 1.0, "sdirk2", "f32"),
       (17, 3.0, "midpoint1", "f16"), (64, 0.2, "dirk3", "f16"), (80, 0.2, "midpoint1", "f32"),
       (33, 1.0, "sdirk2", "f32"), (12, 7.0, "dirk3", "f32")]


def solo(rk, n, kappa, tab, storage, seed, dt, steps):
    desc, sol, t, u0 = job_args(rk, n, kappa, tab, storage, seed)
    with rk.Problem(desc, sol, tableau=t, u0=u0) as p:
        rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
        return p.state()


def oracle_run(n, kappa, tab, seed, dt, steps):
    """The FP64 oracle on the same seeded problem, solved to 1e-13."""
    u0 = synth.heat_modes(seed=seed, n_random=4).evaluate(n)
    return dirk.integrate(u0, dt, steps, tableau.get(tab), operators.HeatOperator(n, kappa),
                          dirk.Solver("cg", bs=8, tol_rel=1e-13, max_iter=5000))


def test_results_same_alone_and_in_mix(rk):
    """Jobs submitted back to back share the device (their step ranges overlap
    in the server's ticks); every result equals the job run alone through
    the server and through rk_integrate, and the FP64 oracle within the
    precision pair's bound."""
    dt = 1e-3
    steps = [3, 5, 4, 6, 2, 3, 5, 4]
    srv = rk.rk_server_create(8 << 30, 16)
    try:
        # the first job alone
        n, kap, tab, st = MIX[0]
        d, s, t, u0 = job_args(rk, n, kap, tab, st, 0)
        jid = rk.rk_submit_job(srv, d, s, *t, u0, dt, steps[0])
        alone = np.empty(n ** 3)
        rk.rk_wait_job(srv, jid, alone, allow_not_converged=True)
        # the whole mix, submitted back to back so that jobs overlap
        ids = []
        for i, (n, kap, tab, st) in enumerate(MIX):
            d, s, t, u0 = job_args(rk, n, kap, tab, st, i)
            ids.append(rk.rk_submit_job(srv, d, s, *t, u0, dt, steps[i]))
        outs, infos = [], []
        for i, jid in enumerate(ids):
            out = np.empty(MIX[i][0] ** 3)
            stats, info = rk.rk_wait_job_info(srv, jid, out, allow_not_converged=True)
            outs.append(out)
            infos.append(info)
    finally:
        rk.rk_server_destroy(srv)
    assert rel_l2(outs[0], alone) < BOUND["f32"]
    for i, info in enumerate(infos):
        assert info.steps == steps[i]
        assert 0.0 <= info.t_submit <= info.t_admit <= info.t_first_step <= info.t_done
        assert info.last_tick - info.first_tick + 1 >= steps[i]
    # co-residency: the jobs whose tick ranges overlap the longest job's were
    # stepped in the same rounds, i.e. concurrently on the device
    longest = int(np.argmax(steps))
    lo, hi = infos[longest].first_tick, infos[longest].last_tick
    together = [i for i, f in enumerate(infos) if f.first_tick <= hi and f.last_tick >= lo]
    assert len(together) >= 4, [(f.first_tick, f.last_tick) for f in infos]
    for i, (n, kap, tab, st) in enumerate(MIX):
        ref = solo(rk, n, kap, tab, st, i, dt, steps[i])
        assert rel_l2(outs[i], ref) < BOUND[st], (i, n, tab, st)
        exact = oracle_run(n, kap, tab, i, dt, steps[i])
        assert rel_l2(outs[i], exact) < BOUND[st], (i, n, tab, st, rel_l2(outs[i], exact))


def test_admission_under_budget_and_errors(rk):
    dt = 1e-3
    n = 48
    d, s, t, u0 = job_args(rk, n, 1.0, "sdirk2", "f32", 3)
    one = 8 * n ** 3 * 3 + 4 * n ** 3 * 4 + 8 * n ** 3 * 2 + 4 * n ** 3 * 3 + (1 << 20)
    srv = rk.rk_server_create(int(2.5 * one), 4)  # about two jobs resident at a time
    try:
        ids = [rk.rk_submit_job(srv, d, s, *t, u0, dt, 2) for _ in range(5)]
        outs = []
        for jid in ids:
            out = np.empty(n ** 3)
            rk.rk_wait_job(srv, jid, out)
            outs.append(out)
        for o in outs[1:]:
            assert rel_l2(o, outs[0]) < 1e-6
        big = rk.problem_desc(n=256, kappa=1.0)
        with pytest.raises(rk.RKError) as e:
            rk.rk_submit_job(srv, big, s, *t, synth.sine_mode(256), dt, 1)
        assert e.value.status == rk.RK_ERR_OOM
        with pytest.raises(rk.RKError) as e:
            rk.rk_poll_job(srv, 123456)
        assert e.value.status == rk.RK_ERR_NOT_FOUND
    finally:
        rk.rk_server_destroy(srv)


def test_poll_reports_completion(rk):
    srv = rk.rk_server_create(1 << 30, 4)
    try:
        d, s, t, u0 = job_args(rk, 16, 1.0, "sdirk2", "f32", 1)
        jid = rk.rk_submit_job(srv, d, s, *t, u0, 1e-3, 2)
        t0 = time.time()
        while not rk.rk_poll_job(srv, jid):
            assert time.time() - t0 < 60
            time.sleep(0.01)
        st, lat = rk.rk_wait_job(srv, jid)
        assert st.solves >= 1 and lat > 0
    finally:
        rk.rk_server_destroy(srv)


def test_new_problem_kinds_same_alone_and_in_mix(rk):
    """Jobs of every operator and solver option through the server -- periodic
    advection (GMRES), heat with a forcing term, the tensor-core
    fast-diagonalization preconditioner, a compressed GMRES basis -- mixed with
    plain heat jobs: each result equals the same problem stepped alone."""
    dt, steps = 1e-3, 3
    beta = (1.0, 1.0, 1.0)
    jobs = [
        (rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=24, vel=beta),
         rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, bj_block=8, tol_rel=1e-8, storage="f32", max_iter=2000),
         "dirk3", synth.gaussian_bump_periodic(24)),
        (rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=20, vel=beta),
         rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, bj_block=8, tol_rel=1e-8, storage="f32", max_iter=2000,
                        basis="bf16"),
         "sdirk2", synth.gaussian_bump_periodic(20)),
        (rk.problem_desc(n=32, kappa=1.0, source=synth.sine_mode(32)),
         rk.solver_desc(bj_block=8, tol_rel=1e-7, storage="f32", max_iter=2000),
         "sdirk2", np.zeros(32 ** 3)),
        (rk.problem_desc(n=64, kappa=1.0),
         rk.solver_desc(tol_rel=1e-7, storage="f32", max_iter=200, precond="fdm"),
         "dirk3", synth.heat_modes(seed=5, n_random=4).evaluate(64)),
        (rk.problem_desc(n=40, kappa=0.5),
         rk.solver_desc(bj_block=8, tol_rel=1e-7, storage="f32", max_iter=2000),
         "sdirk2", synth.heat_modes(seed=6, n_random=4).evaluate(40)),
    ]
    srv = rk.rk_server_create(8 << 30, 8)
    try:
        ids = [rk.rk_submit_job(srv, d, s, *rk.tableaux.get(t), u0, dt, steps) for d, s, t, u0 in jobs]
        outs = []
        for (d, s, t, u0), jid in zip(jobs, ids):
            out = np.empty(d.n ** 3)
            rk.rk_wait_job(srv, jid, out, allow_not_converged=True)
            outs.append(out)
    finally:
        rk.rk_server_destroy(srv)
    oracles = [
        lambda: dirk.integrate(jobs[0][3], dt, steps, tableau.get("dirk3"),
                               operators.CSROperator(24, operators.adv_periodic_csr(24, beta)),
                               dirk.Solver("gmres", bs=8, tol_rel=1e-13, max_iter=5000)),
        lambda: dirk.integrate(jobs[1][3], dt, steps, tableau.get("sdirk2"),
                               operators.CSROperator(20, operators.adv_periodic_csr(20, beta)),
                               dirk.Solver("gmres", bs=8, tol_rel=1e-13, max_iter=5000)),
        lambda: dirk.integrate(jobs[2][3], dt, steps, tableau.get("sdirk2"), operators.HeatOperator(32, 1.0),
                               dirk.Solver("cg", bs=8, tol_rel=1e-13), source=synth.sine_mode(32)),
        lambda: dirk.integrate(jobs[3][3], dt, steps, tableau.get("dirk3"), operators.HeatOperator(64, 1.0),
                               dirk.Solver("cg", tol_rel=1e-13, precond="fdm")),
        lambda: dirk.integrate(jobs[4][3], dt, steps, tableau.get("sdirk2"), operators.HeatOperator(40, 0.5),
                               dirk.Solver("cg", bs=8, tol_rel=1e-13)),
    ]
    for (d, s, t, u0), out, orc in zip(jobs, outs, oracles):
        with rk.Problem(d, s, tableau=t, u0=u0) as p:
            rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
            ref = p.state()
        assert rel_l2(out, ref) < 1e-6, (d.op, d.n)
        # FP32 solves (BF16 basis for the compressed GMRES job) against the oracle
        assert rel_l2(out, orc()) < 1e-6, (d.op, d.n)


def test_nonfinite_job_fails_alone(rk):
    """A job whose state turns non-finite fails with RK_ERR_NONFINITE; jobs
    submitted with it (batched with it when they share a tick) complete and
    match the oracle."""
    dt, steps = 1e-3, 4
    srv = rk.rk_server_create(8 << 30, 16)
    try:
        good = [(24, 1.0, "sdirk2", "f32"), (40, 0.5, "dirk3", "f32"), (32, 2.0, "sdirk2", "f32")]
        d, s, t, _u = job_args(rk, 28, 1.0, "sdirk2", "f32", 0)
        bad_u0 = synth.sine_mode(28)
        bad_u0[5] = np.nan
        ids = [rk.rk_submit_job(srv, d, s, *t, bad_u0, dt, steps)]
        for i, (n, kap, tab, st) in enumerate(good):
            dd, ss, tt, u0 = job_args(rk, n, kap, tab, st, 60 + i)
            ids.append(rk.rk_submit_job(srv, dd, ss, *tt, u0, dt, steps))
        with pytest.raises(rk.RKError) as e:
            rk.rk_wait_job(srv, ids[0], None)
        assert e.value.status == rk.RK_ERR_NONFINITE
        for jid, (i, (n, kap, tab, st)) in zip(ids[1:], enumerate(good)):
            out = np.empty(n ** 3)
            rk.rk_wait_job(srv, jid, out, allow_not_converged=True)
            ref = oracle_run(n, kap, tab, 60 + i, dt, steps)
            assert rel_l2(out, ref) < BOUND[st], (n, tab)
    finally:
        rk.rk_server_destroy(srv)
