"""Guard bands around every device block of a problem (RK_GUARD_BYTES): no
kernel of the tested paths writes outside its buffers.  The substitute for a
device memory checker; the paths are the ones of the parity tests, on small
grids with ragged tiles and odd line lengths."""
import os

import numpy as np
import pytest

import synth
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    lib = require_gpu()
    os.environ["RK_GUARD_BYTES"] = "4096"
    yield lib
    os.environ.pop("RK_GUARD_BYTES", None)


def _check(rk, p):
    bad, blocks = rk.rk_check_guards(p.h)
    assert blocks > 0
    assert bad == 0


HEAT = [(37, "f32", "bj", "sdirk2"), (64, "f32", "bj", "dirk3"), (33, "f16", "bj", "4s3pB"), (21, "bf16", "bj", "sdirk2"),
        (24, "f64", "bj", "dirk3"), (32, "f32", "fdm", "sdirk2"), (24, "f16", "fdm", "sdirk2")]


@pytest.mark.parametrize("n,storage,precond,tab", HEAT)
def test_heat_paths_stay_inside_their_buffers(rk, n, storage, precond, tab):
    u0 = synth.heat_modes(seed=n, n_random=4).evaluate(n)
    sol = rk.solver_desc(bj_block=8, tol_rel=1e-6 if storage in ("f32", "f64") else 1e-3, storage=storage,
                         correct=0 if storage == "f64" else 1, max_iter=2000, precond=precond)
    with rk.Problem(rk.problem_desc(n=n, kappa=1.3), sol, tableau=rk.tableaux.get(tab), u0=u0) as p:
        rk.rk_integrate(p.h, 1e-3, 2, allow_not_converged=True)
        _check(rk, p)


def test_refinement_and_batch_stay_inside_their_buffers(rk):
    n = 29
    u0 = synth.heat_modes(seed=3, n_random=4).evaluate(n)
    sol = rk.solver_desc(bj_block=8, tol_rel=1e-6, storage="f32", correct=1, max_iter=2000, max_refine=3,
                         tol_true=1e-9)
    with rk.Problem(rk.problem_desc(n=n, kappa=2.0), sol, tableau=rk.tableaux.get("dirk3"), u0=u0) as p:
        rk.rk_integrate(p.h, 1e-3, 2, allow_not_converged=True)
        _check(rk, p)
    ps = [rk.Problem(rk.problem_desc(n=m, kappa=1.0),
                     rk.solver_desc(bj_block=8, tol_rel=1e-6, storage="f32", correct=1, max_iter=2000),
                     tableau=rk.tableaux.get("sdirk2"), u0=synth.sine_mode(m)) for m in (5, 17, 40, 64)]
    rk.rk_integrate_batch([p.h for p in ps], 1e-3, 3)
    for p in ps:
        _check(rk, p)
        p.close()


@pytest.mark.parametrize("basis", [None, "bf16"])
def test_gmres_paths_stay_inside_their_buffers(rk, basis):
    n = 19
    kap = synth.kappa_field(n, seed=0)
    kw = {} if basis is None else {"basis": basis}
    sol = rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=1e-7, storage="f32", correct=1,
                         max_iter=800, bj_adapt_tau=1e-2, **kw)
    with rk.Problem(rk.problem_desc(op=rk.RK_OP_ADVDIFF_CSR, n=n, kappa_field=kap, vel=(1.0, 0.5, 0.25)), sol,
                    tableau=rk.tableaux.get("dirk3"), u0=synth.gaussian_bump(n)) as p:
        rk.rk_integrate(p.h, 5e-4, 2, allow_not_converged=True)
        _check(rk, p)


@pytest.mark.parametrize("n", [18, 23])
def test_periodic_fdm_path_stays_inside_its_buffers(rk, n):
    sol = rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=1e-6, storage="f32", correct=1,
                         max_iter=400, precond="fdm")
    with rk.Problem(rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=n, vel=(1.0, 1.0, 1.0)), sol,
                    tableau=rk.tableaux.get("4s3pB"), u0=synth.gaussian_bump_periodic(n)) as p:
        rk.rk_integrate(p.h, 0.05, 2, allow_not_converged=True)
        _check(rk, p)


def test_guards_see_a_changed_guard_byte(rk):
    """The check itself: one guard byte changed through the test hook
    (inside the allocation, host-side) is reported as one corrupted byte."""
    n = 12
    with rk.Problem(rk.problem_desc(n=n, kappa=1.0), rk.solver_desc(bj_block=8, tol_rel=1e-6, storage="f32"),
                    tableau=rk.tableaux.get("sdirk2"), u0=synth.sine_mode(n)) as p:
        assert rk.rk_check_guards(p.h)[0] == 0
        rk.rk_guard_poke(p.h, 0, 7)
        assert rk.rk_check_guards(p.h)[0] == 1
