"""The paper's own test problems (Sec. 5.2) through the C ABI, against the
float64 oracle and the closed forms: the heat equation with the sine forcing
and u(0) = 0 (Sec. 5.2.1) and periodic advection with central differences
(Sec. 5.2.2), solved with GMRES + block-Jacobi."""
import math

import numpy as np
import pytest

import synth
from closed_forms import forced_sine_after, plane_wave_after
from gpu_util import rel_l2, require_gpu, rng_vec
from oracle import dirk, fdm, krylov, operators, tableau

pytestmark = pytest.mark.gpu

BETA = (1.0, 1.0, 1.0)


@pytest.fixture(scope="module")
def rk():
    return require_gpu()


def periodic(rk, n, storage="f64", bs=8, tol=1e-12, restart=30, correct=None, max_iter=2000, tab=None, u0=None,
             beta=BETA):
    return rk.Problem(rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=n, vel=beta),
                      rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=restart, bj_block=bs, tol_rel=tol,
                                     storage=storage, correct=correct, max_iter=max_iter),
                      tableau=tab, u0=u0)


def forced_heat(rk, n, storage="f64", bs=8, tol=1e-12, correct=None, max_iter=3000, tab=None, precond="bj"):
    return rk.Problem(rk.problem_desc(n=n, kappa=1.0, source=synth.sine_mode(n)),
                      rk.solver_desc(bj_block=bs, tol_rel=tol, storage=storage, correct=correct,
                                     max_iter=max_iter, precond=precond),
                      tableau=tab, u0=np.zeros(n ** 3))


# ---------------------------------------------------------------- periodic advection
@pytest.mark.parametrize("n", [3, 4, 7, 16, 33])
def test_periodic_operator_f64(rk, n):
    beta = (1.0, -0.5, 0.25)
    x = rng_vec(n, n + 40)
    with periodic(rk, n, beta=beta) as p:
        y = np.empty_like(x)
        rk.rk_apply_op(p.h, x, y)
    ref = operators.adv_periodic_csr(n, beta) @ x
    np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("storage,tol", [("f64", 1e-14), ("f32", 2e-6), ("f16", 2e-3)])
def test_periodic_block_jacobi(rk, storage, tol):
    n, bs, shift = 20, 8, 2e-3  # n > bs: the periodic corner of a line stays outside every block
    r = rng_vec(n, 5)
    with periodic(rk, n, storage=storage, bs=bs) as p:
        z = np.empty_like(r)
        rk.rk_apply_precond(p.h, shift, r, z)
    M = krylov.shifted(operators.adv_periodic_csr(n, BETA), shift)
    ref = krylov.BlockJacobi(M, n, bs).apply(r)
    assert rel_l2(z, ref) < tol


@pytest.mark.parametrize("storage,tol,bound", [("f64", 1e-12, 1e-10), ("f32", 1e-7, 1e-6)])
def test_periodic_gmres_solve(rk, storage, tol, bound):
    n, shift = 24, 3e-3
    g = operators.adv_periodic_csr(n, BETA) @ synth.gaussian_bump_periodic(n)
    with periodic(rk, n, storage=storage, bs=8, tol=tol) as p:
        k = np.empty_like(g)
        st = rk.rk_solve(p.h, shift, g, k)
    M = krylov.shifted(operators.adv_periodic_csr(n, BETA), shift)
    x = krylov.gmres(lambda v: M @ v, krylov.BlockJacobi(M, n, 8).apply, g, restart=30, tol_rel=1e-14).x
    assert st.iters_total > 0 and rel_l2(k, x) < bound


@pytest.mark.parametrize("name", ["sdirk2", "dirk3", "4s3pB"])
def test_periodic_plane_wave_closed_form(rk, name):
    """FP64 path: a Fourier mode is advanced by R(dt lambda) per step exactly."""
    n, dt, steps, k = 32, 2e-3, 10, (1, 2, 1)
    A_hi, A_lo, b = tableau.get(name)
    u0 = synth.plane_wave_periodic(n, k)
    with periodic(rk, n, tab=name, u0=u0) as p:
        rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    disc, _ = plane_wave_after(n, BETA, k, dt, steps, A_hi + A_lo, b)
    assert rel_l2(u, disc) < 1e-10


@pytest.mark.parametrize("storage,tol,bound", [("f64", 1e-12, 1e-10), ("f32", 1e-7, 1e-6), ("f16", 1e-3, 5e-3),
                                               ("bf16", 1e-3, 5e-3)])
def test_periodic_bump_step_parity(rk, storage, tol, bound):
    """The Gaussian bump of Sec. 5.2.2, DIRK3, mixed precision vs the FP64
    oracle (same tableau and operator, GMRES to 1e-13)."""
    n, dt, steps = 24, 2e-3, 5
    u0 = synth.gaussian_bump_periodic(n)
    with periodic(rk, n, storage=storage, tol=tol, correct=None if storage == "f64" else 1, tab="dirk3",
                  u0=u0) as p:
        rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
        u = p.state()
    op = operators.CSROperator(n, operators.adv_periodic_csr(n, BETA))
    ref = dirk.integrate(u0, dt, steps, tableau.get("dirk3"), op, dirk.Solver("gmres", bs=8, tol_rel=1e-13))
    assert rel_l2(u, ref) < bound
    assert abs(u.sum() - u0.sum()) < 1e-6 * abs(u0.sum())  # conservation of the skew operator


def test_periodic_rejects_small_grids(rk):
    with pytest.raises(rk.RKError) as e:
        periodic(rk, 2)
    assert e.value.status == rk.RK_ERR_ARG


# ---------------------------------------------------------------- heat with forcing, u(0) = 0
@pytest.mark.parametrize("name", ["sdirk2", "dirk3", "midpoint1"])
def test_forced_heat_fp64_closed_form(rk, name):
    n, dt, steps = 20, 2e-3, 12
    A_hi, A_lo, b = tableau.get(name)
    with forced_heat(rk, n, tab=name) as p:
        rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    disc, _ = forced_sine_after(n, 1.0, dt, steps, A_hi + A_lo, b)
    assert rel_l2(u, disc) < 1e-10


@pytest.mark.parametrize("storage,precond,tol,bound", [("f32", "bj", 1e-7, 1e-6), ("f32", "fdm", 1e-7, 1e-6),
                                                       ("f16", "bj", 1e-3, 5e-3), ("bf16", "fdm", 1e-3, 5e-3)])
def test_forced_heat_mixed_vs_oracle(rk, storage, precond, tol, bound):
    n, dt, steps = 32, 1e-3, 10
    g = synth.sine_mode(n)
    with forced_heat(rk, n, storage=storage, tol=tol, correct=1, tab="sdirk2", precond=precond) as p:
        rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
        u = p.state()
    ref = dirk.integrate(np.zeros(n ** 3), dt, steps, tableau.get("sdirk2"), operators.HeatOperator(n, 1.0),
                         dirk.Solver("cg", bs=8, tol_rel=1e-13), source=g)
    assert rel_l2(u, ref) < bound


def test_forced_heat_apply_op_excludes_the_forcing(rk):
    n = 12
    x = rng_vec(n, 3)
    with forced_heat(rk, n) as p:
        y = np.empty_like(x)
        rk.rk_apply_op(p.h, x, y)
    np.testing.assert_allclose(y, operators.heat_apply(x, n, 1.0), rtol=1e-13, atol=1e-9)


def test_forced_heat_paper_solution_256(rk):
    """The heat test of Sec. 5.2.1 at 256^3 to t = 0.02 with FP32 + FDM: the
    fully discrete closed form holds, and the distance to the paper's
    analytic u_a is the discretisation error."""
    n, dt, steps = 256, 1e-3, 20
    A_hi, A_lo, b = tableau.get("sdirk2")
    with forced_heat(rk, n, storage="f32", tol=1e-6, correct=1, tab="sdirk2", precond="fdm") as p:
        st = rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    disc, _ = forced_sine_after(n, 1.0, dt, steps, A_hi + A_lo, b)
    ua = synth.sine_mode(n) * (1.0 - math.exp(-3.0 * math.pi ** 2 * dt * steps)) / (3.0 * math.pi ** 2)
    assert rel_l2(u, disc) < 1e-6
    assert rel_l2(u, ua) < 5e-5 and st.iters_max <= 8  # closed forms: 2.94e-5


def test_forced_problems_rejected_by_batch(rk):
    with forced_heat(rk, 16, storage="f32", tol=1e-6, tab="sdirk2") as p:
        with pytest.raises(rk.RKError) as e:
            rk.rk_integrate_batch([p.h], 1e-3, 1)
        assert e.value.status == rk.RK_ERR_ARG


# ------------------------------------------- complex fast diagonalization (periodic)
def periodic_fdm(rk, n, storage="f32", tol=1e-7, correct=None, tab=None, u0=None, beta=BETA, max_iter=200,
                 basis=None):
    kw = {} if basis is None else {"basis": basis}
    return rk.Problem(rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=n, vel=beta),
                      rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, tol_rel=tol, storage=storage,
                                     correct=correct, max_iter=max_iter, precond="fdm", **kw),
                      tableau=tab, u0=u0)


@pytest.mark.parametrize("n,beta,shift,storage,bound", [(20, BETA, 0.05, "f32", 2e-6), (33, (1.0, 0.5, 0.25), 0.3, "f32", 2e-6),
                                                        (17, BETA, 0.1, "f64", 1e-12), (64, BETA, 0.1, "f32", 2e-6),
                                                        (20, (1.0, 0.5, 0.25), 0.3, "f64", 1e-12),
                                                        (32, BETA, 0.1, "f64", 1e-12), (200, BETA, 0.1, "f32", 2e-6)])
def test_periodic_fdm_apply_matches_oracle(rk, n, beta, shift, storage, bound):
    """The six complex Fourier passes apply P^-1 of the periodic advection
    stage matrix: against the oracle's fast diagonalization (LAPACK Schur
    basis), for grids that fill the 32-line tiles and grids that do not.
    n = 20, 32, 64 and 200 run the compile-time small transforms (FP32 and
    FP64); n = 17 and 33 (a prime and 3 x 11) the table passes."""
    r = synth.gaussian_bump_periodic(n) + 0.1 * np.random.default_rng(n).standard_normal(n ** 3)
    with periodic_fdm(rk, n, storage=storage, beta=beta) as p:
        z = np.empty_like(r)
        rk.rk_apply_precond(p.h, shift, r, z)
    ref = fdm.PeriodicFastDiagonalization(n, beta, shift).apply(r)
    assert rel_l2(z, ref) < bound


@pytest.mark.parametrize("storage,tol,bound", [("f32", 1e-7, 1e-6), ("f64", 1e-12, 1e-10)])
def test_periodic_fdm_gmres_few_iterations(rk, storage, tol, bound):
    """GMRES preconditioned by the exact inverse converges in a handful of
    iterations even at a large step (where block-Jacobi GMRES stalls), to the
    oracle's dense-accuracy solution."""
    n, shift = 24, 0.1 * 0.4358665215
    g = operators.adv_periodic_csr(n, BETA) @ synth.gaussian_bump_periodic(n)
    with periodic_fdm(rk, n, storage=storage, tol=tol) as p:
        k = np.empty_like(g)
        st = rk.rk_solve(p.h, shift, g, k)
    M = krylov.shifted(operators.adv_periodic_csr(n, BETA), shift)
    ref = fdm.PeriodicFastDiagonalization(n, BETA, shift).apply(g)
    np.testing.assert_allclose(M @ ref, g, rtol=0, atol=1e-10 * np.abs(g).max())
    assert rel_l2(k, ref) < bound
    assert st.iters_total <= 4


def test_periodic_fdm_step_large_tau_vs_oracle(rk):
    """A mixed-precision DIRK3 step of the Gaussian bump at tau = 1/10 (beyond
    block-Jacobi GMRES): the FP32 solves with the complex fast diagonalization
    stay within the FP32 bound of the oracle's FP64 step."""
    n, dt, steps = 32, 0.1, 2
    u0 = synth.gaussian_bump_periodic(n)
    with periodic_fdm(rk, n, tol=1e-8, correct=1, tab="dirk3", u0=u0) as p:
        st = rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    ref = dirk.integrate(u0, dt, steps, tableau.dirk3(), operators.PeriodicOperator(n, BETA),
                         dirk.Solver("gmres", tol_rel=1e-13, restart=30, precond="fdm"))
    assert rel_l2(u, ref) < 1e-6
    assert st.iters_total <= 8 * st.solves
