"""Pins for oracle.dirk: the whole step against R(tau L) (Sec. 2.3) by dense
eigendecomposition (heat) and by the Kronecker stage system of Eq. RKstep
(advection-diffusion), the sine-mode closed form, observed temporal order,
axis-permutation symmetry, and the plain/corrected forms."""
import math

import numpy as np
import pytest

import synth
from oracle import dirk, operators, tableau
from closed_forms import R_scalar, mode_sum_after, rel_l2, sine_eigenvalue

ALL = ["midpoint1", "midpoint2", "sdirk2", "dirk3", "4s3pA", "4s3pB", "4s3pC"]


@pytest.mark.parametrize("name", ALL)
def test_heat_step_equals_R_of_eigenvalues(name):
    n, kappa, dt, steps = 5, 0.8, 4e-3, 3
    op = operators.HeatOperator(n, kappa)
    A_hi, A_lo, b = tableau.get(name)
    L = op.csr().toarray()
    lam, Q = np.linalg.eigh(L)
    u0 = np.random.default_rng(7).standard_normal(n ** 3)
    Rl = np.array([R_scalar(A_hi + A_lo, b, dt * l).real for l in lam])
    exact = Q @ (Rl ** steps * (Q.T @ u0))
    got = dirk.integrate(u0, dt, steps, (A_hi, A_lo, b), op, dirk.Solver("cg", bs=3, tol_rel=1e-14))
    assert rel_l2(got, exact) < 1e-11


@pytest.mark.parametrize("name", ["sdirk2", "dirk3", "4s3pB", "midpoint1"])
def test_advdiff_step_equals_kronecker_stage_system(name):
    n, dt = 4, 2e-3
    L = operators.advdiff_csr(n, synth.kappa_field(n, seed=9), (1.0, 0.5, 0.25))
    op = operators.CSROperator(n, L)
    A_hi, A_lo, b = tableau.get(name)
    A = A_hi + A_lo
    q, N = len(b), n ** 3
    Ld = L.toarray()
    u0 = synth.gaussian_bump(n) + 0.1 * np.random.default_rng(2).standard_normal(N)
    # Eq. RKstep for f(u) = L u: K = (I_q (x) L)(e (x) u + tau (A (x) I) K)
    big = np.eye(q * N) - dt * np.kron(A, Ld)
    K = np.linalg.solve(big, np.kron(np.ones(q), Ld @ u0)).reshape(q, N)
    exact = u0 + dt * (b @ K)
    got = dirk.rk_step(u0, dt, (A_hi, A_lo, b), op, dirk.Solver("gmres", bs=2, tol_rel=1e-14, restart=10))
    assert rel_l2(got, exact) < 1e-11


@pytest.mark.parametrize("name", ["sdirk2", "dirk3", "4s3pC"])
def test_sine_mode_sum_closed_form(name):
    n, kappa, dt, steps = 12, 1.0, 1e-3, 5
    modes = synth.heat_modes(seed=0, n_random=6).modes
    u0 = synth.ModeSum(modes).evaluate(n)
    A_hi, A_lo, b = tableau.get(name)
    got = dirk.integrate(u0, dt, steps, (A_hi, A_lo, b), operators.HeatOperator(n, kappa),
                         dirk.Solver("cg", bs=4, tol_rel=1e-13))
    exact = mode_sum_after(modes, n, kappa, dt, steps, A_hi + A_lo, b)
    assert rel_l2(got, exact) < 1e-11


@pytest.mark.parametrize("name,order", [("midpoint1", 2), ("sdirk2", 2), ("dirk3", 3), ("4s3pB", 3), ("4s3pC", 3)])
def test_observed_temporal_order(name, order):
    """Semi-discrete exact solution exp(lambda t) phi for one sine mode."""
    n, kappa, T = 6, 1.0, 0.2
    op = operators.HeatOperator(n, kappa)
    phi = synth.sine_mode(n, 1, 1, 1)
    lam = sine_eigenvalue(n, kappa, 1, 1, 1)
    exact = math.exp(lam * T) * phi
    errs = []
    for nsteps in (80, 160, 320):
        u = dirk.integrate(phi, T / nsteps, nsteps, tableau.get(name), op, dirk.Solver("cg", bs=6, tol_rel=1e-14))
        errs.append(np.linalg.norm(u - exact))
    p1 = math.log2(errs[0] / errs[1])
    p2 = math.log2(errs[1] / errs[2])
    assert abs(p2 - order) < 0.1 and abs(p1 - order) < 0.15, (errs, p1, p2)


def test_axis_permutation_symmetry():
    n = 7
    x, y, z = synth.grid_coords(n)
    u0 = (np.sin(math.pi * x) * np.sin(math.pi * y) * np.sin(math.pi * z) * (1 + x * y * z)).ravel()
    u = dirk.integrate(u0, 2e-3, 3, tableau.get("dirk3"), operators.HeatOperator(n, 1.0),
                       dirk.Solver("cg", bs=7, tol_rel=1e-14))
    U = u.reshape(n, n, n)
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)]:
        np.testing.assert_allclose(U, U.transpose(perm), atol=1e-12 * np.abs(U).max())


def test_plain_and_corrected_agree_to_solver_tolerance():
    n = 10
    op = operators.HeatOperator(n, 1.0)
    u0 = synth.heat_modes(seed=1, n_random=4).evaluate(n)
    s = dirk.Solver("cg", bs=5, tol_rel=1e-13)
    a = dirk.integrate(u0, 1e-3, 4, tableau.get("4s3pB"), op, s, corrected=True)
    b = dirk.integrate(u0, 1e-3, 4, tableau.get("4s3pB"), op, s, corrected=False)
    assert rel_l2(a, b) < 1e-10


def test_continuous_decay_config1_shape():
    """32^3, SDIRK2, dt = 1e-3, 20 steps: close to exp(-3 pi^2 t) u0 (spatial
    plus temporal error) and equal to R(dt lambda_1)^20 u0 to solver accuracy."""
    n = 32
    u0 = synth.sine_mode(n)
    A_hi, A_lo, b = tableau.sdirk2()
    u = dirk.integrate(u0, 1e-3, 20, (A_hi, A_lo, b), operators.HeatOperator(n, 1.0),
                       dirk.Solver("cg", bs=1, tol_rel=1e-12))
    lam = sine_eigenvalue(n, 1.0, 1, 1, 1)
    assert rel_l2(u, R_scalar(A_hi + A_lo, b, 1e-3 * lam).real ** 20 * u0) < 1e-11
    assert rel_l2(u, math.exp(-3 * math.pi ** 2 * 0.02) * u0) < 5e-3


def test_planted_dropped_term_is_caught():
    """Dropping the low-precision history term a^eps_ij k^eps_j (j < i) from
    the stage right-hand side must break the closed-form pin for 4s3pB."""
    n, dt = 5, 1e-2
    op = operators.HeatOperator(n, 1.0)
    A_hi, A_lo, b = tableau.m4s3pB()
    broken = (A_hi, np.diag(np.diag(A_lo)), b)
    phi = synth.sine_mode(n)
    lam = sine_eigenvalue(n, 1.0, 1, 1, 1)
    got = dirk.rk_step(phi, dt, broken, op, dirk.Solver("cg", bs=5, tol_rel=1e-14))
    assert rel_l2(got, R_scalar(A_hi + A_lo, b, dt * lam).real * phi) > 1e-3
