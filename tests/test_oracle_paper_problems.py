"""Pins of the oracle on the paper's own test problems (Sec. 5.2): the heat
equation with the sine forcing and zero initial state (Sec. 5.2.1) and the
periodic advection equation with central differences (Sec. 5.2.2)."""
import math

import numpy as np
import pytest

import synth
from closed_forms import forced_sine_after, periodic_wave_eigenvalue, plane_wave_after
from oracle import dirk, operators, tableau

BETA = (1.0, 1.0, 1.0)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------- periodic advection operator
def test_periodic_operator_brute_force():
    # loop evaluation of -sum_d beta_d (u(x+h e_d) - u(x-h e_d)) / (2h), periodic
    n, beta = 5, (1.0, -0.7, 0.3)
    L = operators.adv_periodic_csr(n, beta)
    u = np.random.default_rng(1).standard_normal(n ** 3)
    U = u.reshape(n, n, n)
    out = np.zeros_like(U)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                s = 0.0
                s -= beta[0] * (U[k, j, (i + 1) % n] - U[k, j, (i - 1) % n]) * n / 2.0
                s -= beta[1] * (U[k, (j + 1) % n, i] - U[k, (j - 1) % n, i]) * n / 2.0
                s -= beta[2] * (U[(k + 1) % n, j, i] - U[(k - 1) % n, j, i]) * n / 2.0
                out[k, j, i] = s
    assert np.allclose(L @ u, out.ravel(), rtol=0, atol=1e-12)


def test_periodic_operator_is_skew_and_conservative():
    n = 7
    L = operators.adv_periodic_csr(n, BETA)
    assert abs(L + L.T).max() < 1e-12  # skew-symmetric: energy conserving
    assert np.allclose(np.asarray(L.sum(axis=1)).ravel(), 0.0)  # constants are in the kernel
    assert np.allclose(np.asarray(L.sum(axis=0)).ravel(), 0.0)  # sum(u) is conserved
    assert L.diagonal().max() == 0.0


@pytest.mark.parametrize("k", [(1, 0, 0), (1, 1, 1), (2, 3, 1), (4, 0, 5)])
def test_periodic_operator_fourier_eigenvalues(k):
    n = 12
    L = operators.adv_periodic_csr(n, BETA)
    x, y, z = synth.periodic_coords(n)
    phi = np.exp(2j * math.pi * (k[0] * x + k[1] * y + k[2] * z)).ravel()
    lam = periodic_wave_eigenvalue(n, BETA, k)
    assert abs(lam.real) == 0.0
    assert np.allclose(L @ phi, lam * phi, atol=1e-10)


def test_periodic_operator_commutes_with_grid_shifts():
    n = 6
    L = operators.adv_periodic_csr(n, (1.0, 0.5, 0.25))
    u = np.random.default_rng(2).standard_normal(n ** 3)
    shift = lambda v: np.roll(v.reshape(n, n, n), (1, 2, 3), axis=(0, 1, 2)).ravel()
    assert np.allclose(L @ shift(u), shift(L @ u), atol=1e-12)


def test_planted_sign_error_breaks_the_eigenvalue_pin():
    n, k = 10, (1, 2, 0)
    L = -operators.adv_periodic_csr(n, BETA)  # advection in the wrong direction
    x, y, z = synth.periodic_coords(n)
    phi = np.exp(2j * math.pi * (k[0] * x + k[1] * y + k[2] * z)).ravel()
    lam = periodic_wave_eigenvalue(n, BETA, k)
    assert not np.allclose(L @ phi, lam * phi, atol=1e-6)


# ---------------------------------------------------------------- stepping, closed forms
@pytest.mark.parametrize("name", ["sdirk2", "dirk3", "4s3pB"])
def test_oracle_plane_wave_matches_closed_form(name):
    n, dt, steps, k = 8, 4e-3, 10, (1, 1, 0)
    L = operators.adv_periodic_csr(n, BETA)
    op = operators.CSROperator(n, L)
    u0 = synth.plane_wave_periodic(n, k)
    A_hi, A_lo, b = tableau.get(name)
    u = dirk.integrate(u0, dt, steps, (A_hi, A_lo, b), op, dirk.Solver("gmres", bs=4, tol_rel=1e-13))
    disc, _ = plane_wave_after(n, BETA, k, dt, steps, A_hi + A_lo, b)
    assert rel(u, disc) < 1e-10


@pytest.mark.parametrize("name", ["sdirk2", "dirk3", "midpoint1"])
def test_oracle_forced_heat_matches_closed_form(name):
    # Sec. 5.2.1: u_t = Lap u + g, g the sine mode, u(0) = 0
    n, dt, steps = 9, 2e-3, 15
    op = operators.HeatOperator(n, 1.0)
    g = synth.sine_mode(n)
    A_hi, A_lo, b = tableau.get(name)
    u = dirk.integrate(np.zeros(n ** 3), dt, steps, (A_hi, A_lo, b), op, dirk.Solver("cg", bs=3, tol_rel=1e-13),
                       source=g)
    disc, _ = forced_sine_after(n, 1.0, dt, steps, A_hi + A_lo, b)
    assert rel(u, disc) < 1e-10


def test_forced_heat_closed_form_approaches_the_paper_solution():
    # as h, dt -> 0 the discrete solution tends to u_a = g (1 - e^{-3 pi^2 t}) / (3 pi^2)
    t = 0.1
    errs = []
    for n, dt in ((15, 0.01), (31, 0.005), (63, 0.0025)):
        A_hi, A_lo, b = tableau.get("sdirk2")
        disc, _ = forced_sine_after(n, 1.0, dt, int(round(t / dt)), A_hi + A_lo, b)
        ua = synth.sine_mode(n) * (1.0 - math.exp(-3.0 * math.pi ** 2 * t)) / (3.0 * math.pi ** 2)
        errs.append(rel(disc, ua))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3
    assert errs[0] / errs[1] > 3.0  # second order in h and dt


def test_oracle_forced_heat_temporal_order():
    # against the semi-discrete exact solution (no spatial error): order 2 for SDIRK2
    n = 7
    op = operators.HeatOperator(n, 1.0)
    g = synth.sine_mode(n)
    tab = tableau.get("sdirk2")
    errs = []
    for steps in (10, 20, 40):
        dt = 0.04 / steps
        u = dirk.integrate(np.zeros(n ** 3), dt, steps, tab, op, dirk.Solver("cg", bs=7, tol_rel=1e-14), source=g)
        _, cont = forced_sine_after(n, 1.0, dt, steps, tab[0] + tab[1], tab[2])
        errs.append(rel(u, cont))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < o < 2.3 for o in orders), orders


def test_oracle_periodic_mixed_step_stays_close_to_fp64():
    # the Gaussian bump of Sec. 5.2.2 advected a few steps; GMRES to 1e-13
    n, dt = 10, 5e-3
    L = operators.adv_periodic_csr(n, BETA)
    op = operators.CSROperator(n, L)
    u0 = synth.gaussian_bump_periodic(n)
    u = dirk.integrate(u0, dt, 6, tableau.get("dirk3"), op, dirk.Solver("gmres", bs=5, tol_rel=1e-13))
    # skew L: the discrete energy changes only by the damping of the L-stable method
    assert np.linalg.norm(u) <= np.linalg.norm(u0) + 1e-12
    assert abs(u.sum() - u0.sum()) < 1e-9 * abs(u0.sum())
