"""Pins of the oracle's fast-diagonalization preconditioner (Sec. 3, Eqs.
preconbasic, Pinvform, TensorDecomp) against the mathematics: the textbook
sine eigenpairs of tridiag(-1, 2, -1), dense inverses, the operator itself
and the one-iteration convergence of CG with an exact preconditioner."""
import math

import numpy as np
import scipy.sparse as sp
import pytest

from oracle import dirk, fdm, krylov, operators
from synth import SplitMix64

from closed_forms import sine_eigenvalue


def rand_vec(n, seed):
    g = SplitMix64(seed)
    return np.array([g.uniform() - 0.5 for _ in range(n)])


def test_line_eigenpairs_are_the_sine_basis():
    # K1D = tridiag(-1,2,-1) has eigenvectors sin(j k pi/(n+1)) and eigenvalues
    # 4 sin^2(k pi / (2(n+1))), k = 1..n: the LAPACK decomposition must match
    n, kappa, s = 11, 0.7, 3e-3
    P = fdm.FastDiagonalization(n, kappa, s)
    c = s * kappa * (n + 1) ** 2
    mu = np.array([4.0 * math.sin(k * math.pi / (2 * (n + 1))) ** 2 for k in range(1, n + 1)])
    assert np.allclose(P.lam_a, 1.0 + c * mu, rtol=1e-13, atol=0)
    assert np.allclose(P.lam_b, c * mu, rtol=1e-12, atol=0)
    j = np.arange(1, n + 1)
    S = math.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, j) * math.pi / (n + 1))
    # eigenvectors agree up to sign
    for Q in (P.Qa, P.Qb):
        dots = np.abs(np.sum(S * Q, axis=0))
        assert np.allclose(dots, 1.0, atol=1e-12)


def test_pd_holds_the_3d_eigenvalues():
    # P_D entries are 1 - s lambda_m for the sine-mode eigenvalues of L
    n, kappa, s = 7, 1.3, 2e-3
    P = fdm.FastDiagonalization(n, kappa, s)
    for (kx, ky, kz) in [(1, 1, 1), (2, 5, 7), (7, 7, 7), (3, 1, 6)]:
        want = 1.0 - s * sine_eigenvalue(n, kappa, kx, ky, kz)
        assert math.isclose(P.pd[kz - 1, ky - 1, kx - 1], want, rel_tol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 6])
def test_fdm_equals_dense_inverse(n):
    kappa, s = 0.9, 5e-3
    M = np.eye(n ** 3) - s * operators.heat_csr(n, kappa).toarray()
    Minv = np.linalg.inv(M)
    P = fdm.FastDiagonalization(n, kappa, s)
    for seed in range(3):
        r = rand_vec(n ** 3, 100 + seed)
        assert np.allclose(P.apply(r), Minv @ r, rtol=0, atol=1e-12 * np.abs(Minv @ r).max() + 1e-15)


def test_fdm_inverts_the_operator():
    # (I - s L) P^-1 v = v with L applied by the independently pinned stencil
    n, kappa, s = 12, 1.0, 1e-3
    P = fdm.FastDiagonalization(n, kappa, s)
    v = rand_vec(n ** 3, 7)
    w = P.apply(v)
    back = w - s * operators.heat_apply(w, n, kappa)
    assert np.linalg.norm(back - v) <= 1e-12 * np.linalg.norm(v)


def test_fdm_tensor_factors_act_on_the_right_index():
    # Eq. TensorDecomp: T_R contracts i (x), T_M j (y), T_L k (z) of x_{i+jn+kn^2};
    # check each factor against its Kronecker matrix
    n = 4
    Q = np.linalg.qr(np.arange(1.0, n * n + 1).reshape(n, n) ** 0.5)[0]
    I = np.eye(n)
    x = rand_vec(n ** 3, 3)
    x3 = x.reshape(n, n, n)
    assert np.allclose(fdm._t_r(Q, x3).reshape(-1), np.kron(I, np.kron(I, Q)) @ x)
    assert np.allclose(fdm._t_m(Q, x3).reshape(-1), np.kron(I, np.kron(Q, I)) @ x)
    assert np.allclose(fdm._t_l(Q, x3).reshape(-1), np.kron(Q, np.kron(I, I)) @ x)


def test_fdm_is_symmetric_positive_definite():
    n, kappa, s = 4, 1.0, 1e-2
    P = fdm.FastDiagonalization(n, kappa, s)
    Pm = np.column_stack([P.apply(e) for e in np.eye(n ** 3)])
    assert np.allclose(Pm, Pm.T, atol=1e-14)
    assert np.linalg.eigvalsh(Pm).min() > 0


def test_cg_with_fdm_converges_in_one_iteration():
    # an exact preconditioner: the first CG step solves the system
    n, kappa, s = 16, 1.0, 1e-3
    P = fdm.FastDiagonalization(n, kappa, s)
    g = rand_vec(n ** 3, 11)
    apply_A = lambda v: v - s * operators.heat_apply(v, n, kappa)
    res = krylov.pcg(apply_A, P.apply, g, tol_rel=1e-10, max_iter=50)
    assert res.converged and res.iters == 1
    bj = krylov.BlockJacobi(krylov.shifted(operators.heat_csr(n, kappa), s), n, 8)
    res_bj = krylov.pcg(apply_A, bj.apply, g, tol_rel=1e-10, max_iter=500)
    assert res_bj.iters > 5
    assert np.linalg.norm(res.x - res_bj.x) <= 1e-9 * np.linalg.norm(res_bj.x)


def test_planted_mistake_in_pd_is_caught():
    # a dropped direction in P_D breaks the inverse
    n, kappa, s = 6, 1.0, 1e-2
    P = fdm.FastDiagonalization(n, kappa, s)
    P.pd = P.lam_b[None, :, None] + P.lam_a[None, None, :]  # the z direction dropped
    v = rand_vec(n ** 3, 5)
    w = P.apply(v)
    back = w - s * operators.heat_apply(w, n, kappa)
    assert np.linalg.norm(back - v) > 1e-3 * np.linalg.norm(v)


def test_step_with_fdm_matches_block_jacobi_step():
    from oracle import tableau
    n, kappa, dt = 10, 1.0, 1e-3
    op = operators.HeatOperator(n, kappa)
    u0 = rand_vec(n ** 3, 21)
    tab = tableau.get("sdirk2")
    a = dirk.integrate(u0, dt, 3, tab, op, dirk.Solver("cg", bs=4, tol_rel=1e-13))
    b = dirk.integrate(u0, dt, 3, tab, op, dirk.Solver("cg", tol_rel=1e-13, precond="fdm"))
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(a)


@pytest.mark.parametrize("n,beta,s", [(4, (1.0, 1.0, 1.0), 0.1), (6, (1.0, 0.5, 0.25), 0.03), (7, (0.3, 1.0, 2.0), 1.0)])
def test_periodic_fdm_inverts_the_stage_matrix(n, beta, s):
    """The complex fast diagonalization of the periodic advection stage matrix
    is its exact inverse: P^-1 (I - s L) x = x for the independently pinned
    periodic operator, the dense inverse on the smallest grid, and a real
    result for real input."""
    L = operators.adv_periodic_csr(n, beta)
    M = (sp.identity(n ** 3) - s * L).tocsr()
    P = fdm.PeriodicFastDiagonalization(n, beta, s)
    x = np.random.default_rng(n).standard_normal(n ** 3)
    np.testing.assert_allclose(P.apply(M @ x), x, rtol=0, atol=1e-11 * np.abs(x).max())
    if n <= 4:
        np.testing.assert_allclose(P.apply(x), np.linalg.solve(M.toarray(), x), rtol=0, atol=1e-12)


def test_periodic_difference_spectrum_closed_form():
    """The eigenvalues of the periodic central difference are
    i sin(2 pi k / n) / h, k = 0 .. n-1 (Fourier modes)."""
    n = 9
    mu = np.linalg.eigvals(fdm.periodic_difference(n))
    want = 1j * np.sin(2.0 * np.pi * np.arange(n) / n) * n
    np.testing.assert_allclose(np.sort(mu.imag), np.sort(want.imag), atol=1e-10)
    assert np.abs(mu.real).max() < 1e-10


def test_periodic_fdm_solver_one_iteration():
    """GMRES with the oracle's periodic fast diagonalization converges in one
    Arnoldi step (exact preconditioner) and the step with it equals the step
    solved densely."""
    n, s = 6, 0.2
    op = operators.PeriodicOperator(n, (1.0, 0.5, 0.25))
    g = np.random.default_rng(1).standard_normal(n ** 3)
    res = dirk.Solver("gmres", tol_rel=1e-12, precond="fdm").solve(op, s, g)
    assert res.converged and res.iters <= 2
    M = (sp.identity(n ** 3) - s * op.csr()).toarray()
    np.testing.assert_allclose(res.x, np.linalg.solve(M, g), rtol=0, atol=1e-10 * np.abs(g).max())
