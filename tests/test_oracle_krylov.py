"""Pins for oracle.krylov: dense direct solves, exact-preconditioner and
small-dimension termination, GMRES residual monotonicity, block layout."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import krylov, operators


def _heat_system(n, kappa, s):
    return krylov.shifted(operators.heat_csr(n, kappa), s)


@pytest.mark.parametrize("n,bs", [(3, 1), (5, 2), (6, 4), (6, 8)])
def test_pcg_matches_dense_solve(n, bs):
    M = _heat_system(n, 1.3, 2e-2)
    g = np.random.default_rng(0).standard_normal(n ** 3)
    bj = krylov.BlockJacobi(M, n, bs)
    res = krylov.pcg(lambda v: M @ v, bj.apply, g, tol_rel=1e-14, max_iter=500)
    assert res.converged
    x = np.linalg.solve(M.toarray(), g)
    np.testing.assert_allclose(res.x, x, rtol=0, atol=1e-11 * np.abs(x).max())


def test_pcg_n1_one_iteration():
    M = _heat_system(1, 1.0, 0.1)
    res = krylov.pcg(lambda v: M @ v, lambda r: r, np.array([2.0]), tol_rel=1e-15)
    assert res.iters == 1 and res.converged
    assert res.x[0] == pytest.approx(2.0 / M[0, 0], rel=1e-15)


def test_pcg_exact_preconditioner_one_iteration():
    # blocks = whole x-lines and no y/z coupling (n = 1 in y and z is impossible
    # on a cube), so use a matrix whose only couplings are along x
    n = 5
    T = sp.diags([-np.ones(n - 1), 3 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    M = sp.kron(sp.identity(n * n), T).tocsr()
    bj = krylov.BlockJacobi(M, n, n)
    g = np.arange(n ** 3, dtype=float)
    res = krylov.pcg(lambda v: M @ v, bj.apply, g, tol_rel=1e-13)
    assert res.iters == 1 and res.converged


@pytest.mark.parametrize("n,bs", [(7, 3), (8, 8), (5, 1)])
def test_block_jacobi_layout_and_blocks(n, bs):
    M = _heat_system(n, 1.0, 1e-2)
    bj = krylov.BlockJacobi(M, n, bs)
    covered = np.concatenate([(starts[:, None] + np.arange(m)[None, :]).ravel() for m, starts, _ in bj.groups])
    assert sorted(covered.tolist()) == list(range(n ** 3))
    # applying to M e restricted to a block returns the block-local part exactly
    D = np.zeros((n ** 3, n ** 3))
    for m, starts, inv in bj.groups:
        for s0, B in zip(starts, inv):
            D[s0:s0 + m, s0:s0 + m] = np.linalg.inv(B)
    Md = M.toarray()
    mask = D != 0
    np.testing.assert_allclose(D[mask], Md[mask], atol=1e-12)
    r = np.random.default_rng(1).standard_normal(n ** 3)
    np.testing.assert_allclose(D @ bj.apply(r), r, atol=1e-10)


@pytest.mark.parametrize("n,vel", [(4, (1.0, 0.5, 0.25)), (5, (-2.0, 1.0, 0.0))])
def test_gmres_matches_dense_solve(n, vel):
    L = operators.advdiff_csr(n, synth.kappa_field(n, seed=2), vel)
    M = krylov.shifted(L, 1e-2)
    g = np.random.default_rng(3).standard_normal(n ** 3)
    bj = krylov.BlockJacobi(M, n, 2)
    res = krylov.gmres(lambda v: M @ v, bj.apply, g, restart=7, tol_rel=1e-13, max_iter=2000)
    assert res.converged
    x = np.linalg.solve(M.toarray(), g)
    np.testing.assert_allclose(res.x, x, atol=1e-10 * np.abs(x).max())
    assert res.res_norm <= 1e-12 * np.linalg.norm(g)


def test_gmres_full_terminates_in_N_steps_and_residual_monotone():
    n = 2
    L = operators.advdiff_csr(n, synth.kappa_field(n, seed=5), (1.0, -1.0, 0.5))
    M = krylov.shifted(L, 0.05).toarray()
    g = np.random.default_rng(4).standard_normal(n ** 3)
    hist = []

    def apply_A(v):
        return M @ v

    res = krylov.gmres(apply_A, lambda r: r, g, restart=n ** 3, tol_rel=1e-12, max_iter=n ** 3)
    assert res.converged and res.iters <= n ** 3
    # residual of the k-step minimiser is non-increasing in k (fresh runs with k steps)
    for k in range(1, n ** 3 + 1):
        rk = krylov.gmres(apply_A, lambda r: r, g, restart=k, tol_rel=0.0, max_iter=k)
        hist.append(np.linalg.norm(g - M @ rk.x))
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))


def test_solvers_zero_rhs_and_abs_tol():
    M = _heat_system(3, 1.0, 1e-2)
    z = np.zeros(27)
    assert krylov.pcg(lambda v: M @ v, lambda r: r, z).iters == 0
    assert krylov.gmres(lambda v: M @ v, lambda r: r, z).iters == 0
    g = np.full(27, 1e-3)
    assert krylov.pcg(lambda v: M @ v, lambda r: r, g, tol_rel=0.0, tol_abs=1.0).iters == 0
