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


def _advdiff_system(n, s):
    return krylov.shifted(operators.advdiff_csr(n, synth.kappa_field(n, seed=1), (1.0, 0.5, 0.25)), s)


@pytest.mark.parametrize("n,bs,s", [(6, 4, 3e-3), (7, 8, 1e-2), (9, 2, 5e-2)])
def test_adaptive_block_jacobi_choice_and_rounding(n, bs, s):
    """Adaptive precision: every block's choice follows kappa_1 * 2^-11 <= tau
    with kappa_1 from LAPACK's 1-norm condition number of that block taken
    one by one, and its inverse equals the dense inverse rounded once to FP16
    or FP32 accordingly (tau set between two blocks' condition numbers, so
    both precisions occur)."""
    M = _advdiff_system(n, s)
    probe = krylov.AdaptiveBlockJacobi(M, n, bs, tau=1e-2)
    kap = np.sort(np.concatenate(probe.kappas))
    mid = len(kap) // 2
    tau = 0.5 * (kap[mid - 1] + kap[mid]) * krylov.U_HALF
    if kap[mid - 1] == kap[mid]:
        pytest.skip("no gap between the middle condition numbers")
    A = krylov.AdaptiveBlockJacobi(M, n, bs, tau=tau)
    assert 0 < A.low_blocks < A.total_blocks
    Md = M.toarray()
    for m, starts, inv in A.groups:
        for st, Binv in zip(starts, inv):
            B = Md[st:st + m, st:st + m]
            kappa = np.linalg.cond(B, 1)
            exact = np.linalg.inv(B)
            want = exact.astype(np.float16 if kappa * 2.0 ** -11 <= tau else np.float32).astype(np.float64)
            np.testing.assert_array_equal(Binv, want)


def test_adaptive_block_jacobi_limits():
    """tau = 0 keeps every block in FP32 (the FP32-rounded plain block-Jacobi);
    a huge tau stores every block in FP16; the apply is linear."""
    n, bs, s = 6, 4, 1e-2
    M = _advdiff_system(n, s)
    plain = krylov.BlockJacobi(M, n, bs)
    hi = krylov.AdaptiveBlockJacobi(M, n, bs, tau=0.0)
    lo = krylov.AdaptiveBlockJacobi(M, n, bs, tau=1e30)
    assert hi.low_blocks == 0 and lo.low_blocks == lo.total_blocks
    r = np.random.default_rng(3).standard_normal(n ** 3)
    for (m, st, inv), (_, _, inv32) in zip(plain.groups, hi.groups):
        np.testing.assert_array_equal(inv.astype(np.float32).astype(np.float64), inv32)
    for (m, st, inv), (_, _, inv16) in zip(plain.groups, lo.groups):
        np.testing.assert_array_equal(inv.astype(np.float16).astype(np.float64), inv16)
    np.testing.assert_allclose(hi.apply(2.0 * r), 2.0 * hi.apply(r), rtol=1e-15)
    assert np.linalg.norm(lo.apply(r) - plain.apply(r)) / np.linalg.norm(plain.apply(r)) < 2e-3
