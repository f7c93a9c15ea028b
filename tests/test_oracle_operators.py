"""Pins for oracle.operators: sine-mode eigenpairs of the heat stencil, a
Kronecker-sum construction of the Laplacian (the K1D = tridiag(-1,2,-1)
structure of Sec. 5.2.1), and a brute-force loop evaluation of the upwind
advection-diffusion operator on tiny grids."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import operators
from closed_forms import sine_eigenvalue


@pytest.mark.parametrize("n,kappa,modes", [(5, 1.0, (1, 1, 1)), (8, 0.3, (2, 1, 3)), (13, 2.0, (4, 4, 1))])
def test_heat_sine_eigenpairs(n, kappa, modes):
    phi = synth.sine_mode(n, *modes)
    lam = sine_eigenvalue(n, kappa, *modes)
    np.testing.assert_allclose(operators.heat_apply(phi, n, kappa), lam * phi, rtol=0, atol=1e-9 * abs(lam))


def test_heat_kronecker_sum_and_csr():
    n, kappa = 4, 0.7
    h = 1.0 / (n + 1)
    T = sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]).toarray()  # -K1D
    I = np.eye(n)
    # lexicographic i + j n + k n^2: x is the fastest (rightmost) Kronecker factor
    L = kappa / h ** 2 * (np.kron(I, np.kron(I, T)) + np.kron(I, np.kron(T, I)) + np.kron(T, np.kron(I, I)))
    E = np.eye(n ** 3)
    Ls = np.stack([operators.heat_apply(E[:, c], n, kappa) for c in range(n ** 3)], axis=1)
    np.testing.assert_allclose(Ls, L, atol=1e-10)
    np.testing.assert_allclose(operators.heat_csr(n, kappa).toarray(), L, atol=1e-10)


def _advdiff_bruteforce(n, kap, vel):
    """Row-by-row loop evaluation of L as a dense matrix."""
    h = 1.0 / (n + 1)
    N = n ** 3
    L = np.zeros((N, N))
    K = kap.reshape(n, n, n)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                P = i + j * n + k * n * n
                for d, (di, dj, dk) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
                    for s in (-1, 1):
                        ii, jj, kk = i + s * di, j + s * dj, k + s * dk
                        inside = 0 <= ii < n and 0 <= jj < n and 0 <= kk < n
                        if inside:
                            Q = ii + jj * n + kk * n * n
                            kf = 0.5 * (K[k, j, i] + K[kk, jj, ii])
                            L[P, Q] += kf / h ** 2
                            L[P, P] -= kf / h ** 2
                        else:
                            L[P, P] -= K[k, j, i] / h ** 2
                    v = vel[d]
                    # upwind difference of v_d du/dx_d moved to the right-hand side
                    if v >= 0:
                        L[P, P] -= v / h
                        ii, jj, kk = i - di, j - dj, k - dk
                        if 0 <= ii < n and 0 <= jj < n and 0 <= kk < n:
                            L[P, ii + jj * n + kk * n * n] += v / h
                    else:
                        L[P, P] += v / h
                        ii, jj, kk = i + di, j + dj, k + dk
                        if 0 <= ii < n and 0 <= jj < n and 0 <= kk < n:
                            L[P, ii + jj * n + kk * n * n] -= v / h
    return L


@pytest.mark.parametrize("n,vel", [(3, (1.0, 0.5, 0.25)), (4, (-0.3, 0.0, 2.0)), (2, (0.0, 0.0, 0.0))])
def test_advdiff_bruteforce(n, vel):
    kap = synth.kappa_field(n, seed=3)
    A = operators.advdiff_csr(n, kap, vel).toarray()
    np.testing.assert_allclose(A, _advdiff_bruteforce(n, kap, vel), rtol=1e-13, atol=1e-9)


def test_advdiff_properties():
    n = 6
    kap = synth.kappa_field(n, seed=1)
    D = operators.advdiff_csr(n, kap, (0, 0, 0)).toarray()
    np.testing.assert_allclose(D, D.T, atol=1e-9)              # diffusion part symmetric
    assert np.all(np.linalg.eigvalsh(D) < 0)                     # and negative definite
    A = operators.advdiff_csr(n, kap, (1.0, 0.5, 0.25)).toarray()
    off = A - np.diag(np.diag(A))
    assert np.all(off >= 0)                                      # M-matrix sign pattern
    assert np.all(A.sum(axis=1) <= 1e-9)                         # non-positive row sums
    # rows of interior nodes (all six neighbours inside) sum to zero when u is constant
    i = j = k = 2
    assert abs(A[i + j * n + k * n * n].sum()) < 1e-8
    # constant kappa, zero velocity: the heat operator
    np.testing.assert_allclose(operators.advdiff_csr(n, np.full(n ** 3, 1.7), (0, 0, 0)).toarray(),
                               operators.heat_csr(n, 1.7).toarray(), atol=1e-10)


def test_planted_wrong_spacing_is_caught():
    """With the printed h = 1/(n-1) (instead of 1/(n+1)) the eigen pin fails."""
    n = 9
    phi = synth.sine_mode(n, 1, 1, 1)
    h_bad = 1.0 / (n - 1)
    lam = sine_eigenvalue(n, 1.0, 1, 1, 1)
    Lphi = operators.heat_apply(phi, n, 1.0) * ((1.0 / (n + 1)) ** 2 / h_bad ** 2)
    assert np.max(np.abs(Lphi - lam * phi)) > 1e-3 * abs(lam)
