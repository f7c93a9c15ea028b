"""Fast-diagonalization preconditioner (Sec. 3, Eqs. preconbasic, Pinvform,
TensorDecomp), float64.  TEST INFRASTRUCTURE ONLY.

On the unit cube with a uniform Cartesian grid the preconditioner has the
Kronecker-sum form

    P = I (x) I (x) A + I (x) B (x) I + C (x) I (x) I           (Eq. preconbasic)

with n x n one-dimensional operators A (x), B (y), C (z).  With the spectral
decompositions A = Q_A Lambda_A Q_A^-1 (and likewise B, C),

    P^-1 = (Q_C (x) Q_B (x) Q_A) P_D^-1 (Q_C^-1 (x) Q_B^-1 (x) Q_A^-1)  (Eq. Pinvform)

where P_D is diagonal, and the Kronecker factor splits into the three
tensor operations T_L T_M T_R of Eq. TensorDecomp.  The tensor operations act
on the lexicographic vector x_{i + j n + k n^2} (Sec. 4):

    (T_R x)_{ijk} = sum_q Q_{iq} x_{qjk},   (T_M x)_{ijk} = sum_q Q_{jq} x_{iqk},
    (T_L x)_{ijk} = sum_q Q_{kq} x_{ijq}.

For the constant-coefficient heat stage system (I - s L) k = g with
L = kappa/h^2 (7-point Laplacian) the splitting is exact with the settings of
Sec. 5.2.1: A = I + (s kappa/h^2) K1D and B = C = (s kappa/h^2) K1D,
K1D = tridiag(-1, 2, -1), so P is the system matrix itself and
preconditioned CG converges in one iteration in exact arithmetic.  The
one-dimensional decompositions are taken from LAPACK (numpy.linalg.eigh);
the tests pin them to the closed-form sine eigenpairs.
"""
from __future__ import annotations

import numpy as np

from .operators import grid_h


def line_operators(n: int, kappa: float, s: float):
    """The one-dimensional factors (A, B = C) of Sec. 5.2.1:
    A = I + (s kappa / h^2) K1D (x), B = C = (s kappa / h^2) K1D (y, z)."""
    c = s * kappa / grid_h(n) ** 2
    K = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return np.eye(n) + c * K, c * K


def _t_r(Q, x3):
    """T_R: contract the x index (fastest; x3 is indexed [k, j, i])."""
    return np.einsum("iq,kjq->kji", Q, x3, optimize=True)


def _t_m(Q, x3):
    """T_M: contract the y index."""
    return np.einsum("jq,kqi->kji", Q, x3, optimize=True)


def _t_l(Q, x3):
    """T_L: contract the z index."""
    return np.einsum("kq,qji->kji", Q, x3, optimize=True)


class FastDiagonalization:
    """z = P^-1 r for the heat stage matrix I - s L (Eq. Pinvform)."""

    def __init__(self, n: int, kappa: float, s: float):
        self.n = n
        A, B = line_operators(n, kappa, s)
        self.lam_a, self.Qa = np.linalg.eigh(A)  # A = Q_A diag(lam_a) Q_A^T, Q_A orthogonal
        self.lam_b, self.Qb = np.linalg.eigh(B)  # B = C
        # P_D = I (x) I (x) Lambda_A + I (x) Lambda_B (x) I + Lambda_C (x) I (x) I,
        # indexed [k, j, i]
        self.pd = self.lam_b[:, None, None] + self.lam_b[None, :, None] + self.lam_a[None, None, :]

    def apply(self, r):
        n, Qa, Qb = self.n, self.Qa, self.Qb
        x = np.asarray(r, dtype=np.float64).reshape(n, n, n)
        # (Q_C^-1 (x) Q_B^-1 (x) Q_A^-1) = T_L^-1 T_M^-1 T_R^-1, applied right to
        # left; Q^-1 = Q^T for the orthogonal eigenvector matrices
        x = _t_r(Qa.T, x)
        x = _t_m(Qb.T, x)
        x = _t_l(Qb.T, x)
        x = x / self.pd
        x = _t_r(Qa, x)
        x = _t_m(Qb, x)
        x = _t_l(Qb, x)
        return x.reshape(-1)


def periodic_difference(n: int):
    """The one-dimensional periodic central difference D (Sec. 5.2.2): the
    matrix Tridiag(-1, 0, 1) with the periodic corner entries, over 2h,
    h = 1/n."""
    h = 1.0 / n
    K = np.zeros((n, n))
    for i in range(n):
        K[i, (i + 1) % n] += 1.0
        K[i, (i - 1) % n] -= 1.0
    return K / (2.0 * h)


class PeriodicFastDiagonalization:
    """z = P^-1 r for the periodic advection stage matrix I - s L,
    L = -sum_d beta_d D_d (Sec. 5.2.2), by the complex fast diagonalization of
    Eq. Pinvform.  The Kronecker-sum splitting of Eq. preconbasic is exact
    with A = I + s beta_x D, B = s beta_y D, C = s beta_z D: the three factors
    are polynomials in the same circulant D, so they share its (complex)
    eigenvector matrix Q, and P_D = Lambda_C (+) Lambda_B (+) Lambda_A with
    Lambda_A = 1 + s beta_x mu, Lambda_B = s beta_y mu, Lambda_C = s beta_z mu
    for the eigenvalues mu of D.  D is normal, so its complex Schur
    decomposition D = Q T Q^H (LAPACK, scipy.linalg.schur) has a diagonal T and
    a unitary Q: Q^-1 = Q^H, also where eigenvalues repeat (mu_k = mu_{n/2-k})."""

    def __init__(self, n: int, beta, s: float):
        import scipy.linalg
        self.n = n
        T, self.Q = scipy.linalg.schur(periodic_difference(n).astype(np.complex128), output="complex")
        self.mu = np.diag(T)
        self.Qinv = self.Q.conj().T
        la = 1.0 + s * beta[0] * self.mu
        lb = s * beta[1] * self.mu
        lc = s * beta[2] * self.mu
        self.pd = lc[:, None, None] + lb[None, :, None] + la[None, None, :]  # indexed [k, j, i]

    def apply(self, r):
        n, Q, Qi = self.n, self.Q, self.Qinv
        x = np.asarray(r, dtype=np.float64).reshape(n, n, n).astype(np.complex128)
        x = _t_r(Qi, x)
        x = _t_m(Qi, x)
        x = _t_l(Qi, x)
        x = x / self.pd
        x = _t_r(Q, x)
        x = _t_m(Q, x)
        x = _t_l(Q, x)
        return x.real.reshape(-1)
