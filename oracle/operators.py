"""Semi-discrete operators L of du/dt = L u on the unit cube (Sec. 3; Sec. 5.2).

Unknowns live on the n^3 interior nodes x_i = (i+1) h, h = 1/(n+1), with
homogeneous Dirichlet values on the boundary (heat, advection-diffusion), or
on the periodic grid x_i = i h, h = 1/n (periodic advection), numbered
lexicographically u[i + j n + k n^2] (the numbering of Sec. 4.2).  In numpy a
field is viewed as an (n, n, n) array indexed [k, j, i].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def grid_h(n: int) -> float:
    return 1.0 / (n + 1)


def heat_apply(u: np.ndarray, n: int, kappa: float) -> np.ndarray:
    """(L u)_ijk = kappa/h^2 (sum of the six neighbours - 6 u_ijk), neighbours
    outside the grid being zero: the second-order central 7-point Laplacian
    of the heat test case (Sec. 5.2.1) scaled by the diffusivity."""
    h = grid_h(n)
    U = np.asarray(u, dtype=np.float64).reshape(n, n, n)
    out = -6.0 * U
    out[:, :, 1:] += U[:, :, :-1]
    out[:, :, :-1] += U[:, :, 1:]
    out[:, 1:, :] += U[:, :-1, :]
    out[:, :-1, :] += U[:, 1:, :]
    out[1:, :, :] += U[:-1, :, :]
    out[:-1, :, :] += U[1:, :, :]
    return (kappa / (h * h)) * out.ravel()


def advdiff_csr(n: int, kappa: np.ndarray, vel=(1.0, 0.5, 0.25)) -> sp.csr_matrix:
    """CSR matrix of L u = div(kappa grad u) - v . grad u.

    Diffusion: for each of the six faces of node P, kappa_f (u_Q - u_P)/h^2
    with kappa_f the arithmetic mean of kappa_P and kappa_Q; on a boundary
    face the ghost value is u_Q = 0 and kappa_f = kappa_P.
    Advection: first-order upwind, -v_d (u_P - u_{P-e_d})/h for v_d >= 0 and
    -v_d (u_{P+e_d} - u_P)/h for v_d < 0, ghost values zero.
    `kappa` holds the diffusivity at the n^3 nodes (flat, lexicographic)."""
    N = n ** 3
    h = grid_h(n)
    kap = np.asarray(kappa, dtype=np.float64).reshape(n, n, n)
    idx = np.arange(N).reshape(n, n, n)
    rows, cols, vals = [], [], []
    diag = np.zeros((n, n, n))
    inv_h2 = 1.0 / (h * h)
    for axis, vd in zip((2, 1, 0), vel):  # axis 2 = x, 1 = y, 0 = z
        for s in (-1, 1):
            # slices selecting nodes P whose neighbour P + s e_d is interior
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if s == 1:
                src[axis] = slice(0, n - 1)
                dst[axis] = slice(1, n)
            else:
                src[axis] = slice(1, n)
                dst[axis] = slice(0, n - 1)
            src, dst = tuple(src), tuple(dst)
            kf = 0.5 * (kap[src] + kap[dst])
            rows.append(idx[src].ravel())
            cols.append(idx[dst].ravel())
            vals.append((kf * inv_h2).ravel())
            diag[src] -= kf * inv_h2
            # boundary face on side s: ghost u = 0, kappa_f = kappa_P
            bnd = [slice(None)] * 3
            bnd[axis] = n - 1 if s == 1 else 0
            diag[tuple(bnd)] -= kap[tuple(bnd)] * inv_h2
            # upwind advection: the upstream neighbour is P - e_d for v_d >= 0
            upstream = -1 if vd >= 0 else 1
            if s == upstream:
                rows.append(idx[src].ravel())
                cols.append(idx[dst].ravel())
                vals.append(np.full(idx[src].size, abs(vd) / h))
        diag -= abs(vd) / h
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def adv_periodic_csr(n: int, beta=(1.0, 1.0, 1.0)) -> sp.csr_matrix:
    """CSR matrix of L u = -div(beta u) = -sum_d beta_d D_d u for constant beta
    on the periodic grid x_i = i h, h = 1/n (the advection test of Sec. 5.2.2):
    D_d is the second-order central difference (u(x + h e_d) - u(x - h e_d)) /
    (2h), i.e. the 1-D matrix Tridiag(-1, 0, 1) + K^(B) / (2h) with the periodic
    corner entries K^(B).  Written as a sum of Kronecker products."""
    h = 1.0 / n
    K = np.zeros((n, n))
    for i in range(n):
        K[i, (i + 1) % n] += 1.0
        K[i, (i - 1) % n] -= 1.0
    D = sp.csr_matrix(K / (2.0 * h))
    I = sp.identity(n, format="csr")
    Dx = sp.kron(I, sp.kron(I, D))
    Dy = sp.kron(I, sp.kron(D, I))
    Dz = sp.kron(D, sp.kron(I, I))
    return (-(beta[0] * Dx + beta[1] * Dy + beta[2] * Dz)).tocsr()


def heat_csr(n: int, kappa: float) -> sp.csr_matrix:
    """The heat operator as a CSR matrix: advdiff_csr with constant kappa and
    zero velocity."""
    return advdiff_csr(n, np.full(n ** 3, float(kappa)), vel=(0.0, 0.0, 0.0))


class HeatOperator:
    """Constant-coefficient heat operator, applied matrix-free."""

    def __init__(self, n: int, kappa: float):
        self.n, self.kappa = n, float(kappa)
        self.N = n ** 3

    def apply(self, u):
        return heat_apply(u, self.n, self.kappa)

    def csr(self):
        return heat_csr(self.n, self.kappa)


class CSROperator:
    """Operator given by an assembled CSR matrix (advection-diffusion)."""

    def __init__(self, n: int, A: sp.csr_matrix):
        self.n, self.A = n, A
        self.N = A.shape[0]

    def apply(self, u):
        return self.A @ u

    def csr(self):
        return self.A


class PeriodicOperator(CSROperator):
    """The periodic advection operator of Sec. 5.2.2 (CSR) with its velocity,
    so that a solver can build the complex fast diagonalization for it."""

    def __init__(self, n: int, beta=(1.0, 1.0, 1.0)):
        super().__init__(n, adv_periodic_csr(n, beta))
        self.beta = tuple(float(b) for b in beta)
