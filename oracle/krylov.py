"""Stage-system solvers in float64 (Sec. 3, Eq. corelinear).

The stage system is (I - s L) k = g with s = tau a_ii > 0 (the
stage-derivative form of (a_ii I + tau K) x = b).  Heat systems are SPD and
solved by preconditioned CG, advection-diffusion systems by right-
preconditioned restarted GMRES (Sec. 3).  Both stop when the residual 2-norm
is below tol_rel times the right-hand side's 2-norm OR below tol_abs
(the either-or rule of Sec. 5.3), start from zero and give up after max_iter
iterations.

The preconditioner is block-Jacobi over x-line segments: every x-line of n
nodes is cut into consecutive blocks of `bs` nodes, the last block of a line
holding the n mod bs remainder.  Each diagonal block of I - s L is inverted
densely (LAPACK LU with partial pivoting) in float64.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def line_blocks(n: int, bs: int):
    """Block layout on one x-line: list of (offset, size)."""
    out = []
    i = 0
    while i < n:
        m = min(bs, n - i)
        out.append((i, m))
        i += m
    return out


class BlockJacobi:
    """z = D^{-1} r, D the x-line-segment block diagonal of a matrix M."""

    def __init__(self, M: sp.csr_matrix, n: int, bs: int):
        self.n, self.bs = n, bs
        Mc = M.tocsr()
        nlines = n * n
        self.groups = []  # (size, row offsets within a line, inverses (nlines*nb, m, m))
        by_size = {}
        for off, m in line_blocks(n, bs):
            by_size.setdefault(m, []).append(off)
        for m, offs in by_size.items():
            starts = (np.arange(nlines)[:, None] * n + np.array(offs)[None, :]).ravel()
            rows = starts[:, None] + np.arange(m)[None, :]
            blocks = np.empty((starts.size, m, m))
            for a in range(m):          # entry (a, b) of every block at once
                for b in range(m):
                    blocks[:, a, b] = np.asarray(Mc[rows[:, a], rows[:, b]]).ravel()
            inv = np.linalg.inv(blocks)  # LU with partial pivoting per block
            self.groups.append((m, starts, inv))

    def apply(self, r):
        z = np.empty_like(r)
        for m, starts, inv in self.groups:
            gidx = starts[:, None] + np.arange(m)[None, :]
            z[gidx] = np.einsum("bij,bj->bi", inv, r[gidx])
        return z


# unit roundoff of IEEE half precision (10 stored mantissa bits)
U_HALF = 2.0 ** -11


class AdaptiveBlockJacobi(BlockJacobi):
    """Block-Jacobi whose inverted diagonal blocks are stored in a precision
    chosen block by block from the block's conditioning (the adaptive-precision
    block-Jacobi of Ginkgo named in Sec. 1): a block whose 1-norm condition
    number kappa_1(D_b) = ||D_b||_1 ||D_b^-1||_1 satisfies
    kappa_1 * u_half <= tau keeps its inverse in FP16, every other block in
    `high` (FP32).  The inverse is formed in float64 and rounded once; the
    apply is float64 arithmetic on the rounded entries."""

    def __init__(self, M: sp.csr_matrix, n: int, bs: int, tau: float = 1e-2, high=np.float32):
        super().__init__(M, n, bs)
        self.tau = tau
        self.low_blocks = 0
        self.total_blocks = 0
        self.kappas = []  # per block group: kappa_1 of every block
        Mc = M.tocsr()
        out = []
        for m, starts, inv in self.groups:
            rows = starts[:, None] + np.arange(m)[None, :]
            blocks = np.empty((starts.size, m, m))
            for a in range(m):
                for b in range(m):
                    blocks[:, a, b] = np.asarray(Mc[rows[:, a], rows[:, b]]).ravel()
            # 1-norm: largest column sum of absolute values
            kappa = np.abs(blocks).sum(axis=1).max(axis=1) * np.abs(inv).sum(axis=1).max(axis=1)
            low = kappa * U_HALF <= tau
            rounded = np.where(low[:, None, None], inv.astype(np.float16).astype(np.float64),
                               inv.astype(high).astype(np.float64))
            self.kappas.append(kappa)
            self.low_blocks += int(low.sum())
            self.total_blocks += int(low.size)
            out.append((m, starts, rounded))
        self.groups = out


def shifted(L_csr: sp.csr_matrix, s: float) -> sp.csr_matrix:
    """I - s L as a CSR matrix."""
    return (sp.identity(L_csr.shape[0], format="csr") - s * L_csr).tocsr()


class SolveResult:
    def __init__(self, x, iters, converged, res_norm, rhs_norm):
        self.x, self.iters, self.converged = x, iters, converged
        self.res_norm, self.rhs_norm = res_norm, rhs_norm


def pcg(apply_A, apply_M, b, tol_rel=1e-12, tol_abs=0.0, max_iter=1000):
    """Preconditioned conjugate gradients from x0 = 0 (Hestenes-Stiefel with
    left preconditioner M ~ A^{-1}).  `iters` counts matrix products."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = math.sqrt(float(r @ r))
    rnorm = bnorm
    if rnorm <= tol_abs or rnorm <= tol_rel * bnorm or bnorm == 0.0:
        return SolveResult(x, 0, True, rnorm, bnorm)
    z = apply_M(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < max_iter:
        q = apply_A(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rnorm = math.sqrt(float(r @ r))
        if rnorm <= tol_abs or rnorm <= tol_rel * bnorm:
            return SolveResult(x, it, True, rnorm, bnorm)
        z = apply_M(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return SolveResult(x, it, False, rnorm, bnorm)


def gmres(apply_A, apply_M, b, restart=30, tol_rel=1e-8, tol_abs=0.0, max_iter=1000):
    """Right-preconditioned restarted GMRES(m) from x0 = 0: Arnoldi on
    A M^{-1} with modified Gram-Schmidt, Givens rotations for the
    least-squares problem, x = x0 + M^{-1} V y at the end of each cycle.
    The stopping test uses the rotated residual |g_{j+1}|, which equals the
    true residual norm of the right-preconditioned system.  `iters` counts
    Arnoldi steps."""
    b = np.asarray(b, dtype=np.float64)
    N = b.size
    x = np.zeros_like(b)
    bnorm = math.sqrt(float(b @ b))
    if bnorm == 0.0 or bnorm <= tol_abs:
        return SolveResult(x, 0, True, bnorm, bnorm)
    it = 0
    r = b.copy()
    beta = bnorm
    while True:
        if beta <= tol_abs or beta <= tol_rel * bnorm:
            return SolveResult(x, it, True, beta, bnorm)
        if it >= max_iter:
            return SolveResult(x, it, False, beta, bnorm)
        m = restart
        V = np.zeros((m + 1, N))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        res = beta
        for j in range(m):
            w = apply_A(apply_M(V[j]))
            for i in range(j + 1):
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = math.sqrt(float(w @ w))
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            denom = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / denom
            sn[j] = H[j + 1, j] / denom
            H[j, j] = denom
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            res = abs(g[j + 1])
            if res <= tol_abs or res <= tol_rel * bnorm or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x += apply_M(V[:j_done].T @ y)
        r = b - apply_A(x)
        beta = math.sqrt(float(r @ r))
        if res <= tol_abs or res <= tol_rel * bnorm:
            return SolveResult(x, it, True, beta, bnorm)
