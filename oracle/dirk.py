"""The perturbed (mixed-precision) DIRK step, evaluated entirely in float64.

For du/dt = f(u) = L u (+ a fixed forcing vector, the heat test of Sec. 5.2.1)
and a tableau split A = A_hi + A_lo (Sec. 2.2), stage i is

    y_i = u_n + tau sum_{j<i} (a^h_ij f(y_j) + a^eps_ij f^eps(y_j))
              + tau a^eps_ii f^eps(y_i)                      (Eqs. mpAstep1-4)

and u_{n+1} = u_n + tau sum_j b_j f(y_j)                     (Eq. RKstep).

With r_i the explicit part, the implicit stage is solved for the stage
derivative k^eps_i = f^eps(y_i) = L y_i:  (I - tau a_ii L) k^eps_i = L r_i,
then y_i = r_i + tau a_ii k^eps_i and the high-precision derivative is the
explicit evaluation k_i = f(y_i) = L y_i (Sec. 2.1 step 2, Sec. 4.2: explicit
operations and linear combinations in high precision).  An explicit stage
(a_ii = 0) has y_i = r_i and k^eps_i = k_i.

Here every operation is float64, so k_i and k^eps_i differ only by the solver
tolerance; the GPU library runs the solve in low precision.  With
corrected=False the step is the plain DIRK baseline that uses the solver's
k^eps_i directly as k_i (no extra operator application).
"""
from __future__ import annotations

import weakref

import numpy as np

from . import fdm, krylov


class Solver:
    """Stage solver settings: 'cg' (heat) or 'gmres' (advection-diffusion);
    precond 'bj' (x-line block-Jacobi of size bs) or 'fdm' (fast
    diagonalization: the constant-coefficient heat operator, or the periodic
    advection operator given as operators.PeriodicOperator)."""

    def __init__(self, method="cg", bs=8, tol_rel=1e-12, tol_abs=0.0, max_iter=2000, restart=30, precond="bj"):
        self.method, self.bs, self.precond = method, bs, precond
        self.tol_rel, self.tol_abs = tol_rel, tol_abs
        self.max_iter, self.restart = max_iter, restart
        # preconditioners per operator object and shift; an entry disappears
        # with its operator, so a later operator never meets a stale one
        self._cache = weakref.WeakKeyDictionary()

    def solve(self, op, s, g):
        """Solve (I - s L) k = g."""
        per_op = self._cache.setdefault(op, {})
        key = (float(s), self.precond, self.bs)
        if key not in per_op:
            if self.precond == "fdm" and hasattr(op, "beta"):
                per_op[key] = fdm.PeriodicFastDiagonalization(op.n, op.beta, s).apply
            elif self.precond == "fdm":
                per_op[key] = fdm.FastDiagonalization(op.n, op.kappa, s).apply
            else:
                M = krylov.shifted(op.csr(), s)
                per_op[key] = krylov.BlockJacobi(M, op.n, self.bs).apply
        apply_M = per_op[key]
        apply_A = lambda v: v - s * op.apply(v)
        if self.method == "cg":
            return krylov.pcg(apply_A, apply_M, g, self.tol_rel, self.tol_abs, self.max_iter)
        return krylov.gmres(apply_A, apply_M, g, self.restart, self.tol_rel, self.tol_abs, self.max_iter)


def rk_step(u, dt, tableau, op, solver: Solver, corrected=True, stats=None, source=None):
    """One step u_n -> u_{n+1} of the split tableau (A_hi, A_lo, b) for
    du/dt = L u + source (source: a fixed forcing vector or None)."""
    A_hi, A_lo, b = tableau
    q = len(b)
    u = np.asarray(u, dtype=np.float64)
    k = [None] * q
    ke = [None] * q
    for i in range(q):
        r = u.copy()
        for j in range(i):
            if A_hi[i, j] != 0.0:
                r += dt * A_hi[i, j] * k[j]
            if A_lo[i, j] != 0.0:
                r += dt * A_lo[i, j] * ke[j]
        a = A_lo[i, i]
        f = (lambda y: op.apply(y)) if source is None else (lambda y: op.apply(y) + source)
        if a != 0.0:
            # stage derivative k = f(y), y = r + dt a k:  (I - dt a L) k = f(r)
            g = f(r)
            res = solver.solve(op, dt * a, g)
            if stats is not None:
                stats.append((res.iters, res.converged))
            ke[i] = res.x
            if corrected:
                k[i] = f(r + dt * a * ke[i])
            else:
                k[i] = ke[i]
        else:
            k[i] = f(r)
            ke[i] = k[i]
    out = u.copy()
    for j in range(q):
        if b[j] != 0.0:
            out += dt * b[j] * k[j]
    return out


def integrate(u0, dt, nsteps, tableau, op, solver: Solver, corrected=True, stats=None, source=None):
    u = np.asarray(u0, dtype=np.float64).copy()
    for _ in range(nsteps):
        u = rk_step(u, dt, tableau, op, solver, corrected, stats, source)
    return u
