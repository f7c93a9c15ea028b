"""Butcher tableaux split into high- and low-precision parts, and R(z).

A tableau is stored as (A_hi, A_lo, b): A = A_hi + A_lo, where A_hi holds
the coefficients that multiply high-precision stage derivatives f(y_j) and
A_lo those that multiply the low-precision ones f^eps(y_j) (Sec. 2.2, the
superscript-epsilon coefficients).  A_hi is strictly lower triangular and
A_lo lower triangular; a stage i with A_lo[i, i] != 0 is implicit and is
solved in low precision.  c is the row sum of A (Sec. 2.2.1) and is not used
because the test problems are autonomous.
"""
from __future__ import annotations

import math

import numpy as np


def _tab(A_hi, A_lo, b):
    return (np.array(A_hi, dtype=np.float64), np.array(A_lo, dtype=np.float64),
            np.array(b, dtype=np.float64))


def midpoint(corrections: int = 1):
    """Implicit midpoint with `corrections` explicit FP64 correction stages
    (Sec. 2.1, Fig. fig_Aq_rat; App. A): stage 1 solves y = u + tau/2 f^eps(y)
    in low precision, stage m+1 is y_m = u + tau/2 f(y_{m-1}), and
    u_{n+1} = u + tau f(y_last).  corrections=0 is the plain midpoint rule."""
    q = corrections + 1
    A_hi = np.zeros((q, q))
    A_lo = np.zeros((q, q))
    A_lo[0, 0] = 0.5
    for i in range(1, q):
        A_hi[i, i - 1] = 0.5
    b = np.zeros(q)
    b[-1] = 1.0
    return A_hi, A_lo, b


def m4s3pA():
    """Method 4s3pA (Sec. 2.2.1, Table ButchertabA).  Stages 1 and 3 are
    implicit in low precision; the low-precision term a31^eps f^eps(y1) of
    stage 3 follows Eq. mpAstep3.  Not A-stable (Sec. 2.3)."""
    a11e = 0.788675134594813
    a21 = 0.211324865405187
    a31e, a31 = 0.051944240459852, 0.709495523817170
    a32 = -0.86531425061942
    a33e = 0.788675134594813
    a41, a42, a43 = 0.705123240545107, 0.943370088535775, -0.859818194486069
    A_hi = [[0, 0, 0, 0], [a21, 0, 0, 0], [a31, a32, 0, 0], [a41, a42, a43, 0]]
    A_lo = [[a11e, 0, 0, 0], [0, 0, 0, 0], [a31e, 0, a33e, 0], [0, 0, 0, 0]]
    return _tab(A_hi, A_lo, [0.0, 0.5, 0.0, 0.5])


# Table ButchertabB prints a_{4,2}^eps = 0.051944240459852, the same digits as
# 4s3pA's a_{3,1}^eps.  With that value the method fails b.c = 1/2 and is not
# stable at z = -1.  The value that makes c_4 = 1 and restores every order-3
# condition and b^T A^eps e = 0 is -1.5 - a_{4,2}.
M4S3PB_A42_EPS_PRINTED = 0.051944240459852
M4S3PB_A42_EPS = -1.5 - 2.367724727682735


def m4s3pB(a42e: float = M4S3PB_A42_EPS):
    """Method 4s3pB (Sec. 2.2.2, Table ButchertabB): every stage implicit in
    low precision with a_ii^eps = 1/2, A-stable.  `a42e` defaults to the
    corrected a_{4,2}^eps (the printed value is a transcription slip)."""
    A_hi = [[0, 0, 0, 0],
            [2.543016042796356, 0, 0, 0],
            [2.451484396921318, 0.024108961241221, 0, 0],
            [2.073861819468268, 2.367724727682735, 1.711868223075524, 0]]
    A_lo = [[0.5, 0, 0, 0],
            [-2.376349376129689, 0.5, 0, 0],
            [-2.951484396921318, 0.475891038758779, 0.5, 0],
            [-0.573861819468268, a42e, -1.211868223075524, 0.5]]
    return _tab(A_hi, A_lo, [1.5, -1.5, 0.5, 0.5])


def m4s3pC():
    """Method 4s3pC (Sec. 2.2.3, Table ButchertabC): DIRK with four different
    low-precision diagonal entries."""
    A_hi = [[0, 0, 0, 0],
            [-0.050470366527530, 0, 0, 0],
            [0.368613367355336, 0.273504374252976, 0, 0],
            [1.803794668975043, 0.097485042980759, -1.895660952342050, 0]]
    A_lo = [[0.511243008730995, 0, 0, 0],
            [-1.999347282862640, 1.957161067302390, 0, 0],
            [0.443312893511937, -0.573131033672219, 0.128283796414019, 0],
            [-2.0, -0.160330320741428, 0.579597314161362, 1.484688928981990]]
    b = [0.002837446974069, 0.336264433650450, 0.806376720267787, -0.145478600892306]
    return _tab(A_hi, A_lo, b)


def sdirk2():
    """Two-stage, order-2, L-stable SDIRK with gamma = 1 - 1/sqrt(2)
    (R. Alexander, SIAM J. Numer. Anal. 14 (1977)).  Not in the paper; split
    as A_lo = diag(A) (the implicit solves) and A_hi = the strictly lower part."""
    g = 1.0 - 1.0 / math.sqrt(2.0)
    A = np.array([[g, 0.0], [1.0 - g, g]])
    return np.tril(A, -1), np.diag(np.diag(A)), np.array([1.0 - g, g])


def dirk3_gamma() -> float:
    """Root in (0.4, 0.5) of x^3 - 3x^2 + 3x/2 - 1/6 (bisection to 1 ulp)."""
    f = lambda x: ((x - 3.0) * x + 1.5) * x - 1.0 / 6.0
    lo, hi = 0.4, 0.5
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid in (lo, hi):
            break
        if (f(lo) < 0) == (f(mid) < 0):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def dirk3():
    """Three-stage, order-3, L-stable stiffly accurate DIRK of Alexander
    (1977): gamma from dirk3_gamma(), a21 = (1-gamma)/2,
    b1 = -(6g^2 - 16g + 1)/4, b2 = (6g^2 - 20g + 5)/4, b3 = g, last row = b.
    Not in the paper; split as for sdirk2."""
    g = dirk3_gamma()
    b1 = -(6 * g * g - 16 * g + 1) / 4.0
    b2 = (6 * g * g - 20 * g + 5) / 4.0
    A = np.array([[g, 0, 0], [(1 - g) / 2.0, g, 0], [b1, b2, g]])
    return np.tril(A, -1), np.diag(np.diag(A)), np.array([b1, b2, g])


PRESETS = {
    "midpoint0": lambda: midpoint(0),
    "midpoint1": lambda: midpoint(1),
    "midpoint2": lambda: midpoint(2),
    "4s3pA": m4s3pA,
    "4s3pB": m4s3pB,
    "4s3pC": m4s3pC,
    "sdirk2": sdirk2,
    "dirk3": dirk3,
}


def get(name: str):
    return PRESETS[name]()


def stability_function(A_hi, A_lo, b, z):
    """R(z) = 1 + z b^T (I - z A)^{-1} e with A = A_hi + A_lo (Sec. 2.3).
    `z` may be a scalar or an array of complex/real values."""
    A = np.asarray(A_hi) + np.asarray(A_lo)
    q = A.shape[0]
    e = np.ones(q)
    zs = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    out = np.empty(zs.shape, dtype=np.complex128)
    for idx, zz in np.ndenumerate(zs):
        out[idx] = 1.0 + zz * (np.asarray(b) @ np.linalg.solve(np.eye(q) - zz * A, e))
    if np.isscalar(z) or np.ndim(z) == 0:
        return out[0]
    return out
