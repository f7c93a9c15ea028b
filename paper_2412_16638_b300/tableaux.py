"""Split Butcher tableaux (A_hi, A_lo, b) passed to rk_set_tableau.

A = A_hi + A_lo; A_hi (strictly lower) multiplies FP64 stage derivatives,
A_lo (lower, with the implicit diagonal) multiplies the low-precision ones.
Coefficients of 4s3pA/B/C are those of Sec. 2.2 (Tables ButchertabA, B, C);
in 4s3pB the entry a_{4,2}^eps is -3.867724727682735 (= -1.5 - a_{4,2}), the
value that satisfies the order-3 conditions, in place of the printed
0.051944240459852.  SDIRK2 and DIRK3 are Alexander's (1977) L-stable
methods, not in the paper, split with the whole diagonal in A_lo.
"""
from __future__ import annotations

import math

_G2 = 1.0 - math.sqrt(0.5)
# gamma of the 3-stage method: root in (0.4, 0.5) of x^3 - 3x^2 + 3x/2 - 1/6
_G3 = 0.43586652150845899941601945


def _zeros(q):
    return [[0.0] * q for _ in range(q)]


def midpoint(corrections=1):
    q = corrections + 1
    ah, al = _zeros(q), _zeros(q)
    al[0][0] = 0.5
    for i in range(1, q):
        ah[i][i - 1] = 0.5
    b = [0.0] * q
    b[-1] = 1.0
    return ah, al, b


def _table(entries_hi, entries_lo, b):
    q = len(b)
    ah, al = _zeros(q), _zeros(q)
    for (i, j), v in entries_hi.items():
        ah[i - 1][j - 1] = v
    for (i, j), v in entries_lo.items():
        al[i - 1][j - 1] = v
    return ah, al, list(b)


PRESETS = {
    "midpoint0": lambda: midpoint(0),
    "midpoint1": lambda: midpoint(1),
    "midpoint2": lambda: midpoint(2),
    "4s3pA": lambda: _table(
        {(2, 1): 0.211324865405187, (3, 1): 0.709495523817170, (3, 2): -0.86531425061942,
         (4, 1): 0.705123240545107, (4, 2): 0.943370088535775, (4, 3): -0.859818194486069},
        {(1, 1): 0.788675134594813, (3, 1): 0.051944240459852, (3, 3): 0.788675134594813},
        (0.0, 0.5, 0.0, 0.5)),
    "4s3pB": lambda: _table(
        {(2, 1): 2.543016042796356, (3, 1): 2.451484396921318, (3, 2): 0.024108961241221,
         (4, 1): 2.073861819468268, (4, 2): 2.367724727682735, (4, 3): 1.711868223075524},
        {(1, 1): 0.5, (2, 2): 0.5, (3, 3): 0.5, (4, 4): 0.5,
         (2, 1): -2.376349376129689, (3, 1): -2.951484396921318, (3, 2): 0.475891038758779,
         (4, 1): -0.573861819468268, (4, 2): -3.867724727682735, (4, 3): -1.211868223075524},
        (1.5, -1.5, 0.5, 0.5)),
    "4s3pC": lambda: _table(
        {(2, 1): -0.050470366527530, (3, 1): 0.368613367355336, (3, 2): 0.273504374252976,
         (4, 1): 1.803794668975043, (4, 2): 0.097485042980759, (4, 3): -1.895660952342050},
        {(1, 1): 0.511243008730995, (2, 1): -1.999347282862640, (2, 2): 1.957161067302390,
         (3, 1): 0.443312893511937, (3, 2): -0.573131033672219, (3, 3): 0.128283796414019,
         (4, 1): -2.0, (4, 2): -0.160330320741428, (4, 3): 0.579597314161362, (4, 4): 1.484688928981990},
        (0.002837446974069, 0.336264433650450, 0.806376720267787, -0.145478600892306)),
    "sdirk2": lambda: _table({(2, 1): 1.0 - _G2}, {(1, 1): _G2, (2, 2): _G2}, (1.0 - _G2, _G2)),
    "dirk3": lambda: _table(
        {(2, 1): (1.0 - _G3) / 2.0,
         (3, 1): -(6 * _G3 ** 2 - 16 * _G3 + 1) / 4.0,
         (3, 2): (6 * _G3 ** 2 - 20 * _G3 + 5) / 4.0},
        {(1, 1): _G3, (2, 2): _G3, (3, 3): _G3},
        (-(6 * _G3 ** 2 - 16 * _G3 + 1) / 4.0, (6 * _G3 ** 2 - 20 * _G3 + 5) / 4.0, _G3)),
}


def get(name):
    """(A_hi, A_lo, b) as nested Python lists."""
    return PRESETS[name]()
