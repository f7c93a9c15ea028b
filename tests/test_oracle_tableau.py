"""Pins for oracle.tableau: printed coefficients (Sec. 2.2 tables), order
conditions, the perturbation condition b^T A^eps e = 0, and R(z) against the
closed form of App. A."""
import json
import math
import os

import numpy as np
import pytest

from oracle import tableau
from closed_forms import R_midpoint, R_scalar

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tableaux_printed.json")))


def _parts(name):
    A_hi, A_lo, b = tableau.get(name)
    return A_hi, A_lo, b, A_hi + A_lo


def _order_conditions(A, b):
    c = A.sum(axis=1)
    return {
        1: b.sum() - 1.0,
        2: b @ c - 0.5,
        3: (b @ (c * c) - 1.0 / 3.0, b @ (A @ c) - 1.0 / 6.0),
    }


@pytest.mark.parametrize("name", ["4s3pA", "4s3pB", "4s3pC"])
def test_presets_match_printed_tables(name):
    A_hi, A_lo, b, _ = _parts(name)
    g = GOLD[name]
    for key, val in g.items():
        if key == "b":
            np.testing.assert_array_equal(b, np.array(val))
            continue
        i, j = int(key[1]) - 1, int(key[2]) - 1
        got = A_lo[i, j] if key.endswith("e") else A_hi[i, j]
        if name == "4s3pB" and key == "a42e":
            # the one corrected entry: printed value is a copy of 4s3pA's a31^eps
            assert val == GOLD["4s3pA"]["a31e"]
            assert got == pytest.approx(-1.5 - g["a42"], abs=0)
            continue
        assert got == val, (name, key)


@pytest.mark.parametrize("name,order", [("midpoint0", 2), ("midpoint1", 2), ("midpoint2", 2),
                                        ("sdirk2", 2), ("dirk3", 3), ("4s3pA", 3),
                                        ("4s3pB", 3), ("4s3pC", 3)])
def test_order_conditions(name, order):
    _, _, b, A = _parts(name)
    oc = _order_conditions(A, b)
    assert abs(oc[1]) < 1e-13
    assert abs(oc[2]) < 1e-13
    if order >= 3:
        assert abs(oc[3][0]) < 1e-13 and abs(oc[3][1]) < 1e-13
    else:
        assert abs(oc[3][0]) > 1e-3 or abs(oc[3][1]) > 1e-3


def test_4s3pB_as_printed_fails_and_fix_is_unique():
    A_hi, A_lo, b = tableau.m4s3pB(tableau.M4S3PB_A42_EPS_PRINTED)
    A = A_hi + A_lo
    assert abs(b @ A.sum(axis=1) - 0.5) > 1.0           # b.c = 2.46 as printed
    assert abs(tableau.stability_function(A_hi, A_lo, b, -1.0)) > 1.0
    # b.c = 1/2 is linear in a42^eps with slope b_4 = 1/2: solve it directly
    b4 = b[3]
    c_rest = A.sum(axis=1)
    a42e_from_bc = tableau.M4S3PB_A42_EPS_PRINTED - (b @ c_rest - 0.5) / b4
    assert a42e_from_bc == pytest.approx(tableau.M4S3PB_A42_EPS, abs=1e-12)


@pytest.mark.parametrize("name", ["4s3pA", "4s3pB", "4s3pC"])
def test_perturbation_condition(name):
    _, A_lo, b, _ = _parts(name)
    assert abs(b @ A_lo.sum(axis=1)) < 1e-12


@pytest.mark.parametrize("corr", [0, 1, 2, 5])
def test_midpoint_R_closed_form(corr):
    A_hi, A_lo, b = tableau.midpoint(corr)
    for z in [-1.0, -10.0, 0.3, 1j, -2 + 3j]:
        assert tableau.stability_function(A_hi, A_lo, b, z) == pytest.approx(R_midpoint(z), rel=1e-11)
    if corr <= 1:
        assert tableau.stability_function(A_hi, A_lo, b, -1e4) == pytest.approx(R_midpoint(-1e4), rel=1e-10)
    assert tableau.stability_function(A_hi, A_lo, b, -1.0).real == pytest.approx(1.0 / 3.0, rel=1e-14)


def test_midpoint_corrections_amplify_rounding():
    """Sec. 2.1: the corrections are a fixed-point iteration that diverges when
    |z/2| > 1.  In floating point the stage values of M with p corrections
    carry rounding errors amplified by about |z/2|^p, so R(-1e4) evaluated in
    float64 is far from the exact (2+z)/(2-z) for p = 5 but not for p = 1."""
    z = -1e4
    e1 = abs(tableau.stability_function(*tableau.midpoint(1), z) - R_midpoint(z))
    e5 = abs(tableau.stability_function(*tableau.midpoint(5), z) - R_midpoint(z))
    assert e1 < 1e-9 and e5 > 1e-3


@pytest.mark.parametrize("name", ["4s3pB", "4s3pC", "sdirk2", "dirk3", "midpoint1"])
def test_A_stable_on_imaginary_axis_and_left_plane(name):
    A_hi, A_lo, b, A = _parts(name)
    ys = np.linspace(-50, 50, 401)
    assert np.all(np.abs(tableau.stability_function(A_hi, A_lo, b, 1j * ys)) <= 1.0 + 1e-10)
    xs = -np.logspace(-3, 6, 50)
    assert np.all(np.abs(tableau.stability_function(A_hi, A_lo, b, xs)) <= 1.0 + 1e-10)


@pytest.mark.parametrize("name", ["sdirk2", "dirk3"])
def test_L_stable(name):
    A_hi, A_lo, b, _ = _parts(name)
    assert abs(tableau.stability_function(A_hi, A_lo, b, -1e12)) < 1e-6


def test_4s3pA_not_A_stable():
    A_hi, A_lo, b, _ = _parts("4s3pA")
    zs = -np.logspace(-2, 4, 200)
    assert np.max(np.abs(tableau.stability_function(A_hi, A_lo, b, zs))) > 1.0


def test_stability_function_matches_plain_definition():
    for name in tableau.PRESETS:
        A_hi, A_lo, b, A = _parts(name)
        for z in [-0.7, -33.0, 0.1 + 2j]:
            assert tableau.stability_function(A_hi, A_lo, b, z) == pytest.approx(R_scalar(A, b, z), rel=1e-12)


def test_dirk3_gamma_root():
    g = tableau.dirk3_gamma()
    assert abs(g ** 3 - 3 * g * g + 1.5 * g - 1.0 / 6.0) < 1e-15
    assert 0.4358665215 < g < 0.4358665216


def test_tableaux_shapes_lower_triangular():
    for name in tableau.PRESETS:
        A_hi, A_lo, b, _ = _parts(name)
        assert np.all(np.triu(A_hi) == 0.0)
        assert np.all(np.triu(A_lo, 1) == 0.0)


def test_planted_wrong_coefficient_is_caught():
    """A mutation in the oracle's tableau (one sign flipped) must fail a pin."""
    A_hi, A_lo, b = tableau.m4s3pC()
    A_hi = A_hi.copy()
    A_hi[3, 2] = -A_hi[3, 2]
    oc = _order_conditions(A_hi + A_lo, b)
    assert abs(oc[2]) > 1e-3 or abs(oc[3][1]) > 1e-3
