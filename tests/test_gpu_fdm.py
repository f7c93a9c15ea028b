"""Parity of the tensor-core fast-diagonalization preconditioner (Sec. 3,
Eqs. preconbasic, Pinvform, TensorDecomp) and of CG / the DIRK step that use
it, against the float64 oracle, through the C ABI.

Tolerance of a single application P^-1 r: six passes, each rounding its
operands to the tensor-core input type (TF32: 10 mantissa bits, truncated;
FP16: 10 bits; BF16: 7 bits) and its output to the storage type, so at most
about 3 roundings of unit u per pass enter; with 6 passes the relative error
is bounded (to first order, without cancellation) by 18 u:
TF32 18 * 2^-10 = 1.8e-2, FP16 18 * 2^-11 = 8.8e-3, BF16 18 * 2^-8 = 7.0e-2.
"""
import numpy as np
import pytest

import synth
from closed_forms import mode_sum_after
from gpu_util import rel_l2, require_gpu, rng_vec
from oracle import dirk, fdm, krylov, operators, tableau

pytestmark = pytest.mark.gpu

BOUND = {"f32": 18 * 2.0 ** -10, "f16": 18 * 2.0 ** -11, "bf16": 18 * 2.0 ** -8}


@pytest.fixture(scope="module")
def rk():
    return require_gpu()


def make(rk, n, kappa=1.0, storage="f32", tol=1e-6, correct=None, max_iter=200, tab=None, u0=None, **kw):
    return rk.Problem(rk.problem_desc(n=n, kappa=kappa),
                      rk.solver_desc(tol_rel=tol, storage=storage, correct=correct, max_iter=max_iter,
                                     precond="fdm", **kw),
                      tableau=tab, u0=u0)


# n = 8, 24: the only / last 128-row tile ragged (64, 576 rows) and the 128-byte
# K block partly beyond n; n = 48: 1.5 K blocks (FP32); n = 136, 200, 256: two
# N tiles (the second one ragged for 136 and 200)
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("n", [8, 16, 24, 48, 64, 136, 200, 256])
def test_fdm_apply_matches_oracle(rk, n, storage):
    shift = 3e-4
    r = rng_vec(n, 7 * n + 1)
    with make(rk, n, kappa=0.8, storage=storage) as p:
        z = np.empty_like(r)
        rk.rk_apply_precond(p.h, shift, r, z)
    ref = fdm.FastDiagonalization(n, 0.8, shift).apply(r)
    err = rel_l2(z, ref)
    assert err < BOUND[storage], err


@pytest.mark.parametrize("n", [20, 36])
def test_fdm_apply_ragged_fp32(rk, n):
    shift = 1e-3
    r = rng_vec(n, 3 * n)
    with make(rk, n, storage="f32") as p:
        z = np.empty_like(r)
        rk.rk_apply_precond(p.h, shift, r, z)
    ref = fdm.FastDiagonalization(n, 1.0, shift).apply(r)
    assert rel_l2(z, ref) < BOUND["f32"]


def test_fdm_apply_is_linear_and_repeatable(rk):
    n, shift = 64, 5e-4
    a, b = rng_vec(n, 1), rng_vec(n, 2)
    with make(rk, n) as p:
        za, zb, zab, za2 = (np.empty_like(a) for _ in range(4))
        rk.rk_apply_precond(p.h, shift, a, za)
        rk.rk_apply_precond(p.h, shift, b, zb)
        rk.rk_apply_precond(p.h, shift, a + b, zab)
        rk.rk_apply_precond(p.h, shift, a, za2)
    assert np.array_equal(za, za2)  # fixed summation order: bitwise repeatable
    assert rel_l2(zab, za + zb) < 2 * BOUND["f32"]


@pytest.mark.parametrize("storage,tol,bound", [("f32", 1e-6, 1e-5), ("f16", 1e-3, 5e-3), ("bf16", 5e-3, 2e-2)])
@pytest.mark.parametrize("n", [32, 64])
def test_fdm_cg_solve_matches_oracle(rk, n, storage, tol, bound):
    shift = 2.5e-4
    g = operators.heat_apply(synth.heat_modes(seed=4, n_random=8).evaluate(n), n, 1.0)
    with make(rk, n, storage=storage, tol=tol) as p:
        k = np.empty_like(g)
        st = rk.rk_solve(p.h, shift, g, k)
    P = fdm.FastDiagonalization(n, 1.0, shift)
    apply_A = lambda v: v - shift * operators.heat_apply(v, n, 1.0)
    ref = krylov.pcg(apply_A, P.apply, g, tol_rel=1e-13)
    assert ref.iters == 1
    assert rel_l2(k, ref.x) < bound
    # a nearly exact preconditioner: a handful of iterations, where block-Jacobi needs tens
    assert 1 <= st.iters_total <= 8


def test_fdm_step_parity_fp32(rk):
    """Mixed FP32 + FDM DIRK steps stay within the FP32 bound of the FP64
    oracle (same tableau, FP64 solves to 1e-13)."""
    n, dt, steps = 48, 1e-3, 5
    u0 = synth.heat_modes(seed=0).evaluate(n)
    for name in ("sdirk2", "dirk3"):
        with make(rk, n, storage="f32", tol=1e-7, correct=1, tab=name, u0=u0) as p:
            st = rk.rk_integrate(p.h, dt, steps)
            u = p.state()
        ref = dirk.integrate(u0, dt, steps, tableau.get(name), operators.HeatOperator(n, 1.0),
                             dirk.Solver("cg", tol_rel=1e-13, precond="fdm"))
        assert rel_l2(u, ref) < 1e-6
        assert st.iters_max <= 8


@pytest.mark.parametrize("storage,bound", [("f16", 5e-3), ("bf16", 5e-3)])
def test_fdm_step_parity_16bit(rk, storage, bound):
    n, dt, steps = 32, 1e-3, 5
    u0 = synth.heat_modes(seed=1).evaluate(n)
    with make(rk, n, storage=storage, tol=1e-3, correct=1, tab="sdirk2", u0=u0) as p:
        rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
        u = p.state()
    ref = dirk.integrate(u0, dt, steps, tableau.get("sdirk2"), operators.HeatOperator(n, 1.0),
                         dirk.Solver("cg", tol_rel=1e-13, precond="fdm"))
    assert rel_l2(u, ref) < bound


def test_fdm_full_size_256_closed_form(rk):
    """256^3 with FP32 storage, SDIRK2 and the FDM preconditioner: the fully
    discrete closed form of a mode sum holds at any size."""
    n, dt, steps = 256, 1e-3, 2
    modes = synth.heat_modes(seed=0).modes
    u0 = synth.ModeSum(modes).evaluate(n)
    with make(rk, n, storage="f32", tol=1e-6, correct=1, tab="sdirk2", u0=u0) as p:
        st = rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    A_hi, A_lo, b = tableau.sdirk2()
    exact = mode_sum_after(modes, n, 1.0, dt, steps, A_hi + A_lo, b)
    assert rel_l2(u, exact) < 1e-6
    assert st.solves == 4 and st.iters_max <= 8


def test_fdm_tiled_and_segment_sweeps_agree(rk, monkeypatch):
    n, shift = 64, 2.5e-4
    g = operators.heat_apply(synth.heat_modes(seed=9, n_random=6).evaluate(n), n, 1.0)
    out = []
    for mode in ("tiled", "segments"):
        if mode == "segments":
            monkeypatch.setenv("RK_NO_TILED", "1")
        with make(rk, n, storage="f32", tol=1e-6) as p:
            k = np.empty_like(g)
            st = rk.rk_solve(p.h, shift, g, k)
            out.append((k, st.iters_total))
    assert rel_l2(out[0][0], out[1][0]) < 1e-5
    assert abs(out[0][1] - out[1][1]) <= 1


def test_fdm_zero_rhs(rk):
    n = 32
    with make(rk, n) as p:
        g = np.zeros(n ** 3)
        k = np.ones_like(g)
        st = rk.rk_solve(p.h, 1e-3, g, k)
    assert st.iters_total == 0 and not k.any()


def test_fdm_rejected_by_batch(rk):
    with make(rk, 16, tab="sdirk2", u0=np.zeros(16 ** 3)) as p:
        with pytest.raises(rk.RKError) as e:
            rk.rk_integrate_batch([p.h], 1e-3, 1)
        assert e.value.status == rk.RK_ERR_ARG
