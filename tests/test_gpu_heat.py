"""Parity of the heat path (7-point stencil, block-Jacobi CG, DIRK stage
loop) against the float64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

import synth
from closed_forms import mode_sum_after, sine_eigenvalue, R_scalar
from gpu_util import rel_l2, require_gpu, rng_vec
from oracle import dirk, krylov, operators, tableau

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    return require_gpu()


def make(rk, n, kappa=1.0, storage="f64", bs=8, tol=1e-12, correct=None, max_iter=5000, tab=None, u0=None,
         **kw):
    return rk.Problem(rk.problem_desc(n=n, kappa=kappa),
                      rk.solver_desc(bj_block=bs, tol_rel=tol, storage=storage, correct=correct,
                                     max_iter=max_iter, **kw),
                      tableau=tab, u0=u0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 33, 64])
def test_operator_apply_f64(rk, n):
    x = rng_vec(n, n)
    with make(rk, n, kappa=0.7) as p:
        y = np.empty_like(x)
        rk.rk_apply_op(p.h, x, y)
    ref = operators.heat_apply(x, n, 0.7)
    np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("storage,tol", [("f64", 1e-14), ("f32", 2e-6), ("f16", 2e-3), ("bf16", 1.6e-2)])
@pytest.mark.parametrize("n,bs", [(5, 1), (17, 4), (33, 8), (40, 16), (37, 32), (9, 32), (24, 2)])
def test_block_jacobi_apply(rk, n, bs, storage, tol):
    shift = 3e-4
    r = rng_vec(n, 100 + n)
    with make(rk, n, storage=storage, bs=bs) as p:
        z = np.empty_like(r)
        rk.rk_apply_precond(p.h, shift, r, z)
    M = krylov.shifted(operators.heat_csr(n, 1.0), shift)
    ref = krylov.BlockJacobi(M, n, bs).apply(r)
    assert rel_l2(z, ref) < tol


@pytest.mark.parametrize("n,bs", [(6, 2), (17, 8), (32, 1), (41, 16), (48, 32)])
def test_cg_solve_f64_matches_oracle(rk, n, bs):
    shift = 2.5e-4
    g = operators.heat_apply(synth.heat_modes(seed=3, n_random=8).evaluate(n), n, 1.0)
    with make(rk, n, storage="f64", bs=bs, tol=1e-12) as p:
        k = np.empty_like(g)
        st = rk.rk_solve(p.h, shift, g, k)
    M = krylov.shifted(operators.heat_csr(n, 1.0), shift)
    bj = krylov.BlockJacobi(M, n, bs)
    ref = krylov.pcg(lambda v: M @ v, bj.apply, g, tol_rel=1e-12, max_iter=5000)
    assert ref.converged and st.iters_total > 0
    assert rel_l2(k, ref.x) < 1e-10
    # same algorithm, same stopping rule: iteration counts agree closely
    assert abs(st.iters_total - ref.iters) <= 2


@pytest.mark.parametrize("storage,tol,bound", [("f32", 1e-6, 1e-5), ("f16", 1e-3, 5e-3), ("bf16", 5e-3, 2e-2)])
def test_cg_solve_low_precision(rk, storage, tol, bound):
    n, shift = 33, 2.5e-4
    g = operators.heat_apply(synth.heat_modes(seed=4, n_random=8).evaluate(n), n, 1.0)
    with make(rk, n, storage=storage, bs=8, tol=tol, max_iter=400) as p:
        k = np.empty_like(g)
        rk.rk_solve(p.h, shift, g, k, allow_not_converged=True)
    M = krylov.shifted(operators.heat_csr(n, 1.0), shift)
    x = krylov.pcg(lambda v: M @ v, krylov.BlockJacobi(M, n, 8).apply, g, tol_rel=1e-13).x
    assert rel_l2(k, x) < bound


def test_solve_dense_tiny(rk):
    n, shift = 3, 0.01
    g = rng_vec(n, 7)
    with make(rk, n, storage="f64", bs=2, tol=1e-14) as p:
        k = np.empty_like(g)
        rk.rk_solve(p.h, shift, g, k)
    M = krylov.shifted(operators.heat_csr(n, 1.0), shift).toarray()
    np.testing.assert_allclose(k, np.linalg.solve(M, g), rtol=1e-12, atol=1e-13)


def test_zero_rhs_solves_in_zero_iterations(rk):
    n = 8
    with make(rk, n, storage="f32", bs=4, tol=1e-6) as p:
        k = np.ones(n ** 3)
        st = rk.rk_solve(p.h, 1e-3, np.zeros(n ** 3), k)
    assert st.iters_total == 0 and np.all(k == 0.0)


def test_config1_fp64_step_parity_and_closed_form(rk):
    """32^3, kappa 1, sine mode, SDIRK2, dt 1e-3, 20 steps, all FP64, CG tol
    1e-12 with scalar Jacobi."""
    n, dt, steps = 32, 1e-3, 20
    u0 = synth.sine_mode(n)
    tab = tableau.sdirk2()
    with make(rk, n, storage="f64", bs=1, tol=1e-12, correct=0, tab="sdirk2", u0=u0) as p:
        st = rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    ref = dirk.integrate(u0, dt, steps, tab, operators.HeatOperator(n, 1.0),
                         dirk.Solver("cg", bs=1, tol_rel=1e-12), corrected=True)
    assert rel_l2(u, ref) < 1e-10
    lam = sine_eigenvalue(n, 1.0, 1, 1, 1)
    exact_discrete = R_scalar(tab[0] + tab[1], tab[2], dt * lam).real ** steps * u0
    assert rel_l2(u, exact_discrete) < 1e-10
    assert rel_l2(u, math.exp(-3 * math.pi ** 2 * 0.02) * u0) < 5e-3
    assert st.solves == 2 * steps


@pytest.mark.parametrize("name", ["midpoint1", "sdirk2", "dirk3", "4s3pB", "4s3pC", "4s3pA"])
def test_fp64_corrected_step_parity_all_tableaux(rk, name):
    n, dt, steps = 20, 1e-3, 3
    u0 = synth.heat_modes(seed=1, n_random=8).evaluate(n)
    with make(rk, n, kappa=0.5, storage="f64", bs=4, tol=1e-12, correct=1, tab=name, u0=u0) as p:
        rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    ref = dirk.integrate(u0, dt, steps, tableau.get(name), operators.HeatOperator(n, 0.5),
                         dirk.Solver("cg", bs=4, tol_rel=1e-12))
    assert rel_l2(u, ref) < 1e-10


@pytest.mark.parametrize("storage,tol,bound", [("f32", 1e-7, 1e-6), ("f16", 1e-3, 5e-3), ("bf16", 1e-3, 5e-3)])
@pytest.mark.parametrize("name", ["sdirk2", "dirk3", "4s3pB"])
def test_mixed_precision_step_within_bound(rk, name, storage, tol, bound):
    """Low-precision implicit solves + FP64 explicit corrections stay within
    the stated bound of the FP64 oracle (40^3: ragged with bs=16)."""
    n, dt, steps = 40, 1e-3, 5
    u0 = synth.heat_modes(seed=0).evaluate(n)
    with make(rk, n, storage=storage, bs=16, tol=tol, correct=1, tab=name, u0=u0, max_iter=500) as p:
        rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
        u = p.state()
    ref = dirk.integrate(u0, dt, steps, tableau.get(name), operators.HeatOperator(n, 1.0),
                         dirk.Solver("cg", bs=16, tol_rel=1e-13))
    assert rel_l2(u, ref) < bound


def test_not_converged_keeps_valid_state(rk):
    n = 16
    u0 = synth.sine_mode(n)
    with make(rk, n, storage="f32", bs=4, tol=1e-12, max_iter=2, tab="sdirk2", u0=u0) as p:
        st = rk.rk_integrate(p.h, 1e-3, 1, allow_not_converged=True)
        u = p.state()
    assert st.not_converged == 2 and st.iters_max == 2
    assert np.all(np.isfinite(u)) and rel_l2(u, u0) < 0.1


def test_bad_tableau_rejected(rk):
    with make(rk, 4) as p:
        with pytest.raises(rk.RKError) as e:
            rk.rk_set_tableau(p.h, [[0.0, 1.0], [0.0, 0.0]], [[0.5, 0], [0, 0.5]], [0.5, 0.5])
        assert e.value.status == rk.RK_ERR_ARG
        with pytest.raises(rk.RKError):
            rk.rk_step(p.h, 1e-3)  # no tableau set


def test_device_pointer_state_roundtrip(rk):
    torch = pytest.importorskip("torch")
    n = 12
    u0 = torch.randn(n ** 3, dtype=torch.float64, device="cuda")
    with make(rk, n, storage="f32", bs=4, tol=1e-6, tab="sdirk2") as p:
        rk.rk_set_state(p.h, u0)
        out = torch.empty_like(u0)
        rk.rk_get_state(p.h, out)
        torch.cuda.synchronize()
        assert torch.equal(out, u0)
        y = torch.empty_like(u0)
        rk.rk_apply_op(p.h, u0, y)
    ref = operators.heat_apply(u0.cpu().numpy(), n, 1.0)
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-13, atol=1e-12 * np.abs(ref).max())


def test_full_size_256_closed_form(rk):
    """The benchmarked configuration (256^3, mixed FP32 storage, SDIRK2,
    block-Jacobi 8) on a mode sum: the fully discrete closed form holds at
    any size; two steps stay within 1e-6 of it."""
    n, dt, steps = 256, 1e-3, 2
    modes = synth.heat_modes(seed=0).modes
    u0 = synth.ModeSum(modes).evaluate(n)
    with make(rk, n, storage="f32", bs=8, tol=1e-6, correct=1, tab="sdirk2", u0=u0, max_iter=500) as p:
        st = rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    A_hi, A_lo, b = tableau.sdirk2()
    exact = mode_sum_after(modes, n, 1.0, dt, steps, A_hi + A_lo, b)
    assert rel_l2(u, exact) < 1e-6
    assert st.solves == 4 and st.true_res < 1e-4


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_full_size_256_16bit_storage_closed_form(rk, storage):
    """16-bit storage of the Krylov vectors at the benchmarked size: at 256^3
    the operator's diagonal kappa/h^2 * 6 = 396294 and 1/h^2 = 66049 exceed the
    FP16 range (65504), so the right-hand side is stored as sigma g with
    sigma = 1/||g||_inf and no operator coefficient is ever rounded to 16 bits.
    Two SDIRK2 steps with block-Jacobi CG at tol 1e-3 stay within 5e-3 of the
    fully discrete closed form."""
    n, dt, steps = 256, 1e-3, 2
    modes = synth.heat_modes(seed=0).modes
    u0 = synth.ModeSum(modes).evaluate(n)
    with make(rk, n, storage=storage, bs=8, tol=1e-3, correct=1, tab="sdirk2", u0=u0, max_iter=500) as p:
        st = rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    A_hi, A_lo, b = tableau.sdirk2()
    exact = mode_sum_after(modes, n, 1.0, dt, steps, A_hi + A_lo, b)
    assert np.all(np.isfinite(u))
    assert rel_l2(u, exact) < 5e-3
    assert st.solves == 4 and st.not_converged == 0


@pytest.mark.parametrize("n,storage,bs", [(64, "f32", 8), (96, "f16", 8), (128, "f64", 4), (32, "bf16", 16),
                                          (256, "f32", 32)])
def test_tiled_sweeps_match_segment_sweeps(rk, n, storage, bs, monkeypatch):
    """The TMA-tiled CG sweeps (chosen when n <= 256 and rows are 16-byte
    aligned) and the per-segment sweeps solve the same system to the solver
    tolerance; both agree with the oracle's converged solution."""
    shift = 2.5e-4
    tol = {"f64": 1e-11, "f32": 1e-6, "f16": 1e-3, "bf16": 5e-3}[storage]
    g = operators.heat_apply(synth.heat_modes(seed=6, n_random=6).evaluate(n), n, 1.0)
    out = {}
    for mode in ("tiled", "segments"):
        if mode == "segments":
            monkeypatch.setenv("RK_NO_TILED", "1")
        with make(rk, n, storage=storage, bs=bs, tol=tol, max_iter=3000) as p:
            k = np.empty_like(g)
            st = rk.rk_solve(p.h, shift, g, k, allow_not_converged=True)
            out[mode] = (k, st.iters_total)
    M = krylov.shifted(operators.heat_csr(n, 1.0), shift) if n <= 64 else None
    bound = {"f64": 1e-9, "f32": 2e-5, "f16": 5e-3, "bf16": 3e-2}[storage]
    assert rel_l2(out["tiled"][0], out["segments"][0]) < bound
    assert abs(out["tiled"][1] - out["segments"][1]) <= max(2, out["segments"][1] // 10)
    if M is not None:
        ref = krylov.pcg(lambda v: M @ v, krylov.BlockJacobi(M, n, bs).apply, g, tol_rel=1e-12).x
        assert rel_l2(out["tiled"][0], ref) < bound


def test_tiled_problems_of_different_sizes_interleaved(rk):
    """Problems of different n share the tiled kernels; solving them in turn
    (large, small, large) must keep working (per-kernel launch limits)."""
    shift = 2.5e-4
    probs = {n: make(rk, n, storage="f32", bs=8, tol=1e-6, max_iter=2000) for n in (96, 64)}
    try:
        for n in (96, 64, 96):
            g = operators.heat_apply(synth.heat_modes(seed=n, n_random=4).evaluate(n), n, 1.0)
            k = np.empty_like(g)
            rk.rk_solve(probs[n].h, shift, g, k)
            M = krylov.shifted(operators.heat_csr(n, 1.0), shift)
            assert np.linalg.norm(g - M @ k) / np.linalg.norm(g) < 1e-4
    finally:
        for p in probs.values():
            p.close()


def test_fp32_correction_matches_fp64_stencil(rk):
    """With FP32 k^eps the FP64 correction k = g + shift * L k^eps forms the
    Laplacian as an exact FP32 pair; a ragged-size DIRK3 run must stay within
    the FP32 bound of the oracle and report a small true residual."""
    n, dt = 37, 1e-3
    u0 = synth.heat_modes(seed=2, n_random=6).evaluate(n)
    with make(rk, n, storage="f32", bs=8, tol=1e-7, correct=1, tab="dirk3", u0=u0, max_iter=500) as p:
        st = rk.rk_integrate(p.h, dt, 3)
        u = p.state()
    ref = dirk.integrate(u0, dt, 3, tableau.dirk3(), operators.HeatOperator(n, 1.0),
                         dirk.Solver("cg", bs=8, tol_rel=1e-13))
    assert rel_l2(u, ref) < 1e-6
    assert 0.0 <= st.true_res < 1e-4


@pytest.mark.parametrize("storage,precond", [("f64", "bj"), ("f32", "bj"), ("f16", "bj"), ("f32", "fdm")])
def test_nonfinite_state_reported(rk, storage, precond):
    """A NaN in the state is caught by the fused reductions of the stage solve
    and reported as RK_ERR_NONFINITE (never a hang or a silent result); the
    problem stays usable after a valid state is set again."""
    n = 32
    u0 = synth.sine_mode(n)
    bad = u0.copy()
    bad[n ** 3 // 2 + 5] = np.nan
    with make(rk, n, storage=storage, bs=8, tol=1e-6, tab="sdirk2", u0=bad, precond=precond) as p:
        with pytest.raises(rk.RKError) as e:
            rk.rk_step(p.h, 1e-3)
        assert e.value.status == rk.RK_ERR_NONFINITE
        rk.rk_set_state(p.h, u0)
        rk.rk_integrate(p.h, 1e-3, 2)
        u = p.state()
    assert np.all(np.isfinite(u)) and rel_l2(u, u0) < 0.1


@pytest.mark.parametrize("storage,precond,tol,bound", [("f64", "bj", 1e-12, 1e-10), ("f32", "bj", 1e-7, 1e-6),
                                                       ("f32", "fdm", 1e-7, 1e-6), ("bf16", "bj", 1e-3, 5e-3)])
def test_warm_start_parity_and_fewer_iterations(rk, storage, precond, tol, bound):
    """Stage solves started from the previous step's solution of the same
    stage: the same bound against the (cold-started) oracle, and no more
    iterations than the cold-started library run."""
    n, dt, steps = 40, 1e-3, 6
    u0 = synth.heat_modes(seed=0).evaluate(n)
    iters = {}
    for warm in (False, True):
        with make(rk, n, storage=storage, bs=8, tol=tol, tab="dirk3", u0=u0, max_iter=2000, precond=precond,
                  warm_start=warm, correct=None if storage == "f64" else 1) as p:
            st = rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
            u = p.state()
        iters[warm] = st.iters_total
        ref = dirk.integrate(u0, dt, steps, tableau.get("dirk3"), operators.HeatOperator(n, 1.0),
                             dirk.Solver("cg", bs=8, tol_rel=1e-13))
        assert rel_l2(u, ref) < bound, (warm, rel_l2(u, ref))
    # never more iterations; strictly fewer with block-Jacobi (the fast
    # diagonalization needs 3 iterations per solve at 1e-7 either way)
    assert iters[True] <= iters[False], iters
    if precond == "bj":
        assert iters[True] < iters[False], iters


def test_warm_start_survives_state_and_tableau_changes(rk):
    n = 24
    u0 = synth.sine_mode(n)
    with make(rk, n, storage="f32", bs=8, tol=1e-7, tab="sdirk2", u0=u0, warm_start=True) as p:
        rk.rk_integrate(p.h, 1e-3, 3)
        rk.rk_set_state(p.h, 2.0 * u0)  # a new state: the old solutions are only guesses
        rk.rk_integrate(p.h, 1e-3, 2)
        u = p.state()
        rk.rk_set_tableau(p.h, *rk.tableaux.get("dirk3"))  # new stages: cold start again
        rk.rk_integrate(p.h, 1e-3, 1)
        v = p.state()
    ref = dirk.integrate(2.0 * u0, 1e-3, 2, tableau.get("sdirk2"), operators.HeatOperator(n, 1.0),
                         dirk.Solver("cg", bs=8, tol_rel=1e-13))
    assert rel_l2(u, ref) < 1e-6
    ref2 = dirk.integrate(ref, 1e-3, 1, tableau.get("dirk3"), operators.HeatOperator(n, 1.0),
                          dirk.Solver("cg", bs=8, tol_rel=1e-13))
    assert rel_l2(v, ref2) < 1e-6


def test_large_grid_512_segment_sweeps_closed_form(rk):
    """512^3 (1.3e8 unknowns, beyond the tiled sweeps' n <= 256): the
    per-segment sweeps and 64-bit indexing at size; one SDIRK2 step of the
    (1,1,1) sine mode against the fully discrete closed form, sampled."""
    n, dt = 512, 1e-3
    u0 = synth.sine_mode(n)
    with make(rk, n, storage="f32", bs=8, tol=1e-6, correct=1, tab="sdirk2", u0=u0, max_iter=2000) as p:
        st = rk.rk_step(p.h, dt)
        u = p.state()
    A_hi, A_lo, b = tableau.sdirk2()
    R = complex(R_scalar(A_hi + A_lo, b, dt * sine_eigenvalue(n, 1.0, 1, 1, 1))).real
    assert st.solves == 2 and st.not_converged == 0
    assert rel_l2(u, R * u0) < 1e-6
    # pointwise: the 1e-6 solver tolerance bounds the error in the 2-norm; a
    # sampled point may deviate a few times more (measured 1.9e-6 of max |u0|)
    idx = np.random.default_rng(0).integers(0, n ** 3, 4096)
    np.testing.assert_allclose(u[idx], R * u0[idx], rtol=0, atol=1e-5 * np.abs(u0).max())


@pytest.mark.parametrize("path", ["single", "batch"])
def test_tiny_state_fp32_storage_scale(rk, path):
    """A state 1e-25 times the unit data (what many steps of a stiff problem
    leave): FP32 products of its right-hand side (~1e-21) would underflow and
    break CG; the power-of-two storage scale keeps the step exact up to the
    scale, so the result is 1e-25 times the unit-data result."""
    n, kappa, dt, steps = 24, 2.0, 1e-3, 3
    u1 = synth.heat_modes(seed=7, n_random=6).evaluate(n)
    tab = rk.tableaux.get("sdirk2")
    outs = []
    for scale in (1.0, 1e-25):
        with rk.Problem(rk.problem_desc(n=n, kappa=kappa),
                        rk.solver_desc(bj_block=8, tol_rel=1e-7, storage="f32", correct=1, max_iter=2000),
                        tableau=tab, u0=scale * u1) as p:
            if path == "single":
                rk.rk_integrate(p.h, dt, steps)
            else:
                rk.rk_integrate_batch([p.h], dt, steps)
            outs.append(p.state() / scale)
    ref = dirk.integrate(u1, dt, steps, tableau.get("sdirk2"), operators.HeatOperator(n, kappa),
                         dirk.Solver("cg", bs=8, tol_rel=1e-13))
    assert rel_l2(outs[0], ref) < 1e-6
    assert rel_l2(outs[1], ref) < 1e-6
