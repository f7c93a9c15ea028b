"""Parity of the advection-diffusion path (CSR operator, per-block
block-Jacobi, restarted GMRES, DIRK stages) against the float64 oracle."""
import functools

import numpy as np
import pytest

import synth
from gpu_util import rel_l2, require_gpu, rng_vec
from oracle import dirk, krylov, operators, tableau

pytestmark = pytest.mark.gpu
VEL = (1.0, 0.5, 0.25)


@pytest.fixture(scope="module")
def rk():
    return require_gpu()


def make(rk, n, storage="f64", bs=8, tol=1e-12, restart=30, correct=None, max_iter=4000, tab=None, u0=None,
         seed=0, vel=VEL):
    kap = synth.kappa_field(n, seed=seed)
    return rk.Problem(rk.problem_desc(op=rk.RK_OP_ADVDIFF_CSR, n=n, kappa_field=kap, vel=vel),
                      rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=restart, bj_block=bs, tol_rel=tol,
                                     storage=storage, correct=correct, max_iter=max_iter),
                      tableau=tab, u0=u0)


@functools.lru_cache(maxsize=None)
def oracle_L(n, seed=0, vel=VEL):
    return operators.advdiff_csr(n, synth.kappa_field(n, seed=seed), vel)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33])
def test_csr_operator_f64(rk, n):
    x = rng_vec(n, 40 + n)
    with make(rk, n) as p:
        y = np.empty_like(x)
        rk.rk_apply_op(p.h, x, y)
    ref = oracle_L(n) @ x
    np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 2e-6), ("f16", 2e-3)])
@pytest.mark.parametrize("n,bs", [(9, 4), (16, 8), (20, 16), (13, 32), (6, 1)])
def test_csr_block_jacobi(rk, n, bs, storage, tol):
    shift = 5e-4
    r = rng_vec(n, 7 + n)
    with make(rk, n, storage=storage, bs=bs) as p:
        z = np.empty_like(r)
        rk.rk_apply_precond(p.h, shift, r, z)
    M = krylov.shifted(oracle_L(n), shift)
    ref = krylov.BlockJacobi(M, n, bs).apply(r)
    assert rel_l2(z, ref) < tol


@pytest.mark.parametrize("n,bs,restart", [(4, 2, 5), (12, 8, 30), (21, 16, 10), (24, 8, 64)])
def test_gmres_f64_matches_oracle(rk, n, bs, restart):
    shift = 5e-4
    g = oracle_L(n) @ synth.gaussian_bump(n)
    with make(rk, n, bs=bs, restart=restart, tol=1e-11) as p:
        k = np.empty_like(g)
        st = rk.rk_solve(p.h, shift, g, k)
    M = krylov.shifted(oracle_L(n), shift)
    ref = krylov.gmres(lambda v: M @ v, krylov.BlockJacobi(M, n, bs).apply, g, restart=restart, tol_rel=1e-11,
                       max_iter=4000)
    assert ref.converged
    assert rel_l2(k, ref.x) < 1e-9
    assert abs(st.iters_total - ref.iters) <= 2
    if n <= 12:
        np.testing.assert_allclose(k, np.linalg.solve(M.toarray(), g), rtol=1e-8, atol=1e-9 * np.abs(g).max())


@pytest.mark.parametrize("storage,tol,bound", [("f32", 1e-6, 1e-5), ("f16", 1e-3, 5e-3), ("bf16", 1e-3, 2e-2)])
def test_gmres_low_precision(rk, storage, tol, bound):
    n, shift = 20, 5e-4
    g = oracle_L(n) @ synth.gaussian_bump(n)
    with make(rk, n, storage=storage, bs=8, tol=tol, max_iter=600) as p:
        k = np.empty_like(g)
        rk.rk_solve(p.h, shift, g, k, allow_not_converged=True)
    M = krylov.shifted(oracle_L(n), shift)
    assert rel_l2(k, np.linalg.solve(M.toarray(), g) if n <= 12 else
                  krylov.gmres(lambda v: M @ v, krylov.BlockJacobi(M, n, 8).apply, g, tol_rel=1e-13).x) < bound


@pytest.mark.parametrize("name", ["dirk3", "sdirk2", "4s3pC"])
def test_step_f64_parity(rk, name):
    n, dt, steps = 14, 5e-4, 3
    u0 = synth.gaussian_bump(n)
    with make(rk, n, bs=8, tol=1e-12, correct=1, tab=name, u0=u0) as p:
        rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    ref = dirk.integrate(u0, dt, steps, tableau.get(name), operators.CSROperator(n, oracle_L(n)),
                         dirk.Solver("gmres", bs=8, tol_rel=1e-12, restart=30))
    assert rel_l2(u, ref) < 1e-10


@pytest.mark.parametrize("storage,tol,bound", [("f32", 1e-7, 1e-6), ("f16", 1e-3, 5e-3)])
def test_step_mixed_within_bound(rk, storage, tol, bound):
    n, dt, steps = 18, 5e-4, 4
    u0 = synth.gaussian_bump(n)
    with make(rk, n, storage=storage, bs=8, tol=tol, correct=1, tab="dirk3", u0=u0, max_iter=800) as p:
        rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
        u = p.state()
    ref = dirk.integrate(u0, dt, steps, tableau.dirk3(), operators.CSROperator(n, oracle_L(n)),
                         dirk.Solver("gmres", bs=8, tol_rel=1e-13, restart=30))
    assert rel_l2(u, ref) < bound


def test_config3_full_size_sampled_rows_and_true_residual(rk):
    """192^3 (the advection-diffusion configuration): operator rows sampled
    and evaluated one by one by the oracle's CSR, and the solve's residual
    recomputed by the oracle's CSR product at full size."""
    n, shift = 192, 0.435866521508459 * 5e-4
    N = n ** 3
    u0 = synth.gaussian_bump(n)
    L = oracle_L(n)
    with make(rk, n, storage="f32", bs=8, tol=1e-6, max_iter=600) as p:
        y = np.empty(N)
        rk.rk_apply_op(p.h, u0, y)
        g = y.copy()
        k = np.empty(N)
        st = rk.rk_solve(p.h, shift, g, k)
    rows = np.random.default_rng(0).choice(N, 2000, replace=False)
    ref_rows = L[rows] @ u0
    np.testing.assert_allclose(y[rows], ref_rows, rtol=1e-12, atol=1e-12 * np.abs(ref_rows).max())
    res = g - (k - shift * (L @ k))
    assert np.linalg.norm(res) / np.linalg.norm(g) < 5e-5
    assert st.iters_total < 600


def test_nonfinite_state_reported(rk):
    """GMRES path: an infinite value in the state is reported as
    RK_ERR_NONFINITE."""
    n = 16
    u0 = synth.gaussian_bump(n)
    bad = u0.copy()
    bad[123] = np.inf
    with make(rk, n, storage="f32", tol=1e-6, correct=1, tab="dirk3", u0=bad) as p:
        with pytest.raises(rk.RKError) as e:
            rk.rk_step(p.h, 5e-4)
        assert e.value.status == rk.RK_ERR_NONFINITE


@pytest.mark.parametrize("n,tol", [(16, 1e-6), (33, 1e-7)])
def test_gmres_compressed_basis(rk, n, tol):
    """FP32 GMRES with the Krylov basis stored in BF16 (FP32 arithmetic): the
    solve still reaches the FP32 tolerance on the recursive residual and
    agrees with the oracle's tight solution to the tolerance times a modest
    factor; iterations may grow against the FP32 basis."""
    shift = 4e-4
    g = oracle_L(n) @ synth.gaussian_bump(n)
    out = {}
    for basis in (None, "bf16"):
        p = rk.Problem(rk.problem_desc(op=rk.RK_OP_ADVDIFF_CSR, n=n, kappa_field=synth.kappa_field(n, seed=0),
                                       vel=VEL),
                       rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=tol,
                                      storage="f32", max_iter=2000, basis=basis))
        with p:
            k = np.empty_like(g)
            st = rk.rk_solve(p.h, shift, g, k)
        out[basis] = (k, st.iters_total)
    M = krylov.shifted(oracle_L(n), shift)
    ref = krylov.gmres(lambda v: M @ v, krylov.BlockJacobi(M, n, 8).apply, g, restart=30, tol_rel=1e-13).x
    e32, ebf = rel_l2(out[None][0], ref), rel_l2(out["bf16"][0], ref)
    assert e32 < 50 * tol and ebf < 50 * tol, (e32, ebf)
    assert out["bf16"][1] <= 2 * out[None][1] + 5


def test_step_compressed_basis_within_fp32_bound(rk):
    n, dt, steps = 24, 5e-4, 4
    u0 = synth.gaussian_bump(n)
    p = rk.Problem(rk.problem_desc(op=rk.RK_OP_ADVDIFF_CSR, n=n, kappa_field=synth.kappa_field(n, seed=0), vel=VEL),
                   rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=8, tol_rel=1e-8, storage="f32",
                                  max_iter=3000, correct=1, basis="bf16"),
                   tableau="dirk3", u0=u0)
    with p:
        rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
        u = p.state()
    ref = dirk.integrate(u0, dt, steps, tableau.get("dirk3"), operators.CSROperator(n, oracle_L(n)),
                         dirk.Solver("gmres", bs=8, tol_rel=1e-13))
    assert rel_l2(u, ref) < 1e-6


def _adaptive(rk, n, tau, tol=1e-7, correct=None, tab=None, u0=None, bs=8):
    return rk.Problem(rk.problem_desc(op=rk.RK_OP_ADVDIFF_CSR, n=n, kappa_field=synth.kappa_field(n, seed=0),
                                      vel=VEL),
                      rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, restart=30, bj_block=bs, tol_rel=tol, storage="f32",
                                     max_iter=3000, correct=correct, bj_adapt_tau=tau),
                      tableau=tab, u0=u0)


@pytest.mark.parametrize("n,bs,shift", [(20, 8, 5e-3), (13, 4, 2e-2)])
def test_csr_block_jacobi_adaptive_precision(rk, n, bs, shift):
    """Adaptive-precision block-Jacobi: with tau between two blocks' condition
    numbers, the library stores the same blocks in FP16 as the oracle's rule,
    and z = D^{-1} r matches the oracle's rounded inverses to FP32 arithmetic."""
    M = krylov.shifted(oracle_L(n), shift)
    kap = np.sort(np.concatenate(krylov.AdaptiveBlockJacobi(M, n, bs).kappas))
    mid = len(kap) // 2
    assert kap[mid] > kap[mid - 1]
    tau = 0.5 * (kap[mid - 1] + kap[mid]) * krylov.U_HALF
    ref_bj = krylov.AdaptiveBlockJacobi(M, n, bs, tau=tau)
    r = rng_vec(n, 77)
    with _adaptive(rk, n, tau, bs=bs) as p:
        z = np.empty_like(r)
        rk.rk_apply_precond(p.h, shift, r, z)
        info = rk.rk_get_problem_info(p.h)
    assert info.bj_blocks == ref_bj.total_blocks
    assert info.bj_half_blocks == ref_bj.low_blocks
    assert 0 < ref_bj.low_blocks < ref_bj.total_blocks
    # the library rounds r to FP32 and applies in FP32 arithmetic
    assert rel_l2(z, ref_bj.apply(r.astype(np.float32).astype(np.float64))) < 2e-6


def test_gmres_and_step_with_adaptive_block_jacobi(rk):
    """GMRES with every block stored in FP16 (tau 1e-2: the blocks of this
    operator have kappa_1 < 6) still converges to the oracle's solution at the
    FP32 tolerance, and a mixed-precision step stays within the FP32 bound."""
    n, shift = 24, 5e-4
    g = oracle_L(n) @ synth.gaussian_bump(n)
    with _adaptive(rk, n, 1e-2) as p:
        k = np.empty_like(g)
        st = rk.rk_solve(p.h, shift, g, k)
        info = rk.rk_get_problem_info(p.h)
    assert info.bj_half_blocks == info.bj_blocks > 0
    M = krylov.shifted(oracle_L(n), shift)
    ref = krylov.gmres(lambda v: M @ v, krylov.BlockJacobi(M, n, 8).apply, g, restart=30, tol_rel=1e-13).x
    assert rel_l2(k, ref) < 5e-6 and st.iters_total < 300
    dt, steps = 5e-4, 3
    u0 = synth.gaussian_bump(n)
    with _adaptive(rk, n, 1e-2, tol=1e-8, correct=1, tab="dirk3", u0=u0) as p:
        rk.rk_integrate(p.h, dt, steps)
        u = p.state()
    ref_u = dirk.integrate(u0, dt, steps, tableau.dirk3(), operators.CSROperator(n, oracle_L(n)),
                           dirk.Solver("gmres", bs=8, tol_rel=1e-13, restart=30))
    assert rel_l2(u, ref_u) < 1e-6


def test_tiny_state_fp32_storage_scale_gmres(rk):
    """GMRES path with a state 1e-25 times the bump: the power-of-two storage
    scale keeps the FP32 solve clear of underflow, so the step equals 1e-25
    times the unit-data step."""
    n, dt, steps = 18, 5e-4, 2
    u0 = synth.gaussian_bump(n)
    outs = []
    for scale in (1.0, 1e-25):
        with make(rk, n, storage="f32", bs=8, tol=1e-7, correct=1, tab="dirk3", u0=scale * u0, max_iter=800) as p:
            rk.rk_integrate(p.h, dt, steps, allow_not_converged=True)
            outs.append(p.state() / scale)
    ref = dirk.integrate(u0, dt, steps, tableau.dirk3(), operators.CSROperator(n, oracle_L(n)),
                         dirk.Solver("gmres", bs=8, tol_rel=1e-13, restart=30))
    assert rel_l2(outs[0], ref) < 1e-6
    assert rel_l2(outs[1], ref) < 1e-6
