"""rk_heat_solve_noalloc: the heat stage solve for callers that cannot
allocate device memory (for example code running inside a memory pool that
owns the whole device, or a host program whose allocator policy forbids
cudaMalloc).  Its workspace is a fixed array inside the library, so these
tests check that two calls in a row on the same array give the same answers
as the allocating rk_solve and as the FP64 oracle's CG, that the device's free
memory does not change across a call once the library's device code is loaded,
and that sizes beyond the array are refused.

This file is collected last on purpose: a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

import synth
from gpu_util import rel_l2, require_gpu
from oracle import krylov, operators

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    return require_gpu()


def _reference(rk, n, kappa, shift, bs, tol, g):
    with rk.Problem(rk.problem_desc(n=n, kappa=kappa),
                    rk.solver_desc(bj_block=bs, tol_rel=tol, storage="f32", max_iter=2000)) as p:
        k = np.empty_like(g)
        st = rk.rk_solve(p.h, shift, g, k)
    return k, st.iters_total


def _oracle(n, kappa, shift, bs, g):
    """Solution of (I - shift L) k = g by the FP64 oracle's block-Jacobi CG,
    solved far below the FP32 tolerance."""
    op = operators.HeatOperator(n, kappa)
    M = krylov.BlockJacobi(krylov.shifted(op.csr(), shift), n, bs)
    res = krylov.pcg(lambda v: v - shift * op.apply(v), M.apply, g, 1e-13, 0.0, 5000)
    assert res.converged
    return res.x


@pytest.mark.parametrize("n,bs", [(40, 8), (64, 16), (17, 32)])
def test_noalloc_matches_rk_solve_and_oracle_twice(rk, n, bs):
    import torch
    kappa, shift, tol = 0.8, 3e-4, 1e-7
    rhs = [operators.heat_apply(synth.heat_modes(seed=s, n_random=8).evaluate(n), n, kappa) for s in (11, 12)]
    for g in rhs:  # two calls in a row share the scratch array
        ref, ref_iters = _reference(rk, n, kappa, shift, bs, tol, g)
        gd = torch.from_numpy(g).cuda()
        kd = torch.full_like(gd, float("nan"))
        it = rk.rk_heat_solve_noalloc(n, kappa, shift, bs, tol, 0.0, 2000, gd, kd)
        torch.cuda.synchronize()
        k = kd.cpu().numpy()
        assert np.all(np.isfinite(k))
        assert rel_l2(k, ref) < 1e-6
        assert it == ref_iters
        # FP32 solve to 1e-7 against the FP64 oracle: within the FP32 bound
        assert rel_l2(k, _oracle(n, kappa, shift, bs, g)) < 1e-6


def test_noalloc_leaves_free_device_memory_unchanged(rk):
    """After a first call has loaded the library's device code and array, a
    further call (here of another size) changes the device's free memory by
    nothing: the entry point allocates no device memory."""
    import torch
    kappa, shift = 1.0, 2e-4
    ga = torch.from_numpy(operators.heat_apply(synth.sine_mode(48), 48, kappa)).cuda()
    ka = torch.empty_like(ga)
    gb = torch.from_numpy(operators.heat_apply(synth.heat_modes(seed=3, n_random=4).evaluate(23), 23, kappa)).cuda()
    kb = torch.empty_like(gb)
    rk.rk_heat_solve_noalloc(48, kappa, shift, 8, 1e-6, 0.0, 500, ga, ka)  # may load the module
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rk.rk_heat_solve_noalloc(23, kappa, shift, 8, 1e-6, 0.0, 500, gb, kb)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert rel_l2(kb.cpu().numpy(), _oracle(23, kappa, shift, 8, gb.cpu().numpy())) < 1e-5


def test_noalloc_refuses_oversize_and_bad_args(rk):
    import torch
    n = 65
    gd = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    kd = torch.zeros_like(gd)
    with pytest.raises(rk.RKError) as e:
        rk.rk_heat_solve_noalloc(n, 1.0, 1e-3, 8, 1e-6, 0.0, 100, gd, kd)
    assert e.value.status == rk.RK_ERR_ARG and "outside 1..64" in str(e.value)
    small = torch.zeros(8 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(rk.RKError):
        rk.rk_heat_solve_noalloc(8, 1.0, 1e-3, 3, 1e-6, 0.0, 100, small, small.clone())
