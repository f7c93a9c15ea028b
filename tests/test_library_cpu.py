"""The C-ABI library without a GPU: it loads, exports every entry point that
include/rk.h declares, and rejects bad descriptors before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rk():
    _load_build().build()
    import paper_2412_16638_b300 as mod
    return mod


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "rk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rk_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(rk):
    names = declared_symbols()
    assert len(names) >= 18
    lib = ctypes.CDLL(rk.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(rk.EXPORTED)
    assert "sm_103a" in rk.rk_version()


def test_argument_checks_without_gpu(rk):
    h = ctypes.c_void_p()
    d = rk.problem_desc(n=0)
    s = rk.solver_desc()
    assert rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h)) == rk.RK_ERR_ARG
    assert "n must be" in rk.rk_last_error()
    d = rk.problem_desc(n=8)
    s = rk.solver_desc(bj_block=3)
    assert rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h)) == rk.RK_ERR_ARG
    assert "bj_block" in rk.rk_last_error()
    s = rk.solver_desc(storage="f16", arith=rk.RK_F64)
    assert rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h)) == rk.RK_ERR_ARG
    d = rk.problem_desc(op=rk.RK_OP_ADVDIFF_CSR, n=8)
    s = rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES)
    assert rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h)) == rk.RK_ERR_ARG
    assert "kappa_field" in rk.rk_last_error()
    assert rk._lib.rk_step(None, 1e-3, None) == rk.RK_ERR_ARG
    assert rk._lib.rk_destroy_problem(None) == rk.RK_ERR_ARG


def test_fdm_argument_checks_without_gpu(rk):
    """The fast-diagonalization preconditioner is accepted only where it is
    built: CG on the heat operator, low-precision storage, n <= 256 and
    16-byte rows."""
    h = ctypes.c_void_p()

    def create(d, s):
        return rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h))

    heat = rk.problem_desc(n=64)
    assert create(heat, rk.solver_desc(precond=7)) == rk.RK_ERR_ARG
    assert "preconditioner" in rk.rk_last_error()
    assert create(heat, rk.solver_desc(precond="fdm", storage="f64")) == rk.RK_ERR_ARG
    assert "tensor cores" in rk.rk_last_error()
    assert create(rk.problem_desc(n=300), rk.solver_desc(precond="fdm")) == rk.RK_ERR_ARG
    assert create(rk.problem_desc(n=10), rk.solver_desc(precond="fdm")) == rk.RK_ERR_ARG  # 40-byte rows
    assert create(rk.problem_desc(n=12), rk.solver_desc(precond="fdm", storage="f16")) == rk.RK_ERR_ARG
    assert "16-byte rows" in rk.rk_last_error()
    assert create(heat, rk.solver_desc(precond="fdm", krylov=rk.RK_KRYLOV_GMRES)) == rk.RK_ERR_ARG


def test_periodic_and_forcing_argument_checks_without_gpu(rk):
    h = ctypes.c_void_p()

    def create(d, s):
        return rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h))

    gm = rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES)
    assert create(rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=2, vel=(1, 1, 1)), gm) == rk.RK_ERR_ARG
    assert "n >= 3" in rk.rk_last_error()
    assert create(rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=8, vel=(1, float("nan"), 1)), gm) == rk.RK_ERR_ARG
    assert create(rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=8, vel=(1, 1, 1)), rk.solver_desc()) == rk.RK_ERR_ARG
    assert "CG" in rk.rk_last_error()
    assert create(rk.problem_desc(n=8), gm) == rk.RK_ERR_ARG
    assert create(rk.problem_desc(op=7, n=8), rk.solver_desc()) == rk.RK_ERR_ARG


def test_compressed_basis_argument_checks_without_gpu(rk):
    h = ctypes.c_void_p()
    d = rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=8, vel=(1, 1, 1))

    def create(s):
        return rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h))

    assert create(rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, storage="f64", basis="bf16")) == rk.RK_ERR_ARG
    assert "basis" in rk.rk_last_error()
    assert create(rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, storage="f32", basis="f16")) == rk.RK_ERR_ARG
    heat = rk.problem_desc(n=8)
    assert rk._lib.rk_create_problem(ctypes.byref(heat), ctypes.byref(rk.solver_desc(basis="bf16")), None,
                                     ctypes.byref(h)) == rk.RK_ERR_ARG


def test_warm_start_argument_checks_without_gpu(rk):
    h = ctypes.c_void_p()
    d = rk.problem_desc(n=8)

    def create(s, desc=d):
        return rk._lib.rk_create_problem(ctypes.byref(desc), ctypes.byref(s), None, ctypes.byref(h))

    assert create(rk.solver_desc(storage="f16", warm_start=True)) == rk.RK_ERR_ARG
    assert "warm_start" in rk.rk_last_error()
    per = rk.problem_desc(op=rk.RK_OP_ADV_PERIODIC, n=8, vel=(1, 1, 1))
    assert create(rk.solver_desc(krylov=rk.RK_KRYLOV_GMRES, warm_start=True), per) == rk.RK_ERR_ARG
    s = rk.solver_desc()
    s.warm_start = 2
    assert create(s) == rk.RK_ERR_ARG


def test_package_tableaux_match_oracle(rk):
    """The library's tableau table and the oracle's are typed independently
    from the paper; they must agree."""
    from oracle import tableau
    for name in rk.tableaux.PRESETS:
        mine = [np.array(x) for x in rk.tableaux.get(name)]
        ref = tableau.get(name)
        for a, b in zip(mine, ref):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def _load_build():
    """The build module, loaded by file path so that building never imports
    a stale copy of the library."""
    import importlib.util
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "paper_2412_16638_b300", "build.py")
    if not os.path.exists(path):
        path = os.path.join(os.path.dirname(here), "paper_2412_16638_b300", "build.py")
    spec = importlib.util.spec_from_file_location("_rk_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_solver_option_checks_without_gpu(rk):
    """Options accepted only where they are built: adaptive-precision
    block-Jacobi on the CSR operators with FP32 storage; warm starts not
    combined with refinement.  Checked before any CUDA call."""
    h = ctypes.c_void_p()
    d = rk.problem_desc(n=8)
    s = rk.solver_desc(storage="f32", bj_adapt_tau=1e-2)
    assert rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h)) == rk.RK_ERR_ARG
    assert "adaptive-precision" in rk.rk_last_error()
    s = rk.solver_desc(storage="f32", bj_adapt_tau=-1.0)
    assert rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h)) == rk.RK_ERR_ARG
    s = rk.solver_desc(storage="f32", max_refine=2, tol_true=1e-9, warm_start=True)
    assert rk._lib.rk_create_problem(ctypes.byref(d), ctypes.byref(s), None, ctypes.byref(h)) == rk.RK_ERR_ARG
    assert "warm_start" in rk.rk_last_error()
    assert rk._lib.rk_set_wait_limit(None, 1) == rk.RK_ERR_ARG
    info = rk.rk_problem_info()
    assert rk._lib.rk_get_problem_info(None, ctypes.byref(info)) == rk.RK_ERR_ARG
