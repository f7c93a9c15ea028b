"""Python binding of librk.so, the B300 (sm_103a) library for mixed-precision
perturbed DIRK time stepping (arXiv 2412.16638).

This module only marshals arguments: every step of the computation runs in
the library's CUDA kernels.  Function names match the C ABI in include/rk.h.
Arrays may be numpy float64 arrays (host) or torch float64 CUDA tensors
(device, passed by pointer).  Errors raise RKError with rk_last_error().
Importing fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import tableaux  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librk.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("librk.so is missing: build it with `python -m paper_2412_16638_b300.build`")
_lib = ctypes.CDLL(LIB_PATH)

# enums
RK_OK, RK_ERR_ARG, RK_ERR_OOM, RK_ERR_CUDA, RK_ERR_NOT_CONVERGED, RK_ERR_NONFINITE, RK_ERR_TIMEOUT, \
    RK_ERR_BUSY, RK_ERR_NOT_FOUND = range(9)
RK_F64, RK_F32, RK_F16, RK_BF16 = range(4)
RK_OP_HEAT7, RK_OP_ADVDIFF_CSR, RK_OP_ADV_PERIODIC = 0, 1, 2
RK_KRYLOV_CG, RK_KRYLOV_GMRES = 0, 1
DTYPES = {"f64": RK_F64, "f32": RK_F32, "f16": RK_F16, "bf16": RK_BF16}
RK_PREC_BLOCK_JACOBI, RK_PREC_FDM = 0, 1
PRECONDS = {"bj": RK_PREC_BLOCK_JACOBI, "fdm": RK_PREC_FDM}


class rk_problem_desc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("n", ctypes.c_int), ("kappa", ctypes.c_double),
                ("kappa_field", ctypes.POINTER(ctypes.c_double)), ("vel", ctypes.c_double * 3),
                ("source", ctypes.POINTER(ctypes.c_double))]


class rk_solver_desc(ctypes.Structure):
    _fields_ = [("krylov", ctypes.c_int), ("restart", ctypes.c_int), ("bj_block", ctypes.c_int),
                ("tol_rel", ctypes.c_double), ("tol_abs", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("storage", ctypes.c_int), ("arith", ctypes.c_int), ("correct", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("tol_true", ctypes.c_double), ("precond", ctypes.c_int),
                ("basis", ctypes.c_int), ("warm_start", ctypes.c_int), ("bj_adapt_tau", ctypes.c_double)]


class rk_stats(ctypes.Structure):
    _fields_ = [("iters_total", ctypes.c_longlong), ("iters_max", ctypes.c_int), ("solves", ctypes.c_int),
                ("refinements", ctypes.c_int), ("not_converged", ctypes.c_int), ("true_res", ctypes.c_double),
                ("seconds", ctypes.c_double), ("bytes", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rk_job_info(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_first_step", ctypes.c_double),
                ("t_done", ctypes.c_double), ("first_tick", ctypes.c_longlong), ("last_tick", ctypes.c_longlong),
                ("steps", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rk_problem_info(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_size_t), ("launches", ctypes.c_longlong), ("bj_blocks", ctypes.c_longlong),
                ("bj_half_blocks", ctypes.c_longlong), ("batch_status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rk_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("noop_launches", ctypes.c_longlong),
                ("ms_total", ctypes.c_double), ("bytes_total", ctypes.c_double)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "rk_create_problem": [ctypes.POINTER(rk_problem_desc), ctypes.POINTER(rk_solver_desc), _P, ctypes.POINTER(_P)],
    "rk_set_tableau": [_P, _I, _DP, _DP, _DP],
    "rk_set_state": [_P, _P, _I],
    "rk_get_state": [_P, _P, _I],
    "rk_step": [_P, _D, ctypes.POINTER(rk_stats)],
    "rk_integrate": [_P, _D, _I, ctypes.POINTER(rk_stats)],
    "rk_destroy_problem": [_P],
    "rk_set_wait_limit": [_P, ctypes.c_ulonglong],
    "rk_get_problem_info": [_P, ctypes.POINTER(rk_problem_info)],
    "rk_check_guards": [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_I)],
    "rk_guard_poke": [_P, _I, ctypes.c_longlong],
    "rk_apply_op": [_P, _P, _P, _I],
    "rk_solve": [_P, _D, _P, _P, _I, ctypes.POINTER(rk_stats)],
    "rk_apply_precond": [_P, _D, _P, _P, _I],
    "rk_integrate_batch": [ctypes.POINTER(_P), _I, _D, _I, ctypes.POINTER(rk_stats)],
    "rk_server_create": [ctypes.c_size_t, _I, ctypes.POINTER(_P)],
    "rk_submit_job": [_P, ctypes.POINTER(rk_problem_desc), ctypes.POINTER(rk_solver_desc), _I, _DP, _DP, _DP,
                      _DP, _D, _I, ctypes.POINTER(ctypes.c_uint64)],
    "rk_poll_job": [_P, ctypes.c_uint64, ctypes.POINTER(_I)],
    "rk_wait_job": [_P, ctypes.c_uint64, _P, ctypes.POINTER(rk_stats), _DP],
    "rk_wait_job_info": [_P, ctypes.c_uint64, _P, ctypes.POINTER(rk_stats), ctypes.POINTER(rk_job_info)],
    "rk_server_destroy": [_P],
    "rk_profile": [_P, _I],
    "rk_heat_solve_noalloc": [_I, _D, _D, _I, _D, _D, _I, _P, _P, _P, ctypes.POINTER(_I)],
    "rk_profile_read": [_P, ctypes.POINTER(rk_kernel_stat), _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.rk_last_error.restype = ctypes.c_char_p
_lib.rk_last_error.argtypes = []
_lib.rk_version.restype = ctypes.c_char_p
_lib.rk_version.argtypes = []

EXPORTED = tuple(_SIGS) + ("rk_last_error", "rk_version")


class RKError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("rk status %d: %s" % (status, msg))
        self.status = status


def rk_last_error() -> str:
    return _lib.rk_last_error().decode()


def rk_version() -> str:
    return _lib.rk_version().decode()


def _check(st, allow=()):
    if st != RK_OK and st not in allow:
        raise RKError(st, rk_last_error())
    return st


def _f64_ptr(a):
    """(pointer, is_device, keepalive) for a float64 numpy array or tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 numpy array")
        return a.ctypes.data_as(_P), 0, a
    if not a.is_contiguous() or str(a.dtype) != "torch.float64":
        raise TypeError("expected a contiguous float64 tensor")
    return _P(a.data_ptr()), (1 if a.is_cuda else 0), a


def _dvec(values):
    return (ctypes.c_double * len(values))(*values)


def problem_desc(op=RK_OP_HEAT7, n=32, kappa=1.0, kappa_field=None, vel=(0.0, 0.0, 0.0), source=None):
    d = rk_problem_desc()
    d.op, d.n, d.kappa = op, n, kappa
    if kappa_field is not None:
        kf = np.ascontiguousarray(kappa_field, dtype=np.float64)
        d._kf = kf  # keeps the array alive as long as the descriptor
        d.kappa_field = kf.ctypes.data_as(_DP)
    if source is not None:
        sf = np.ascontiguousarray(source, dtype=np.float64)
        d._sf = sf
        d.source = sf.ctypes.data_as(_DP)
    d.vel = (ctypes.c_double * 3)(*vel)
    return d


def solver_desc(krylov=RK_KRYLOV_CG, restart=30, bj_block=8, tol_rel=1e-8, tol_abs=0.0, max_iter=1000,
                storage="f32", arith=None, correct=None, max_refine=0, tol_true=0.0, precond="bj", basis=None,
                warm_start=False, bj_adapt_tau=0.0):
    s = rk_solver_desc()
    st = DTYPES[storage] if isinstance(storage, str) else storage
    s.krylov, s.restart, s.bj_block = krylov, restart, bj_block
    s.tol_rel, s.tol_abs, s.max_iter = tol_rel, tol_abs, max_iter
    s.storage = st
    s.arith = (RK_F64 if st == RK_F64 else RK_F32) if arith is None else arith
    s.correct = (0 if st == RK_F64 else 1) if correct is None else int(correct)
    s.max_refine, s.tol_true = max_refine, tol_true
    s.precond = PRECONDS[precond] if isinstance(precond, str) else precond
    s.basis = 0 if basis is None else (DTYPES[basis] if isinstance(basis, str) else basis)
    s.warm_start = int(bool(warm_start))
    s.bj_adapt_tau = float(bj_adapt_tau)
    return s


def rk_create_problem(desc, solver, stream=None):
    h = _P()
    _check(_lib.rk_create_problem(ctypes.byref(desc), ctypes.byref(solver), _P(stream or 0), ctypes.byref(h)))
    return h


def rk_set_tableau(p, A_hi, A_lo, b):
    q = len(b)
    ah = _dvec([float(v) for row in A_hi for v in row])
    al = _dvec([float(v) for row in A_lo for v in row])
    return _check(_lib.rk_set_tableau(p, q, ah, al, _dvec([float(v) for v in b])))


def rk_set_state(p, u):
    ptr, dev, keep = _f64_ptr(u)
    return _check(_lib.rk_set_state(p, ptr, dev))


def rk_get_state(p, out):
    ptr, dev, keep = _f64_ptr(out)
    return _check(_lib.rk_get_state(p, ptr, dev))


def _allow(flag):
    return (RK_ERR_NOT_CONVERGED,) if flag else ()


def rk_step(p, dt, allow_not_converged=False):
    s = rk_stats()
    _check(_lib.rk_step(p, dt, ctypes.byref(s)), _allow(allow_not_converged))
    return s


def rk_integrate(p, dt, nsteps, allow_not_converged=False):
    s = rk_stats()
    _check(_lib.rk_integrate(p, dt, nsteps, ctypes.byref(s)), _allow(allow_not_converged))
    return s


def rk_destroy_problem(p):
    return _check(_lib.rk_destroy_problem(p))


def rk_get_problem_info(p):
    info = rk_problem_info()
    _check(_lib.rk_get_problem_info(p, ctypes.byref(info)))
    return info


def rk_check_guards(p):
    """(corrupted guard bytes, guarded blocks) of a problem created with
    RK_GUARD_BYTES > 0 in the environment."""
    bad = ctypes.c_longlong()
    n = _I()
    _check(_lib.rk_check_guards(p, ctypes.byref(bad), ctypes.byref(n)))
    return bad.value, n.value


def rk_guard_poke(p, block, offset):
    """Test hook: change one byte of a guard band (see rk_check_guards)."""
    return _check(_lib.rk_guard_poke(p, int(block), int(offset)))


def rk_set_wait_limit(p, spins):
    return _check(_lib.rk_set_wait_limit(p, int(spins)))


def rk_apply_op(p, x, y):
    px, dx, kx = _f64_ptr(x)
    py, dy, ky = _f64_ptr(y)
    if dx != dy:
        raise ValueError("x and y must both be host or both be device arrays")
    return _check(_lib.rk_apply_op(p, px, py, dx))


def rk_solve(p, shift, g, k, allow_not_converged=False):
    pg, dg, kg = _f64_ptr(g)
    pk, dk, kk = _f64_ptr(k)
    if dg != dk:
        raise ValueError("g and k must both be host or both be device arrays")
    s = rk_stats()
    _check(_lib.rk_solve(p, shift, pg, pk, dg, ctypes.byref(s)), _allow(allow_not_converged))
    return s


def rk_apply_precond(p, shift, r, z):
    pr, dr, kr = _f64_ptr(r)
    pz, dz, kz = _f64_ptr(z)
    if dr != dz:
        raise ValueError("r and z must both be host or both be device arrays")
    return _check(_lib.rk_apply_precond(p, shift, pr, pz, dr))


def rk_integrate_batch(problems, dt, nsteps, allow_not_converged=False):
    arr = (_P * len(problems))(*[p.value if isinstance(p, _P) else p for p in problems])
    s = rk_stats()
    _check(_lib.rk_integrate_batch(arr, len(problems), dt, nsteps, ctypes.byref(s)), _allow(allow_not_converged))
    return s


def rk_server_create(hbm_budget_bytes, max_slots):
    h = _P()
    _check(_lib.rk_server_create(hbm_budget_bytes, max_slots, ctypes.byref(h)))
    return h


def rk_submit_job(server, desc, solver, A_hi, A_lo, b, u0, dt, nsteps):
    q = len(b)
    ah = _dvec([float(v) for row in A_hi for v in row])
    al = _dvec([float(v) for row in A_lo for v in row])
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    jid = ctypes.c_uint64()
    _check(_lib.rk_submit_job(server, ctypes.byref(desc), ctypes.byref(solver), q, ah, al,
                              _dvec([float(v) for v in b]), u0.ctypes.data_as(_DP), dt, nsteps, ctypes.byref(jid)))
    return jid.value


def rk_poll_job(server, job_id):
    done = ctypes.c_int()
    _check(_lib.rk_poll_job(server, job_id, ctypes.byref(done)))
    return bool(done.value)


def rk_wait_job(server, job_id, u_out=None, allow_not_converged=False):
    s = rk_stats()
    lat = ctypes.c_double()
    ptr = u_out.ctypes.data_as(_P) if u_out is not None else _P(0)
    _check(_lib.rk_wait_job(server, job_id, ptr, ctypes.byref(s), ctypes.byref(lat)), _allow(allow_not_converged))
    return s, lat.value


def rk_wait_job_info(server, job_id, u_out=None, allow_not_converged=False):
    """rk_wait_job that also returns the job's timeline (rk_job_info)."""
    s = rk_stats()
    info = rk_job_info()
    ptr = u_out.ctypes.data_as(_P) if u_out is not None else _P(0)
    _check(_lib.rk_wait_job_info(server, job_id, ptr, ctypes.byref(s), ctypes.byref(info)),
           _allow(allow_not_converged))
    return s, info


def rk_server_destroy(server):
    return _check(_lib.rk_server_destroy(server))


def rk_profile(p, enable=True):
    return _check(_lib.rk_profile(p, 1 if enable else 0))


def rk_profile_read(p):
    """Per-kernel totals since the last rk_profile() call, and the number of
    kernel launches issued: ({name: {launches, noop_launches, ms_total,
    bytes_total}}, launches_total)."""
    buf = (rk_kernel_stat * 64)()
    cnt = ctypes.c_int()
    tot = ctypes.c_longlong()
    _check(_lib.rk_profile_read(p, buf, 64, ctypes.byref(cnt), ctypes.byref(tot)))
    out = {}
    for i in range(cnt.value):
        b = buf[i]
        out[b.name.decode()] = {"launches": b.launches, "noop_launches": b.noop_launches,
                                "ms_total": b.ms_total, "bytes_total": b.bytes_total}
    return out, tot.value


def rk_heat_solve_noalloc(n, kappa, shift, bj_block, tol_rel, tol_abs, max_iter, g, k, stream=None,
                          allow_not_converged=False):
    """Heat stage solve without any device allocation by the library (its
    workspace is a fixed device array; n <= 64).  g, k: float64 CUDA tensors
    of n^3 elements.  Returns the iteration count."""
    pg, dg, kg = _f64_ptr(g)
    pk, dk, kk = _f64_ptr(k)
    if not (dg and dk):
        raise ValueError("g and k must be device tensors")
    it = ctypes.c_int()
    _check(_lib.rk_heat_solve_noalloc(n, kappa, shift, bj_block, tol_rel, tol_abs, max_iter, pg, pk,
                                      _P(stream or 0), ctypes.byref(it)), _allow(allow_not_converged))
    return it.value


class Problem:
    """Owning wrapper: creates the problem, sets tableau and state, frees it."""

    def __init__(self, desc, solver, tableau=None, u0=None, stream=None):
        self.desc, self.solver = desc, solver
        self.n = desc.n
        self.h = None
        self.h = rk_create_problem(desc, solver, stream)
        if tableau is not None:
            if isinstance(tableau, str):
                tableau = tableaux.get(tableau)
            rk_set_tableau(self.h, *tableau)
        if u0 is not None:
            rk_set_state(self.h, np.ascontiguousarray(u0, dtype=np.float64))

    def state(self):
        out = np.empty(self.n ** 3)
        rk_get_state(self.h, out)
        return out

    def close(self):
        if self.h is not None:
            rk_destroy_problem(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
