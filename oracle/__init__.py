"""FP64 CPU oracle for the mixed-precision DIRK stage loop (arXiv 2412.16638).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or execute anything in this
package.  The CUDA library never calls it and shares no code with it; the only
common dependency is the seeded input generator in ``synth``.

Everything here is plain numpy/scipy in float64, written to be read against
the paper:

* ``tableau``   -- Butcher tableaux split as A = A^(h) + A^(eps) (Sec. 2.1,
                   Fig. fig_Aq_rat; Sec. 2.2, Tables ButchertabA/B/C) and the
                   stability function R(z) (Sec. 2.3).
* ``operators`` -- the semi-discrete operators du/dt = K u (Sec. 3, Sec. 5.2):
                   7-point heat stencil, upwind advection-diffusion in CSR.
* ``krylov``    -- block-Jacobi, preconditioned CG and restarted GMRES for the
                   stage systems (Sec. 3, Eq. corelinear; stopping rule of
                   Sec. 5.3).
* ``fdm``       -- the fast-diagonalization preconditioner (Sec. 3, Eqs.
                   preconbasic, Pinvform, TensorDecomp) for the heat stage
                   matrix.
* ``dirk``      -- the perturbed stage loop (Sec. 2.2.1, Eqs. mpAstep1-5;
                   Sec. 4.2 precision policy), all in float64.

Parity status: every function is pinned by the CPU tests (order conditions,
the closed-form R(z) of App. A, sine-mode eigenpairs, dense/Kronecker direct
solves, observed order).  The variable-coefficient advection-diffusion
operator at full size has no closed form: beyond the tiny-grid brute-force and
dense pins it is "parity unpinned beyond the oracle".
"""
from . import tableau, operators, krylov, fdm, dirk  # noqa: F401
