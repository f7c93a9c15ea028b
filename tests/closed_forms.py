"""Closed forms that pin the oracle and the GPU path (written from the
mathematics, independent of both implementations).

* Sine modes phi_m(x) = sin(kx pi x) sin(ky pi y) sin(kz pi z) are exact
  eigenvectors of the Dirichlet 7-point Laplacian on the grid x_i = (i+1)h,
  h = 1/(n+1), with eigenvalue
      lambda_m = -4 kappa/h^2 sum_d sin^2(k_d pi h / 2).
* For a linear problem one RK step is u_{n+1} = R(tau L) u_n with the
  stability function R(z) = 1 + z b^T (I - z A)^{-1} e (Sec. 2.3); for the
  implicit midpoint rule with any number of corrections R(z) = (2+z)/(2-z)
  (App. A).  Hence a mode sum evolves as sum_m a_m R(tau lambda_m)^N phi_m.
"""
import math

import numpy as np


def sine_eigenvalue(n, kappa, kx, ky, kz):
    h = 1.0 / (n + 1)
    s = sum(math.sin(k * math.pi * h / 2.0) ** 2 for k in (kx, ky, kz))
    return -4.0 * kappa / (h * h) * s


def R_scalar(A, b, z):
    """Scalar stability function by direct q x q solve (plain definition)."""
    A = np.asarray(A, dtype=np.complex128)
    q = A.shape[0]
    return 1.0 + z * (np.asarray(b) @ np.linalg.solve(np.eye(q) - z * A, np.ones(q)))


def R_midpoint(z):
    return (2.0 + z) / (2.0 - z)


def mode_sum_after(modes, n, kappa, dt, nsteps, A, b):
    """Exact fully discrete solution after nsteps for u0 = sum a_m phi_m."""
    from synth import sine_mode
    out = np.zeros(n ** 3)
    for a, kx, ky, kz in modes:
        lam = sine_eigenvalue(n, kappa, kx, ky, kz)
        g = R_scalar(A, b, dt * lam).real
        out += a * g ** nsteps * sine_mode(n, kx, ky, kz)
    return out


def mode_sum_continuous(modes, n, kappa, t):
    """Continuous-in-time solution exp(-pi^2 kappa |k|^2 t) per mode."""
    from synth import sine_mode
    out = np.zeros(n ** 3)
    for a, kx, ky, kz in modes:
        out += a * math.exp(-math.pi ** 2 * kappa * (kx * kx + ky * ky + kz * kz) * t) * sine_mode(n, kx, ky, kz)
    return out


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
