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


def forced_sine_after(n, kappa, dt, nsteps, A, b, u0_amp=0.0):
    """du/dt = L u + phi with phi the (1,1,1) sine mode and u0 = u0_amp phi:
    the RK step maps the deviation from the fixed point u* = -phi / lambda_1
    by R(dt lambda_1), so u_N = u* + R^N (u0 - u*) exactly (fully discrete).
    Returns (u_N, semi-discrete exact solution at t = N dt)."""
    from synth import sine_mode
    lam = sine_eigenvalue(n, kappa, 1, 1, 1)
    R = complex(R_scalar(A, b, dt * lam)).real
    ustar = -1.0 / lam
    phi = sine_mode(n)
    disc = (ustar + R ** nsteps * (u0_amp - ustar)) * phi
    cont = (ustar + math.exp(lam * dt * nsteps) * (u0_amp - ustar)) * phi
    return disc, cont


def periodic_wave_eigenvalue(n, beta, k):
    """Eigenvalue of L = -sum_d beta_d D_d (central, periodic, h = 1/n) for the
    Fourier mode exp(2 pi i k . x): -i sum_d beta_d sin(2 pi k_d h) / h."""
    h = 1.0 / n
    return -1j * sum(bd * math.sin(2.0 * math.pi * kd * h) / h for bd, kd in zip(beta, k))


def plane_wave_after(n, beta, k, dt, nsteps, A, b):
    """u0 = cos(2 pi k . x) on the periodic grid: u_N = Re(R(dt lam)^N e^{i theta})
    (fully discrete), and Re(e^{lam t} e^{i theta}) (semi-discrete)."""
    from synth import periodic_coords
    x, y, z = periodic_coords(n)
    theta = (2.0 * math.pi * (k[0] * x + k[1] * y + k[2] * z)).ravel()
    lam = periodic_wave_eigenvalue(n, beta, k)
    R = complex(R_scalar(A, b, dt * lam))
    disc = np.real(R ** nsteps * np.exp(1j * theta))
    cont = np.real(np.exp(lam * dt * nsteps) * np.exp(1j * theta))
    return disc, cont
