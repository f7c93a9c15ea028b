"""Seeded synthetic inputs for the DIRK heat / advection-diffusion workloads.

This module is shared by the oracle, the tests and the benchmark. It draws
random numbers and evaluates initial fields and coefficient fields on the
grid; it holds none of the time-stepping or solver arithmetic.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the state advances by the
golden-ratio increment 0x9E3779B97F4A7C15 and each output is the state passed
through the variant-13 mixer of MurmurHash3's finaliser.  Uniform doubles take
the top 53 bits; normal deviates come from the Box-Muller transform.

Grid convention (lexicographic, x fastest): a field on the n^3 interior grid
is a flat float64 array with index i + j*n + k*n*n, the node (i, j, k)
(0-based) sitting at x = (i+1)h, y = (j+1)h, z = (k+1)h with h = 1/(n+1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 stream (one 64-bit state word)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_open(self) -> float:
        """Uniform double in (0, 1]: safe for log()."""
        return ((self.next_u64() >> 11) + 1) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive), by floor of a uniform."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)

    def normal(self) -> float:
        """One standard normal deviate (Box-Muller, cosine branch)."""
        u1 = self.uniform_open()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def split(self) -> "SplitMix64":
        """Child stream seeded from this stream's next output."""
        return SplitMix64(self.next_u64())


def grid_coords(n: int):
    """Node coordinates (x, y, z) as (n,n,n) arrays indexed [k, j, i]."""
    h = 1.0 / (n + 1)
    t = (np.arange(n, dtype=np.float64) + 1.0) * h
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return x, y, z


def sine_mode(n: int, kx: int = 1, ky: int = 1, kz: int = 1) -> np.ndarray:
    """sin(kx pi x) sin(ky pi y) sin(kz pi z) on the interior grid (flat)."""
    h = 1.0 / (n + 1)
    t = (np.arange(n, dtype=np.float64) + 1.0) * h
    sx = np.sin(kx * math.pi * t)
    sy = np.sin(ky * math.pi * t)
    sz = np.sin(kz * math.pi * t)
    return (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]).ravel()


@dataclass
class ModeSum:
    """u0 = sum_m a_m sin(kx_m pi x) sin(ky_m pi y) sin(kz_m pi z)."""
    modes: list = field(default_factory=list)  # list of (a, kx, ky, kz)

    def evaluate(self, n: int) -> np.ndarray:
        h = 1.0 / (n + 1)
        t = (np.arange(n, dtype=np.float64) + 1.0) * h
        out = np.zeros((n, n, n))
        for a, kx, ky, kz in self.modes:
            sx = np.sin(kx * math.pi * t)
            sy = np.sin(ky * math.pi * t)
            sz = np.sin(kz * math.pi * t)
            out += a * (sz[:, None, None] * sy[None, :, None] * sx[None, None, :])
        return out.ravel()


def heat_modes(seed: int = 0, n_random: int = 32, kmax: int = 4, sigma: float = 0.1) -> ModeSum:
    """Unit sine mode plus n_random modes with (kx,ky,kz) uniform in {1..kmax}^3
    (drawn with replacement) and amplitudes N(0, sigma^2), from one SplitMix64
    stream: per mode kx, ky, kz, then the amplitude."""
    rng = SplitMix64(seed)
    modes = [(1.0, 1, 1, 1)]
    for _ in range(n_random):
        kx = rng.randint(1, kmax)
        ky = rng.randint(1, kmax)
        kz = rng.randint(1, kmax)
        a = sigma * rng.normal()
        modes.append((a, kx, ky, kz))
    return ModeSum(modes)


def kappa_field(n: int, seed: int = 0, sigma: float = 0.5, ell: float = 0.1, m_features: int = 256) -> np.ndarray:
    """kappa = exp(g) at the grid nodes, g a stationary Gaussian field with
    standard deviation sigma and correlation length ell, built from
    m_features random Fourier features: g = sigma sqrt(2/M) sum cos(w.x + phi),
    w ~ N(0, ell^-2 I), phi ~ U[0, 2 pi).  Draw order per feature: wx, wy, wz, phi."""
    rng = SplitMix64(seed)
    w = np.empty((m_features, 3))
    phi = np.empty(m_features)
    for m in range(m_features):
        w[m, 0] = rng.normal() / ell
        w[m, 1] = rng.normal() / ell
        w[m, 2] = rng.normal() / ell
        phi[m] = 2.0 * math.pi * rng.uniform()
    x, y, z = grid_coords(n)
    g = np.zeros((n, n, n))
    for m in range(m_features):
        g += np.cos(w[m, 0] * x + w[m, 1] * y + w[m, 2] * z + phi[m])
    g *= sigma * math.sqrt(2.0 / m_features)
    return np.exp(g).ravel()


def gaussian_bump(n: int, width: float = 100.0) -> np.ndarray:
    """exp(-width |x - 1/2|^2) on the interior grid (the advection test's
    initial state); zero boundary values are implied by the grid."""
    x, y, z = grid_coords(n)
    return np.exp(-width * ((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)).ravel()


def periodic_coords(n: int):
    """Node coordinates x_i = i h, h = 1/n, of the periodic grid (the
    advection test), as (n,n,n) arrays indexed [k, j, i]."""
    t = np.arange(n, dtype=np.float64) / n
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return x, y, z


def gaussian_bump_periodic(n: int, width: float = 100.0) -> np.ndarray:
    """exp(-width |x - 1/2|^2) on the periodic grid (flat)."""
    x, y, z = periodic_coords(n)
    return np.exp(-width * ((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)).ravel()


def plane_wave_periodic(n: int, k=(1, 1, 1)) -> np.ndarray:
    """cos(2 pi (k . x)) on the periodic grid (flat)."""
    x, y, z = periodic_coords(n)
    return np.cos(2.0 * math.pi * (k[0] * x + k[1] * y + k[2] * z)).ravel()


@dataclass
class BatchProblem:
    n: int
    kappa: float
    amplitude: float


def batch_problems(count: int = 512, seed: int = 0, nmin: int = 16, nmax: int = 64,
                   kmin: float = 0.1, kmax: float = 10.0) -> list:
    """Independent heat problems: n uniform in {nmin..nmax}, kappa
    log-uniform in [kmin, kmax], initial data amplitude * unit sine mode with
    amplitude uniform in [0.5, 2).  Problem p draws from the child stream
    SplitMix64(seed).split() taken p-th."""
    root = SplitMix64(seed)
    out = []
    for _ in range(count):
        r = root.split()
        n = r.randint(nmin, nmax)
        kappa = math.exp(math.log(kmin) + (math.log(kmax) - math.log(kmin)) * r.uniform())
        amp = 0.5 + 1.5 * r.uniform()
        out.append(BatchProblem(n, kappa, amp))
    return out


@dataclass
class ServeJob:
    arrival: float      # seconds after the start
    n: int
    tableau: str        # "midpoint1" | "sdirk2" | "dirk3"
    storage: str        # "f32" | "f16"
    steps: int
    kappa: float
    amplitude: float


def serve_jobs(count: int = 2000, rate: float = 200.0, seed: int = 0,
               sizes=(32, 64, 96, 128, 192), tableaux=("midpoint1", "sdirk2", "dirk3"),
               storages=("f32", "f16"), steps=(10, 200), kmin=0.1, kmax=10.0) -> list:
    """Poisson arrivals (exponential gaps with mean 1/rate) of heat jobs with
    uniformly drawn size, tableau, storage precision and step count, kappa
    log-uniform, amplitude uniform in [0.5, 2)."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += -math.log(rng.uniform_open()) / rate
        n = sizes[rng.randint(0, len(sizes) - 1)]
        tab = tableaux[rng.randint(0, len(tableaux) - 1)]
        st = storages[rng.randint(0, len(storages) - 1)]
        ns = rng.randint(steps[0], steps[1])
        kappa = math.exp(math.log(kmin) + (math.log(kmax) - math.log(kmin)) * rng.uniform())
        amp = 0.5 + 1.5 * rng.uniform()
        out.append(ServeJob(t, n, tab, st, ns, kappa, amp))
    return out
