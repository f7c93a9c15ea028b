"""Helpers for the GPU parity tests: skip without CUDA, build the library,
run the oracle on the same seeded inputs."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16638_b300.build import build
    build()
    import paper_2412_16638_b300 as rk
    return rk


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rng_vec(n, seed):
    """Seeded test vector (numpy's PCG64; input only)."""
    return np.random.default_rng(seed).standard_normal(n ** 3)
