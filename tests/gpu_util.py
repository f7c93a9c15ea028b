"""Helpers for the GPU parity tests: skip without CUDA, build the library,
run the oracle on the same seeded inputs."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _load_build().build()
    import paper_2412_16638_b300 as rk
    return rk


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rng_vec(n, seed):
    """Seeded test vector (numpy's PCG64; input only)."""
    return np.random.default_rng(seed).standard_normal(n ** 3)


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
