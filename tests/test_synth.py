"""The seeded generators: published SplitMix64 outputs and determinism."""
import json
import os

import numpy as np

import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")))


def test_splitmix64_published_vectors():
    r = synth.SplitMix64(1234567)
    assert [str(r.next_u64()) for _ in range(5)] == GOLD["seed_1234567_first5"]
    r = synth.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [int(h, 16) for h in GOLD["seed_0_first3_hex"]]


def test_generators_deterministic_and_in_range():
    a = synth.heat_modes(seed=5).evaluate(9)
    b = synth.heat_modes(seed=5).evaluate(9)
    assert np.array_equal(a, b)
    m = synth.heat_modes(seed=0)
    assert len(m.modes) == 33 and m.modes[0] == (1.0, 1, 1, 1)
    assert all(1 <= k <= 4 for _, kx, ky, kz in m.modes for k in (kx, ky, kz))
    probs = synth.batch_problems(512, seed=0)
    assert all(16 <= p.n <= 64 and 0.1 <= p.kappa <= 10 for p in probs)
    assert len({p.n for p in probs}) > 40
    kap = synth.kappa_field(6, seed=0)
    assert kap.shape == (216,) and np.all(kap > 0)
    g = np.log(synth.kappa_field(24, seed=0))
    assert 0.2 < g.std() < 0.8       # sigma = 0.5 up to sampling error
    jobs = synth.serve_jobs(200, seed=0)
    gaps = np.diff([0.0] + [j.arrival for j in jobs])
    assert 0.003 < gaps.mean() < 0.008  # mean 1/200 s
