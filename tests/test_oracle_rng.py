"""Pins for the oracle's initial-value generator (CPU only)."""
import json
import os

import numpy as np

from oracle.rng import init_values, splitmix64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64_seed0.json")))
    got = splitmix64(g["seed"], 0, np.arange(3))
    assert [f"{int(v):016x}" for v in got] == g["outputs_hex"]


def test_stream_offsets_are_consistent():
    a = init_values(7, 3, 1000, 0.5)
    b = init_values(7, 3, 600, 0.5, start=400)
    assert np.array_equal(a[400:], b)


def test_values_are_fp32_symmetric_uniform():
    bound = 1.0 / np.sqrt(512.0)
    v = init_values(11, 5, 200_000, bound)
    assert np.array_equal(v, v.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(v) < np.float32(bound))
    n = v.size
    # Uniform(-a, a): mean 0 (sd a/sqrt(3n)), variance a^2/3 (rel. sd ~ sqrt(0.8/n)).
    assert abs(v.mean()) < 5 * bound / np.sqrt(3 * n)
    assert abs(v.var() / (bound ** 2 / 3) - 1) < 5 * np.sqrt(0.8 / n)


def test_tensors_are_decorrelated():
    a = init_values(1, 0, 50_000, 1.0)
    b = init_values(1, 1, 50_000, 1.0)
    c = init_values(2, 0, 50_000, 1.0)
    for x, y in ((a, b), (a, c)):
        r = np.corrcoef(x, y)[0, 1]
        assert abs(r) < 5 / np.sqrt(x.size)
