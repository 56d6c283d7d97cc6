"""Seeded input generator: published test vector, determinism, shapes."""
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    want = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    s = synth.Stream(0, "x")
    s.key = np.uint64(1234567)
    assert [int(v) for v in s.u64(0, 5)] == want


def test_streams_are_counter_based():
    s = synth.Stream(7, "a")
    full = s.normal(0, 1000)
    assert np.array_equal(full[300:700], s.normal(300, 400))
    assert not np.array_equal(full[:10], synth.Stream(7, "b").normal(0, 10))


def test_normal_moments():
    x = synth.Stream(3, "moments").normal(0, 400000)
    assert abs(x.mean()) < 5e-3 and abs(x.std() - 1) < 5e-3
    u = synth.Stream(3, "u").uniform(0, 400000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 3e-3


def test_positions_distinct_sorted():
    p = synth.sample_positions(1, "pos", 1000, 600)
    assert p.size == 600 and np.all(np.diff(p) > 0) and p[0] >= 0 and p[-1] < 1000
    assert synth.sample_positions(1, "pos", 10, 0).size == 0


def test_c1_shapes_and_determinism():
    a, b = synth.config_c1(), synth.config_c1()
    assert a["X"].dtype == np.float32 and a["X"].shape == (500, 500)
    assert a["A1"].shape == (500, 10) and a["A1"].dtype == np.float32
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["A1"], b["A1"])
    assert a["S_idx"].size == 12500
    R = a["X"].astype(np.float64) - a["U"] @ a["V"].T
    R.ravel()[a["S_idx"]] -= a["S_val"]
    assert abs(R.std() - 1e-3) < 5e-5          # only the N(0, 1e-3^2) noise is left
