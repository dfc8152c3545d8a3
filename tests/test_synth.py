"""The seeded generator: reproducible, counter-based, and shaped as requested (CPU only)."""
import math

import numpy as np

from paper_2505_12414_gb300 import synth


def test_splitmix64_reference_values():
    # SplitMix64 from state 0: the first outputs of the published generator
    # (Steele, Lea & Flood 2014; also the seeding routine recommended for xoshiro)
    z = np.array([0], dtype=np.uint64)
    out = []
    state = 0
    for _ in range(3):
        state = (state + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
        out.append(int(synth._mix(np.array([state], dtype=np.uint64))[0]))
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert z.dtype == np.uint64


def test_streams_are_reproducible_and_sliceable():
    a = synth.Stream(123, 4).uniform(1000)
    s = synth.Stream(123, 4)
    b = np.concatenate([s.uniform(300), s.uniform(700)])
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.Stream(123, 5).uniform(1000))
    assert a.min() > 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 4 * math.sqrt(1 / 12 / 1000)


def test_workload_shapes_and_ranges():
    (m,) = synth.mass1d(20000)
    assert m.shape == (20000,) and m.min() >= 5170.0 and m.max() <= 5970.0
    # +-3 sigma around mu holds the signal (0.3 x 0.997) plus 0.7 x 0.24 of the background
    frac = np.mean(np.abs(m - 5279.6) < 60.0)
    assert 0.44 < frac < 0.49
    cols = synth.kstar4d(20000)
    assert len(cols) == 4
    assert np.all(np.abs(cols[1]) <= 1.0) and np.all(np.abs(cols[2]) <= 1.0)
    assert np.all(np.abs(cols[3]) <= math.pi)
    w = synth.weights(10000)
    assert w.min() >= 0.5 and w.max() <= 1.5


def test_poisson_counts():
    k = synth.poisson(4000, 2000.0)
    assert abs(k.mean() - 2000.0) < 4 * math.sqrt(2000.0 / 4000)
    assert abs(k.var() / 2000.0 - 1.0) < 0.1
    off, cols = synth.toys4d(5, 200.0)
    assert off[0] == 0 and len(cols[0]) == off[-1] and np.all(np.diff(off) > 0)
