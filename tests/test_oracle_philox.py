"""Pins of oracle/philox.py: published Philox-4x32-10 known answers."""
import os

import numpy as np

from oracle import philox

HERE = os.path.dirname(__file__)


def test_known_answer_vectors():
    n = 0
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        ctr = [np.array([x], dtype=np.uint64) for x in v[0:4]]
        out = philox.philox4x32_10(ctr, (np.uint64(v[4]), np.uint64(v[5])))
        assert [int(x[0]) for x in out] == v[6:10]
        n += 1
    assert n == 3


def test_uniform_range_and_normal_moments():
    u = philox.uniform53(np.array([0, 0xFFFFFFFF], dtype=np.uint64), np.array([0, 0xFFFFFFFF], dtype=np.uint64))
    assert u[0] == 2.0**-53 and u[1] == 1.0
    g = philox.white_noise(7, 1 << 21)
    assert abs(g.mean()) < 5 * (1 / np.sqrt(g.size))
    assert abs(g.var() - 1) < 5 * np.sqrt(2 / g.size)
    # counter offset gives the same stream
    np.testing.assert_array_equal(philox.white_noise(7, 10, first=100), g[100:110])
