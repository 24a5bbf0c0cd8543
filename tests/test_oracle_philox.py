"""Pins of the oracle's Philox4x32-10 against the published known-answer
vectors (tests/golden/philox_kat.txt) and of its Box-Muller normals."""
import os

import numpy as np

from oracle import philox

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def test_known_answers():
    n = 0
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = philox.philox4x32_10(np.array([v[:4]], dtype=np.uint32), (v[4], v[5]))[0]
        assert [int(x) for x in out] == v[6:10]
        n += 1
    assert n >= 2


def test_normals_moments_and_streams():
    z = philox.normals(400000, seed=123, step=7, sid=1)
    assert abs(z.mean()) < 5e-3 and abs(z.var() - 1) < 1e-2
    assert abs(np.mean(z**4) - 3) < 5e-2
    z2 = philox.normals(400000, seed=123, step=7, sid=2)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 5e-3
    np.testing.assert_array_equal(philox.normals(10, 123, 7, 1), z[:10])
