"""Pins of the oracle's Philox4x32-10 against published known answers and basic statistics."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_known_answers():
    n = 0
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert philox.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])
        n += 1
    assert n == 3


def test_uniform_range_and_moments():
    u = np.array([philox.uniform(12345, philox.PURPOSE_SITE, i, 3, 1, 7, 9) for i in range(4000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / len(u))
    hist, _ = np.histogram(u, bins=10, range=(0, 1))
    chi2 = ((hist - 400) ** 2 / 400).sum()
    assert chi2 < 30  # 9 dof, p ~ 4e-4


def test_counter_words_are_independent_streams():
    base = philox.uniform(1, 0, 0, 0, 0, 0, 0)
    variants = [philox.uniform(1, 1, 0, 0, 0, 0, 0), philox.uniform(1, 0, 1, 0, 0, 0, 0),
                philox.uniform(1, 0, 0, 1, 0, 0, 0), philox.uniform(1, 0, 0, 0, 1, 0, 0),
                philox.uniform(1, 0, 0, 0, 0, 1, 0), philox.uniform(1, 0, 0, 0, 0, 0, 1),
                philox.uniform(2, 0, 0, 0, 0, 0, 0), philox.uniform(1 << 32, 0, 0, 0, 0, 0, 0)]
    assert len(set(variants + [base])) == 9
