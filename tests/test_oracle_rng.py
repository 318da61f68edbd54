"""Pins of the oracle's pair noise (Eq. 7): Philox4x32-10 and the Gaussian transform.

Eq. 7 asks for xi_ij Gaussian, zero mean, unit variance, independent between pairs
and between time steps, and symmetric (xi_ij = xi_ji).  The generator is pinned to
the published known-answer vectors; the transform to the normal law by moments and
a Kolmogorov-Smirnov test; independence by correlations.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox(ctr, key)) == expect


def test_u01_open_interval_and_exact_ends():
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # every value is an odd multiple of 2^-24, exactly representable in binary32
    for x in [1, 511, 512, 123456789, 0x80000000]:
        u = oracle.u01(x)
        assert 0.0 < u < 1.0
        assert np.float32(u) == u


def test_xi_symmetric_in_pair():
    for a, b in [(0, 1), (5, 1000), (77, 76), (123456, 7)]:
        for step in (0, 1, 99):
            assert oracle.xi(a, b, step, 0, 42) == oracle.xi(b, a, step, 0, 42)


def _samples(n, step=0, seed=7, sys=0):
    rng = np.random.default_rng(1)
    ids = rng.integers(0, 1 << 30, size=(n, 2))
    return np.array([oracle.xi(int(a), int(b), step, sys, seed) for a, b in ids]), ids


def test_xi_is_standard_normal():
    from scipy import stats

    x, _ = _samples(100_000)
    n = len(x)
    assert abs(x.mean()) < 5.0 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(stats.skew(x)) < 5.0 * math.sqrt(6.0 / n)
    assert abs(stats.kurtosis(x)) < 5.0 * math.sqrt(24.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-4


def test_xi_independent_between_steps_pairs_and_seeds():
    n = 20_000
    rng = np.random.default_rng(3)
    ids = rng.integers(0, 1 << 20, size=(n, 2))
    a = np.array([oracle.xi(int(i), int(j), 10, 0, 1) for i, j in ids])
    b = np.array([oracle.xi(int(i), int(j), 11, 0, 1) for i, j in ids])      # next step
    c = np.array([oracle.xi(int(i), int(j) + 1, 10, 0, 1) for i, j in ids])  # other pair
    d = np.array([oracle.xi(int(i), int(j), 10, 0, 2) for i, j in ids])      # other seed
    e = np.array([oracle.xi(int(i), int(j), 10, 1, 1) for i, j in ids])      # other system
    lim = 5.0 / math.sqrt(n)
    for other in (b, c, d, e):
        assert abs(np.corrcoef(a, other)[0, 1]) < lim
