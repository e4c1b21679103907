"""Pins of the oracle's noise: Philox4x32-10, the uniform map, Box-Muller
normals and the Exp(1) thresholds of the first-passage test.

The random displacement R_i of Eq. 1 (Sec. II) has zero mean and covariance
2 D dt; each replica gets a unique random-number seed (Sec. II, RSF). Both are
realised with a counter-based Philox stream; these tests tie the oracle's
stream to the published generator and to the normal / exponential laws.
"""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    out = O.philox(ctr, key)
    assert [int(x) for x in out] == expect


def test_philox_batch_matches_single():
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = [0x12345678, 0x9abcdef0]
    many = O.philox_many(ctr, key)
    for j in range(0, 64, 7):
        assert np.array_equal(many[j], O.philox(ctr[j], key))


def test_uniform_open_interval_endpoints():
    assert O.uniform(0) == 2.0**-33
    assert O.uniform(0xFFFFFFFF) == 1.0 - 2.0**-33
    assert O.uniform(0x80000000) == 0.5 + 2.0**-33


def _counters(n, slot=3, stream=0, step=11, chain=5):
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n) % 997
    ctr[:, 1] = slot | (stream << 24)
    ctr[:, 2] = step + np.arange(n) // 997
    ctr[:, 3] = chain
    return ctr


def test_normals_are_standard_normal():
    xi = O.normals3_many(42, _counters(120_000))
    n = xi.shape[0]
    for d in range(3):
        z = xi[:, d]
        assert abs(z.mean()) < 5.0 / np.sqrt(n)
        assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
        assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5.0 * np.sqrt(24.0 / n)
        assert stats.kstest(z, "norm").pvalue > 1e-4
    c = np.corrcoef(xi.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5.0 / np.sqrt(n))


def test_normals_depend_on_every_counter_word():
    base = O.normals3(7, 1, 2, 0, 3, 4)
    for args in [(8, 1, 2, 0, 3, 4), (7, 2, 2, 0, 3, 4), (7, 1, 3, 0, 3, 4),
                 (7, 1, 2, 1, 3, 4), (7, 1, 2, 0, 4, 4), (7, 1, 2, 0, 3, 5)]:
        assert not np.allclose(O.normals3(*args), base)
    assert np.array_equal(O.normals3(7, 1, 2, 0, 3, 4), base)


def test_normals3_uses_the_philox_words_of_its_counter():
    # The stream is a function of the Philox output alone: two counters that
    # share the output words would share normals. Check that the slot and the
    # stream id occupy disjoint bit fields of counter word 1.
    a = O.normals3(9, 0, 5, 1, 0, 0)
    b = O.normals3(9, 0, 5 | (1 << 24), 0, 0, 0)
    assert np.array_equal(a, b)


def test_exp1_thresholds_are_unit_exponential():
    e = np.array([O.exp1(11, i, q, c) for c in range(40) for q in range(3) for i in range(100)])
    n = len(e)
    assert abs(e.mean() - 1.0) < 5.0 / np.sqrt(n)
    assert stats.kstest(e, "expon").pvalue > 1e-4
