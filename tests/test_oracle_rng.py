"""Pins for the oracle's counter-based generator and its uses.

Philox4x32-10 is checked against the published known-answer vectors; the
derived uniforms and bootstrap draws against distributional facts.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert O.philox4x32_10(ctr, key).tolist() == expect


def test_swarm_uniforms_layout_and_range():
    # Each (i, j) draw is lane j%4 of the block at counter (uid, t, i, j/4|purpose<<24).
    seed, uid, t = 0x1234_5678_9ABC, 77, 5
    u = O.swarm_uniforms(seed, uid, t, 3, 10, O.PURPOSE_R1)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(3):
        for j in range(10):
            r = O.philox4x32_10([uid, t, i, (j >> 2) | (O.PURPOSE_R1 << 24)], key)
            assert u[i, j] == np.float32((int(r[j & 3]) >> 8) / 2.0**24)
    assert u.min() >= 0.0 and u.max() < 1.0


def test_swarm_uniforms_are_uniform():
    u = O.swarm_uniforms(99, 3, 1, 1000, 1000, O.PURPOSE_R2).ravel().astype(np.float64)
    counts, _ = np.histogram(u, bins=100, range=(0.0, 1.0))
    expected = u.size / 100
    chi2 = ((counts - expected) ** 2 / expected).sum()
    # 99 degrees of freedom: P(chi2 > 160) < 1e-4
    assert chi2 < 160.0
    assert abs(u.mean() - 0.5) < 1e-3
    # streams of different purposes are not the same numbers
    v = O.swarm_uniforms(99, 3, 1, 1000, 1000, O.PURPOSE_R1).ravel()
    assert np.mean(v == u.astype(np.float32)) < 1e-3


def test_bootstrap_multiplicities():
    n = 100_000
    w = O.bootstrap(7, 3, n)
    assert int(w.sum()) == n
    distinct = np.count_nonzero(w) / n
    # P(sample drawn at least once) = 1 - (1 - 1/n)^n -> 1 - 1/e
    assert abs(distinct - (1.0 - np.exp(-1.0))) < 0.005
    # multiplicities ~ Poisson(1): P(w = 2) = e^-1 / 2
    assert abs(np.mean(w == 2) - np.exp(-1.0) / 2) < 0.005
    assert not np.array_equal(w, O.bootstrap(7, 4, n))
