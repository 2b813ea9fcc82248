"""Pins for the oracle's random-number layer (no GPU).

* Philox4x32-10 against the published known-answer vectors.
* expneg_f32 against exp() in FP64.
* Poisson counts against scipy's Poisson quantile function, and moments.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox, poisson

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out.append((w[:4], w[4:6], w[6:10]))
    return out


def test_philox_known_answers():
    for ctr, key, want in _kat():
        got = philox.philox4x32_10(np.array(ctr, dtype=np.uint64).reshape(4, 1), key)[:, 0]
        assert [int(x) for x in got] == want


def test_philox_vectorised_equals_scalar():
    ctr = philox.counter(np.arange(5), 7, 123456789012, 2)
    many = philox.philox4x32_10(ctr, philox.seed_key(42))
    for k in range(5):
        one = philox.philox4x32_10(ctr[:, k:k + 1], philox.seed_key(42))[:, 0]
        assert np.array_equal(one, many[:, k])


def test_counter_layout():
    c = philox.counter(3, 5, (7 << 32) | 9, 2)
    assert [int(x) for x in c] == [3, 5, 9, (2 << 24) | 7]


def test_uniform_helpers():
    x = np.array([0, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    assert philox.u24(x).tolist() == [0.0, 1.0 - 2.0 ** -24, 0.5]
    assert philox.u24_open0(x).tolist() == [2.0 ** -24, 1.0, 0.5 + 2.0 ** -24]
    assert philox.u53(np.uint32(0xFFFFFFFF), np.uint32(0xFFFFFFFF)) == 1.0 - 2.0 ** -53
    assert philox.u53(np.uint32(0), np.uint32(0)) == 0.0
    # index_below is floor(x n / 2^32): exact against Python integers
    rng = np.random.default_rng(0)
    xs = rng.integers(0, 2 ** 32, 1000, dtype=np.uint64)
    ns = rng.integers(1, 100000, 1000)
    got = philox.index_below(xs, ns)
    want = [(int(a) * int(b)) >> 32 for a, b in zip(xs, ns)]
    assert got.tolist() == want


def test_index_below_is_uniform():
    x = philox.draw(1, np.arange(200000), 0, 0, 1)[0]
    idx = philox.index_below(x, 7)
    counts = np.bincount(idx, minlength=7)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_expneg_f32_accuracy():
    x = np.linspace(0, 32, 200001).astype(np.float32)
    got = poisson.expneg_f32(x).astype(np.float64)
    want = np.exp(-x.astype(np.float64))
    rel = np.abs(got - want) / want
    assert rel.max() < 1e-6
    assert got[0] == 1.0


def test_poisson_inversion_matches_quantile():
    """Away from CDF boundaries the FP32 inversion returns the Poisson
    quantile exactly."""
    rng = np.random.default_rng(1)
    for mu in (0.01, 0.7, 3.0, 9.5, 16.0):
        u = rng.random(20000).astype(np.float32)
        k = poisson.invert_chunk(u, np.full(u.shape, mu, np.float32))
        ref = stats.poisson.ppf(u.astype(np.float64), mu)
        cdf_k = stats.poisson.cdf(ref, mu)
        cdf_km1 = stats.poisson.cdf(ref - 1, mu)
        safe = (np.abs(u - cdf_k) > 1e-5) & (np.abs(u - cdf_km1) > 1e-5)
        assert np.array_equal(k[safe], ref[safe].astype(np.int64)), mu


@pytest.mark.parametrize("mu", [0.01, 1.0, 30.0, 300.0])
def test_poisson_counts_moments(mu):
    n = 200000
    M = poisson.counts(np.full(n, mu), np.arange(n), seed=3, step=11, stream=1)
    se = math.sqrt(mu / n)
    assert abs(M.mean() - mu) < 5 * se
    # variance of a Poisson variable equals its mean
    # sample-variance standard error for Poisson data: sqrt((mu + 2 mu^2) / n) / mu
    assert abs(M.var() / mu - 1.0) < 5 * math.sqrt((1.0 / mu + 2.0) / n)


def test_poisson_chunking():
    n, mu_c = poisson.chunking(np.array([0.0, 1e-9, 16.0, 16.000001, 100.0]))
    assert n.tolist() == [0, 1, 1, 2, 7]
    assert mu_c[4] == np.float32(100.0 / 7)
