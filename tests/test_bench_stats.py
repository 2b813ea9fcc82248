"""The matched-observables comparison of the benchmark (bench.compare_arms),
on synthetic run means: Welch's statistic against its textbook form, the
family-wise false-alarm rate of the "matched" decision between two arms drawn
from the same law (about 5 %), its power against a real offset, and the
exclusion of nearly empty g(r) bins."""
import math

import numpy as np
import pytest

pytest.importorskip("scipy")

import bench


def _arm(rng, runs=8, shift=0.0, nb=80):
    r = np.arange(nb) * 0.1 + 0.05
    g0 = np.where(r < 2.4, 0.0, 1.0 + 1.5 * np.exp(-((r - 2.8) / 0.15) ** 2))
    return {"pe": rng.normal(-12.05 + shift * 0.002, 0.005, runs),
            "T": rng.normal(292.2 + shift * 0.2, 0.25, runs),
            "D": rng.normal(0.107, 0.002, runs),
            "g": g0 + rng.normal(0.0, 0.01, (runs, nb)) * (g0 > 0)}


def test_welch_against_the_textbook_form():
    rng = np.random.default_rng(1)
    a, b = rng.normal(0, 1, 8), rng.normal(0.5, 2, 11)
    t, nu, p = bench._welch(a, b)
    va, vb = a.var(ddof=1) / 8, b.var(ddof=1) / 11
    assert math.isclose(float(t), abs(a.mean() - b.mean()) / math.sqrt(va + vb), rel_tol=1e-12)
    assert math.isclose(float(nu), (va + vb) ** 2 / (va ** 2 / 7 + vb ** 2 / 10), rel_tol=1e-12)
    from scipy import stats
    assert math.isclose(float(p), stats.ttest_ind(a, b, equal_var=False).pvalue, rel_tol=1e-9)


def test_null_false_alarms_near_the_level_and_power_against_an_offset():
    rng = np.random.default_rng(7)
    n = 600
    alarms = sum(not bench.compare_arms(_arm(rng), _arm(rng))["matched"] for _ in range(n))
    # family-wise 5 % by Bonferroni over four tests: at most 5 %, a little less
    assert alarms / n < 0.08, alarms / n
    detect = sum(not bench.compare_arms(_arm(rng, shift=5.0), _arm(rng))["matched"] for _ in range(100))
    assert detect > 90


def test_empty_bins_are_left_out():
    rng = np.random.default_rng(3)
    a, b = _arm(rng), _arm(rng)
    z0 = bench.compare_arms(a, b)
    # one run with a stray pair in an empty bin (every other run and arm 0
    # there, so its standard error is tiny): the bin stays out of the test
    a["g"][0, 10] = 0.02
    z = bench.compare_arms(a, b)
    assert z["g_oo_bins"] == z0["g_oo_bins"] == int(np.sum(np.minimum(a["g"].mean(0), b["g"].mean(0)) >= 0.1))
    assert z["g_oo_bins"] < 80
    assert z["p"]["g"] == z0["p"]["g"]
