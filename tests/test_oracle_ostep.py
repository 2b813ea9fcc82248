"""Pins for the oracle's O step (paper Sec. III.C: the Ornstein-Uhlenbeck
part of the Langevin splitting, v <- c1 v + sqrt((1 - c1^2) k_B T / m) G).

What the mathematics fixes, independently of how o_step writes it:
  * the OU process leaves the Maxwell-Boltzmann law invariant: per component
    Var(v) = k_B T / m (in A^2/fs^2: k_B T * 4.184e-4 / m), whatever the
    friction and time step -- a wrong noise amplitude (a dropped unit factor,
    a sqrt(2) too many, 1 - c1 instead of 1 - c1^2) moves it;
  * the lag-1 autocorrelation of the stationary chain is c1 = exp(-gamma
    delta) -- a wrong friction factor (exp(-gamma delta / 2), the mass in the
    exponent) moves it;
  * the Box-Muller normals are standard: mean 0, variance 1, skewness 0,
    kurtosis 3, with the three components uncorrelated -- a wrong angle
    (sin instead of cos for the third component reuses one), a log without
    the factor -2, or a uniform that reaches 0 would show.
"""
import math

import numpy as np

from oracle.forcefield import ACCEL, KB
from oracle.integrate import o_step

T = 300.0


def test_normals_are_standard():
    n, steps = 20000, 10
    mass = np.full(n, 2.0)
    g = []
    for k in range(steps):
        # from v = 0 one O step returns sd * G: G recovered with the expected sd of the law
        out = o_step(np.zeros((n, 3)), mass, T, gamma=0.1, dt=1.0, seed=3, step=k)
        c1 = math.exp(-0.1)
        g.append(out / math.sqrt((1.0 - c1 * c1) * KB * T * ACCEL / 2.0))
    g = np.concatenate(g).reshape(-1, 3)
    N = len(g)
    for c in range(3):
        x = g[:, c]
        m, v = x.mean(), x.var()
        sk = ((x - m) ** 3).mean() / v ** 1.5
        ku = ((x - m) ** 4).mean() / v ** 2
        assert abs(m) < 5 / math.sqrt(N), (c, m)
        assert abs(v - 1.0) < 5 * math.sqrt(2.0 / N), (c, v)
        assert abs(sk) < 5 * math.sqrt(6.0 / N), (c, sk)
        assert abs(ku - 3.0) < 5 * math.sqrt(24.0 / N), (c, ku)
    cc = np.corrcoef(g.T)
    assert np.all(np.abs(cc[np.triu_indices(3, 1)]) < 5 / math.sqrt(N)), cc


def test_stationary_variance_and_autocorrelation():
    """Many independent atoms of two masses, started at rest, relaxed for
    ten friction times, then sampled: Var = k_B T ACCEL / m per component
    and corr(v_t, v_{t+1}) = exp(-gamma delta)."""
    n = 6000
    mass = np.where(np.arange(n) % 2 == 0, 15.9994, 1.008)
    gamma, dt = 0.05, 1.0
    c1 = math.exp(-gamma * dt)
    v = np.zeros((n, 3))
    burn = int(10 / (gamma * dt))
    for k in range(burn):
        v = o_step(v, mass, T, gamma, dt, seed=11, step=k)
    xs = []
    for k in range(burn, burn + 800):
        v = o_step(v, mass, T, gamma, dt, seed=11, step=k)
        xs.append(v.copy())
    xs = np.array(xs)                               # (steps, n, 3)
    for par, m in ((0, 15.9994), (1, 1.008)):
        sel = xs[:, par::2, :] / math.sqrt(KB * T * ACCEL / m)   # unit variance if the law is right
        var = (sel ** 2).mean()
        # samples of one atom are correlated over ~(1 + c1)/(1 - c1) steps
        n_eff = sel.size * (1 - c1) / (1 + c1)
        assert abs(var - 1.0) < 5 * math.sqrt(2.0 / n_eff), (m, var)
        lag1 = (sel[1:] * sel[:-1]).mean() / var
        assert abs(lag1 - c1) < 5 / math.sqrt(n_eff), (m, lag1, c1)
    # a different friction gives a different lag-1 correlation (the test has power)
    assert abs(math.exp(-0.5 * gamma * dt) - c1) > 8 / math.sqrt(n_eff)
