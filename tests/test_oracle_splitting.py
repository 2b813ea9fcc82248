"""Pins for the oracle's whole BOUNCE step against what the stationary law
and the splitting order fix (paper Sec. III.C-D, Sec. IV.B).

* Three-atom marginal: a bent chain 1-2-3 whose two bonds and angle sit in
  F_0 while the 1-3 pair (a Coulomb-like repulsion) is entirely on the jumps.
  The invariant law is exp(-beta E) in configuration space, so the
  distribution of r_13 is the 3-D quadrature over (r_12, r_23, theta) of
  r_12^2 r_23^2 sin(theta) exp(-beta (U_b + U_b + U_a + W(r_13))).  Its mean
  and its histogram are compared with the oracle's samples; without the jump
  part the mean moves by many standard errors, so a dropped or mis-signed
  jump term (or one applied to the wrong atom) fails.
* Splitting order: BJAOAJB is a symmetric (Strang) splitting, so its
  stationary bias shrinks at least like delta^2.  A two-atom system with a
  bond in F_0 and its own repulsion on the jumps is run at delta = 1, 0.5 and
  0.25 fs: the bias of the mean bond energy (against quadrature) at 0.5 fs is
  at most a third of the bias at 1 fs (a first-order scheme gives a half),
  and at 0.25 fs smaller again.  This is the mechanism behind the heating of
  flexible water with short switching distances: a reflection between B and
  A shifts the bond's shadow energy by O(delta) per event, so the stationary
  excess energy grows like delta^2 (and faster once it feeds back).
"""
import math

import numpy as np
import pytest

from oracle.forcefield import ACCEL, KB, Params
from oracle.integrate import OracleMD, Topology

BETA = 1.0 / (KB * 300.0)
K_COUL = 332.063713


def _replicated(R, per, mass, charge, bonds, bond_k_r0, angles=None, angle_k_t0=None):
    """R copies of a small system 1000 A apart (no pair crosses copies)."""
    a = len(mass)
    q = np.concatenate([per + np.array([1000.0 * r, 0.0, 0.0]) for r in range(R)])
    n = a * R
    off = np.repeat(np.arange(R) * a, len(bonds))[:, None]
    b = np.tile(bonds, (R, 1)) + off
    if angles is not None:
        an = np.tile(angles, (R, 1)) + np.repeat(np.arange(R) * a, len(angles))[:, None]
        ak = np.tile(angle_k_t0, (R, 1))
    else:
        an, ak = np.zeros((0, 3)), np.zeros((0, 2))
    topo = Topology(np.zeros(n, int), np.tile(mass, R), np.tile(charge, R), np.arange(n), b,
                    np.tile(bond_k_r0, (R, 1)), an, ak)
    return q, topo


@pytest.mark.slow
def test_three_atom_r13_marginal():
    R, kb, r0, ka, th0, kq, m = 300, 20.0, 1.5, 10.0, math.radians(100.0), 0.5, 10.0
    per = np.array([[r0 * math.sin(th0 / 2), r0 * math.cos(th0 / 2), 0.0], [0.0, 0.0, 0.0],
                    [-r0 * math.sin(th0 / 2), r0 * math.cos(th0 / 2), 0.0]])
    q, topo = _replicated(R, per, np.full(3, m), np.array([math.sqrt(kq), 0.0, math.sqrt(kq)]),
                          np.array([[0, 1], [1, 2]]), np.array([[kb, r0], [kb, r0]]),
                          np.array([[0, 1, 2]]), np.array([[ka, th0]]))
    z = np.zeros((1, 1))
    p = Params(r_on=1.0, r_off=1.0, r_cut=30.0, lj_sigma=z, lj_eps=z)   # the whole 1-3 pair on the jumps
    rng = np.random.default_rng(1)
    v = rng.standard_normal(q.shape) * math.sqrt(KB * 300.0 * ACCEL / m)
    md = OracleMD(q, v, topo, p, seed=8, gamma=0.02, dt=1.0, skin=20.0)
    samples = []
    for k in range(3300):
        md.step_bounce()
        if k >= 300 and k % 10 == 0:
            samples.append(np.linalg.norm(md.q[0::3] - md.q[2::3], axis=1))
    s = np.array(samples)                               # (time, replica)
    assert md.accepts > 1000                            # the jumps act
    # quadrature over (r12, r23, theta)
    r = np.linspace(0.75, 2.25, 121)
    th = np.linspace(1e-4, math.pi - 1e-4, 181)
    R1, R2, TH = np.meshgrid(r, r, th, indexing="ij")
    r13 = np.sqrt(R1 * R1 + R2 * R2 - 2.0 * R1 * R2 * np.cos(TH))
    E0 = kb * (R1 - r0) ** 2 + kb * (R2 - r0) ** 2 + ka * (TH - th0) ** 2
    jac = R1 * R1 * R2 * R2 * np.sin(TH)
    w_full = jac * np.exp(-BETA * (E0 + K_COUL * kq / r13 - (E0 + K_COUL * kq / r13).min()))
    w_bond = jac * np.exp(-BETA * (E0 - E0.min()))
    mean_full = (r13 * w_full).sum() / w_full.sum()
    mean_bond = (r13 * w_bond).sum() / w_bond.sum()
    blocks = s.mean(1)[: len(s) // 20 * 20].reshape(20, -1).mean(1)
    se = blocks.std(ddof=1) / math.sqrt(20)
    assert abs(mean_full - mean_bond) > 10 * se         # the jump part matters at this precision
    assert abs(s.mean() - mean_full) < 4 * se, (s.mean(), mean_full, se)
    # histogram of r13 against the quadrature (chi^2 per bin with per-bin block errors)
    edges = np.linspace(1.4, 3.4, 11)
    h_ref = np.histogram(r13.ravel(), edges, weights=w_full.ravel())[0] / w_full.sum()
    hb = np.array([np.histogram(x.ravel(), edges)[0] / x.size
                   for x in np.array_split(s[: len(s) // 20 * 20], 20)])
    m_h, se_h = hb.mean(0), hb.std(0, ddof=1) / math.sqrt(20)
    ok = h_ref > 0.01
    chi2 = (((m_h[ok] - h_ref[ok]) / se_h[ok]) ** 2).mean()
    assert chi2 < 4.0, (chi2, m_h, h_ref)


def _bond_bias(dt, R=400, t_fs=1200.0, burn_fs=300.0):
    """Relative bias of <k (r - r0)^2> of a bonded pair (bond in F_0, its
    Coulomb-like repulsion beyond 2 A on the jumps) at time step dt, and its
    block standard error."""
    kb, r0, kq, m = 50.0, 3.0, 0.25, 2.0
    per = np.array([[0.0, 0.0, 0.0], [r0, 0.0, 0.0]])
    q, topo = _replicated(R, per, np.full(2, m), np.full(2, math.sqrt(kq)), np.array([[0, 1]]),
                          np.array([[kb, r0]]))
    z = np.zeros((1, 1))
    p = Params(r_on=2.0, r_off=2.0, r_cut=20.0, lj_sigma=z, lj_eps=z)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(q.shape) * math.sqrt(KB * 300.0 * ACCEL / m)
    md = OracleMD(q, v, topo, p, seed=4, gamma=0.02, dt=dt, skin=10.0)
    burn, steps, every = int(burn_fs / dt), int(t_fs / dt), max(1, int(4 / dt))
    eb = []
    for k in range(burn + steps):
        md.step_bounce()
        if k >= burn and k % every == 0:
            d = np.linalg.norm(md.q[0::2] - md.q[1::2], axis=1)
            eb.append((kb * (d - r0) ** 2).mean())
    eb = np.array(eb)
    x = np.linspace(1.5, 4.5, 300001)
    U = kb * (x - r0) ** 2 + K_COUL * kq / x
    w = x * x * np.exp(-BETA * (U - U.min()))
    ref = (kb * (x - r0) ** 2 * w).sum() / w.sum()
    blocks = eb[: len(eb) // 10 * 10].reshape(10, -1).mean(1)
    return eb.mean() / ref - 1.0, blocks.std(ddof=1) / math.sqrt(10) / ref


@pytest.mark.slow
def test_splitting_bias_is_second_order():
    b1, e1 = _bond_bias(1.0)
    b2, e2 = _bond_bias(0.5)
    b4, e4 = _bond_bias(0.25)
    assert b1 > 8 * e1, (b1, e1)                        # a measurable bias at 1 fs
    assert b2 > 0 and b2 < b1 / 3.0 + 3 * e2, (b1, b2, e2)   # first order would leave b1 / 2
    assert b4 < b2 / 2.0 + 3 * e4, (b2, b4, e4)
