"""Pins for the oracle's integrators (no GPU).

* R_ij preserves ||v_i|| and flips v_i . F_ij (Sec. II.B).
* The thinned jump step J (Sec. III.D + IV.B) has the same law as the exact
  jump chain simulated event by event with competing exponential clocks
  (Sec. III.D first construction), for many partners at fixed q.
* chi == 0 (no long-range part): BOUNCE is bitwise BAOAB.
* Mean kick: for Maxwellian v, E[J(t) v - v] = -t M^-1 F_long + O(t^2).
* Boltzmann marginal: a 2-atom system (bond on F_0, long-range pair on
  jumps) samples r with density r^2 exp(-beta (U_bond + W)).
"""
import math

import numpy as np
import pytest

from oracle import philox
from oracle.bounds import bound_table
from oracle.forcefield import ACCEL, KB, Params, pair_gradient_one
from oracle.integrate import OracleMD, Topology, jump_half
from paper_2002_07109_gb300.water import water_droplet


def _topo(s):
    return Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)


def _star(npart, seed):
    """Atom 0 at the origin with npart partners (alternating charges) at
    4.5 - 9 A in random directions."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((npart, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    q = np.vstack([[0.0, 0.0, 0.0], d * rng.uniform(4.5, 9.0, npart)[:, None]])
    n = npart + 1
    ch = np.ones(n)
    ch[1::2] = -1.0
    topo = Topology(np.zeros(n, int), np.ones(n), ch, np.arange(n), np.zeros((0, 2)), np.zeros((0, 2)),
                    np.zeros((0, 3)), np.zeros((0, 2)))
    z = np.zeros((1, 1))
    p = Params(r_on=4.0, r_off=5.0, r_cut=50.0, lj_sigma=z, lj_eps=z)
    rows = [np.arange(1, n)] + [np.array([0])] * npart
    return q, topo, p, rows


def test_reflection_invariants():
    s = water_droplet(3, seed=1)
    topo = _topo(s)
    p = Params(r_on=4.0, r_off=5.0, r_cut=math.inf, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    md = OracleMD(s.q, s.v, topo, p, seed=3)
    md.ensure_rows()
    v2, rec = jump_half(md.q, s.v, md.row_list, topo, p, md.Lstar, md.beta, 1.0, 3, 0, 1, record=True)
    n1 = np.linalg.norm(s.v, axis=1)
    n2 = np.linalg.norm(v2, axis=1)
    assert np.max(np.abs(n1 - n2) / n1) < 1e-14
    assert rec['accepted'].sum() > 10
    # every accepted proposal satisfied U < ratio <= 1; every rejection U >= ratio
    assert np.all(rec['ratio'] <= 1.0)
    acc = rec['accepted'].astype(bool)
    assert np.all(rec['U'][acc] < rec['ratio'][acc])
    assert np.all(rec['U'][~acc] >= rec['ratio'][~acc])
    # one reflection: v' . F = -v . F, |v'| = |v|
    rng = np.random.default_rng(0)
    v = rng.normal(size=3)
    F = rng.normal(size=3)
    a = v @ F
    w = v - (a + a) / (F @ F) * F
    assert abs(w @ F + a) < 1e-14 and abs(np.linalg.norm(w) - np.linalg.norm(v)) < 1e-14


def test_thinning_matches_exact_jump_chain():
    q, topo, p, rows = _star(24, seed=7)
    L, Ls = bound_table(topo.charge, topo.type, 1, p.lj_sigma, p.lj_eps, p)
    beta = 1.0 / (KB * 300.0)
    G = pair_gradient_one(np.repeat(q[:1], len(q) - 1, 0), q[1:], topo.charge[0], topo.charge[1:], 0.0, 0.0, p)
    v0 = np.array([0.05, -0.02, 0.03])
    nrep = 6000
    rng = np.random.default_rng(11)
    thin = np.zeros((nrep, 3))
    exact = np.zeros((nrep, 3))
    v = np.zeros((len(q), 3))
    v[0] = v0
    for r in range(nrep):
        thin[r] = jump_half(q, v, rows, topo, p, Ls, beta, 1.0, 5, r, 1)[0][0]
        w = v0.copy()
        t = 0.0
        while True:
            rates = beta * np.maximum(0.0, G @ w)
            tot = rates.sum()
            if tot <= 0:
                break
            t += rng.exponential(1.0 / tot)
            if t > 0.5:
                break
            g = G[rng.choice(len(G), p=rates / tot)]
            w = w - 2.0 * (w @ g) / (g @ g) * g
        exact[r] = w
    se = np.sqrt(thin.var(0) / nrep + exact.var(0) / nrep)
    assert np.all(np.abs(thin.mean(0) - exact.mean(0)) < 5 * se)
    p_thin = np.mean(np.all(thin == v0, axis=1))
    p_exact = np.mean(np.all(exact == v0, axis=1))
    assert 0.05 < p_exact < 0.95
    assert abs(p_thin - p_exact) < 5 * math.sqrt(p_exact * (1 - p_exact) * 2 / nrep)
    assert np.allclose(thin.var(0), exact.var(0), rtol=0.1)


def test_bounce_without_long_range_is_bitwise_baoab():
    s = water_droplet(3, seed=5)
    topo = _topo(s)
    inf = math.inf
    p = Params(r_on=inf, r_off=inf, r_cut=inf, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    a = OracleMD(s.q, s.v, topo, p, seed=9)
    b = OracleMD(s.q, s.v, topo, p, seed=9)
    a.run(5, "baoab")
    b.run(5, "bounce")
    assert b.proposals == 0
    assert np.array_equal(a.q, b.q) and np.array_equal(a.v, b.v)


def test_mean_kick_first_order():
    """E[dv] over J(t) equals -t ACCEL F/m to first order in t (Maxwellian v)."""
    q, topo, p, rows = _star(8, seed=3)
    L, Ls = bound_table(topo.charge, topo.type, 1, p.lj_sigma, p.lj_eps, p)
    beta = 1.0 / (KB * 300.0)
    G = pair_gradient_one(np.repeat(q[:1], len(q) - 1, 0), q[1:], topo.charge[0], topo.charge[1:], 0.0, 0.0, p).sum(0)
    rng = np.random.default_rng(2)
    dt = 0.05                                   # half step 0.025 fs: saturation below 1 %
    nrep = 400000
    nb = 20000
    sd = math.sqrt(ACCEL / beta)                # unit masses
    V = rng.standard_normal((nrep, 3)) * sd
    dv = np.zeros((nrep, 3))
    n = len(q)
    qq = np.tile(q, (nb, 1)) + np.repeat(np.arange(nb) * 1000.0, n)[:, None] * np.array([1, 0, 0])
    rr = []
    for b in range(nb):
        base = b * n
        rr.append(base + rows[0])
        rr.extend([np.array([base])] * (n - 1))
    tp = Topology(np.zeros(len(qq), int), np.ones(len(qq)), np.tile(topo.charge, nb),
                  np.arange(len(qq)), np.zeros((0, 2)), np.zeros((0, 2)), np.zeros((0, 3)), np.zeros((0, 2)))
    for r0 in range(0, nrep, nb):
        vv = np.zeros((nb * n, 3))
        vv[0::n] = V[r0:r0 + nb]
        out, _ = jump_half(qq, vv, rr, tp, p, Ls, beta, dt, 17, r0, 1)
        dv[r0:r0 + nb] = out[0::n] - vv[0::n]
    mean = dv.mean(0)
    se = dv.std(0) / math.sqrt(nrep)
    want = -0.5 * dt * ACCEL * G
    assert se.max() < 0.15 * np.abs(want).max()        # the test has power
    assert np.all(np.abs(mean - want) < 5 * se + 0.02 * np.abs(want).max()), (mean, want, se)


@pytest.mark.slow
def test_two_atom_boltzmann_marginal():
    """Bond in F_0, Coulomb-like repulsion entirely on jumps: the sampled mean
    r matches r^2 exp(-beta(U_b + W)) by quadrature (with the jump sign
    flipped it would sample exp(+beta W) and fail), and the velocity
    marginal is Maxwellian (unit variance and kurtosis 3 per component)."""
    nrep = 96
    kq, r0, kb = 0.25, 3.0, 2.0
    q = np.zeros((2 * nrep, 3))
    q[1::2, 0] = r0
    q += np.repeat(np.arange(nrep) * 1000.0, 2)[:, None] * np.array([1, 0, 0])
    mass = np.full(2 * nrep, 10.0)
    ch = np.full(2 * nrep, math.sqrt(kq))
    bonds = np.stack([np.arange(0, 2 * nrep, 2), np.arange(1, 2 * nrep, 2)], 1)
    topo = Topology(np.zeros(2 * nrep, int), mass, ch, np.arange(2 * nrep), bonds, np.tile([kb, r0], (nrep, 1)),
                    np.zeros((0, 3)), np.zeros((0, 2)))
    z = np.zeros((1, 1))
    p = Params(r_on=0.8, r_off=1.2, r_cut=20.0, lj_sigma=z, lj_eps=z)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(q.shape) * math.sqrt(KB * 300 * ACCEL / 10.0)
    md = OracleMD(q, v, topo, p, seed=4, gamma=0.01, dt=1.0, skin=10.0)
    rs, vs = [], []
    for k in range(2500):
        md.step_bounce()
        if k >= 300 and k % 5 == 0:
            d = md.q[0::2] - md.q[1::2]
            rs.append(np.linalg.norm(d, axis=1))
            vs.append(md.v / math.sqrt(KB * 300 * ACCEL / 10.0))
    rs = np.array(rs)
    # the velocity marginal stays Maxwellian (each reflection keeps |v|; a
    # biased thinning or a reflection that changed |v| would heat or cool):
    # unit variance and kurtosis 3 per component, errors from 20 blocks
    z = np.array(vs)
    zb = z[: len(z) // 20 * 20].reshape(20, -1)
    var_b = (zb ** 2).mean(1)
    kurt_b = (zb ** 4).mean(1) / var_b ** 2
    for stat, ref in ((var_b, 1.0), (kurt_b, 3.0)):
        se_s = stat.std(ddof=1) / math.sqrt(len(stat))
        assert abs(stat.mean() - ref) < max(4 * se_s, 0.01 * ref), (stat.mean(), ref, se_s)
    beta = 1.0 / (KB * 300.0)
    x = np.linspace(0.9, 8.0, 400001)
    U = kb * (x - r0) ** 2 + 332.063713 * kq / x
    w = x * x * np.exp(-beta * (U - U.min()))
    mean_ref = (x * w).sum() / w.sum()
    Ub = kb * (x - r0) ** 2
    wb = x * x * np.exp(-beta * (Ub - Ub.min()))
    mean_bond_only = (x * wb).sum() / wb.sum()
    assert mean_ref - mean_bond_only > 0.1          # the jump part matters
    m = rs.mean(1)                                   # per-sample mean over replicas
    blocks = m[: len(m) // 20 * 20].reshape(20, -1).mean(1)
    se = blocks.std(ddof=1) / math.sqrt(20)
    assert abs(rs.mean() - mean_ref) < max(4 * se, 0.01), (rs.mean(), mean_ref, se)
