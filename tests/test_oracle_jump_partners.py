"""Pins of the candidate rows restricted to the partners a jump can draw
(oracle only).

The paper draws the partner J of a jump among the particles interacting with
i (Sec. V).  When the jumps carry only the Lennard-Jones part (Coulomb wholly
in F_0, the first example of Sec. IV.A) with one bound per type, a pair of
types without LJ parameters does not interact through the jump part: for
water, hydrogens neither propose nor are drawn.  Pins: the partner table for
water and the cases that keep full rows; the rows against a brute-force
minimum-image search; the thinned jump chain over the restricted row has the
law of the exact event-driven chain and needs fewer proposals by the row
ratio; the rows follow the displacement of the moving types only.
"""
import math

import numpy as np

from oracle.bounds import bound_table, pair_weights
from oracle.forcefield import KB, Params, pair_gradient_one
from oracle.integrate import OracleMD, Topology, filter_rows, jump_half, jump_partners
from paper_2002_07109_gb300.water import water_box


def _topo(s):
    return Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)


def _water_params(s, coulomb_jumps=False):
    return Params(r_on=4.0, r_off=5.0, r_cut=6.0, ewald_beta=0.3, box=s.box, lj_sigma=s.lj_sigma,
                  lj_eps=s.lj_eps, coulomb_jumps=coulomb_jumps)


def test_water_partners_and_the_cases_with_full_rows():
    s = water_box(3, seed=1)
    p = _water_params(s)
    L, Ls = bound_table(s.charge, s.type, 2, s.lj_sigma, s.lj_eps, p)
    assert Ls[0] > 0 and Ls[1] == 0.0            # H has no LJ: no jump bound
    partner, moving = jump_partners(s.type, Ls, p)
    assert partner.tolist() == [[True, False], [False, False]]
    assert moving.tolist() == [True, False]
    # Coulomb on the jumps: every charged pair interacts through them
    pc = _water_params(s, coulomb_jumps=True)
    Lc, Lsc = bound_table(s.charge, s.type, 2, s.lj_sigma, s.lj_eps, pc)
    assert jump_partners(s.type, Lsc, pc) is None
    # per-type-pair bounds already give zero weight to those partners
    assert jump_partners(s.type, Ls, p, pair_weights(L, Ls)) is None
    # a single LJ type: nothing to leave out
    one = np.zeros(len(s.type), np.int64)
    assert jump_partners(one, Ls[:1], Params(lj_sigma=s.lj_sigma[:1, :1], lj_eps=s.lj_eps[:1, :1],
                                             coulomb_jumps=False)) is None


def test_jump_rows_against_brute_force():
    s = water_box(3, seed=2)
    p = _water_params(s)
    md = OracleMD(s.q, s.v, _topo(s), p, skin=1.0)
    rows = md.jump_rows()
    rl = p.r_cut + 1.0
    n = len(s.q)
    for i in range(n):
        if s.type[i] != 0:
            assert len(rows[i]) == 0
            continue
        want = []
        for j in range(n):
            if s.molecule[j] == s.molecule[i] or s.type[j] != 0:
                continue
            d = s.q[i] - s.q[j]
            d -= s.box * np.rint(d / s.box)
            if float(d @ d) < rl * rl:
                want.append(j)
        assert rows[i].tolist() == want, i
    # the full rows keep the H partners: the restriction drops two thirds
    md.ensure_rows()
    full = sum(len(md.row_list[i]) for i in range(n) if s.type[i] == 0)
    kept = sum(len(r) for r in rows)
    assert abs(kept / full - 1.0 / 3.0) < 0.05


def _star(n, seed):
    """Atom 0 (type 0) at the origin, n partners on a shell at 4.2-5.8 A,
    alternately of type 0 (LJ with atom 0) and type 1 (charged, no LJ)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = 4.2 + 1.6 * rng.random(n)
    q = np.concatenate([np.zeros((1, 3)), d * r[:, None]])
    typ = np.concatenate([[0], np.arange(n) % 2]).astype(np.int64)
    charge = np.where(typ == 0, -0.8, 0.4)
    m = n + 1
    topo = Topology(typ, np.full(m, 16.0), charge, np.arange(m), np.zeros((0, 2)), np.zeros((0, 2)),
                    np.zeros((0, 3)), np.zeros((0, 2)))
    sig = np.array([[3.2, 0.0], [0.0, 0.0]])
    eps = np.array([[2.0, 0.0], [0.0, 0.0]])
    p = Params(r_on=4.0, r_off=6.0, r_cut=math.inf, lj_sigma=sig, lj_eps=eps, coulomb_jumps=False)
    return q, topo, p


def test_restricted_rows_keep_the_law_of_the_jump_chain():
    q, topo, p = _star(24, seed=5)
    L, Ls = bound_table(topo.charge, topo.type, 2, p.lj_sigma, p.lj_eps, p)
    partner, moving = jump_partners(topo.type, Ls, p)
    full = [np.arange(1, len(q))] + [np.zeros(0, np.int64)] * (len(q) - 1)
    rows = filter_rows(full, topo.type, partner)
    assert rows[0].tolist() == list(range(1, len(q), 2))
    beta = 1.0 / (KB * 300.0)
    G = pair_gradient_one(np.repeat(q[:1], len(q) - 1, 0), q[1:], topo.charge[0], topo.charge[1:],
                          p.lj_sigma[0, topo.type[1:]], p.lj_eps[0, topo.type[1:]], p)
    assert np.all(G[1::2] == 0.0) and np.all(np.abs(G[0::2]).sum(1) > 0)
    v0 = np.array([0.4, -0.3, 0.2])
    nrep = 6000
    rng = np.random.default_rng(13)
    thin = np.zeros((nrep, 3))
    exact = np.zeros((nrep, 3))
    M_full = np.zeros(nrep)
    M_kept = np.zeros(nrep)
    v = np.zeros((len(q), 3))
    v[0] = v0
    for r in range(nrep):
        vr, rec = jump_half(q, v, rows, topo, p, Ls, beta, 1.0, 9, r, 1, record=True)
        thin[r] = vr[0]
        M_kept[r] = rec["M"][0]
        M_full[r] = jump_half(q, v, full, topo, p, Ls, beta, 1.0, 9, r, 1, record=True)[1]["M"][0]
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
    # second moments: standard error of a sample variance from the fourth central moment
    def var_se(x):
        c = x - x.mean(0)
        return np.sqrt(((c ** 4).mean(0) - c.var(0) ** 2) / len(x))
    assert np.all(np.abs(thin.var(0) - exact.var(0)) < 5 * np.sqrt(var_se(thin) ** 2 + var_se(exact) ** 2))
    # the Poisson mean follows the row length: half the candidates, half the proposals
    assert abs(M_kept.mean() / M_full.mean() - 0.5) < 0.05


def test_jump_rows_follow_the_moving_types():
    s = water_box(3, seed=3)
    p = _water_params(s)
    md = OracleMD(s.q, s.v, _topo(s), p, skin=1.0)
    md.jump_rows()
    assert md.rebuilds == 1
    h = int(np.nonzero(s.type == 1)[0][0])
    o = int(np.nonzero(s.type == 0)[0][0])
    md.q[h] += np.array([0.6, 0.0, 0.0])          # beyond skin/2, but H is not a moving type
    md.jump_rows()
    assert md.rebuilds == 1
    md.ensure_rows()                               # the full rows (F_0 pairs, energies) do rebuild
    assert md.rebuilds == 1
    md.q[o] += np.array([0.0, 0.6, 0.0])
    md.jump_rows()
    assert md.rebuilds == 2
