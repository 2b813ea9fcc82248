"""Pins of the per-type-pair bounds with two-stage partner choice (oracle only).

The paper notes that the bound L may depend on the types of the two particles
(Sec. V).  With a bound per type pair, the proposals of atom i form the
superposition of one Poisson process per candidate j with rate
beta ||v_i|| Lt_{t_i t_j}; a proposal therefore picks candidate j with
probability Lt_{t_i t_j} / sum_k Lt_{t_i t_k}, and is accepted with probability
max(0, v.F) / (||v|| Lt).  Pins: the weights bound the table; the integer
choice hits every candidate exactly Lq times (enumeration); the thinned jump
chain has the law of the exact chain (independent event-driven simulation);
proposals drop by the predicted factor.
"""
import math

import numpy as np

from oracle.bounds import bound_table, pair_weights
from oracle.forcefield import KB, Params, pair_gradient_one
from oracle.integrate import Topology, jump_half, two_stage_pick, typed_rows


def test_pair_weights_bound_the_table():
    rng = np.random.default_rng(3)
    L = rng.random((3, 3)) * 5.0
    L[1, 2] = 0.0
    Ls = L.max(1)
    Lq, Lt = pair_weights(L, Ls)
    assert Lq.dtype == np.int64 and Lq.max() <= 65537
    assert Lq[1, 2] == 0 and Lt[1, 2] == 0.0
    nz = L > 0
    assert np.all(Lt[nz] >= L[nz])
    assert np.all(Lt[nz] <= L[nz] + 2.0 * Ls[np.nonzero(nz)[0]] * 2.0 ** -16)


def test_two_stage_pick_hits_every_candidate_lq_times():
    counts = np.array([[3, 0, 5, 2]])
    Lq_a = np.array([[7, 4, 3, 11]])
    wq = counts * Lq_a
    C = np.concatenate([[[0]], np.cumsum(wq, 1)], 1)
    S = np.concatenate([[[0]], np.cumsum(counts, 1)], 1)
    W = int(C[0, -1])
    t = np.arange(W)
    J = two_stage_pick(t, np.repeat(C, W, 0), np.repeat(S, W, 0), np.repeat(Lq_a, W, 0))
    hits = np.bincount(J, minlength=counts.sum())
    expect = np.repeat(Lq_a[0], counts[0])
    assert np.array_equal(hits, expect)


def test_typed_rows_regroup_by_type():
    typ = np.array([0, 1, 1, 0, 1, 0, 0])
    rows = [np.array([1, 2, 3, 5, 6]), np.array([0, 4])]
    out, counts = typed_rows(rows, typ, 2)
    assert np.array_equal(out[0], [3, 5, 6, 1, 2]) and np.array_equal(counts[0], [3, 2])
    assert np.array_equal(out[1], [0, 4]) and np.array_equal(counts[1], [1, 1])


def _star2(n, seed):
    """Atom 0 at the origin, n partners of two types (charges +0.8 and -0.3)
    on a shell at 5-9 A: two very different type-pair bounds."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = 5.0 + 4.0 * rng.random(n)
    q = np.concatenate([np.zeros((1, 3)), d * r[:, None]])
    typ = np.concatenate([[0], np.arange(n) % 2]).astype(np.int64)
    charge = np.where(typ == 0, 0.8, -0.3)
    charge[0] = 0.5
    m = n + 1
    topo = Topology(typ, np.full(m, 16.0), charge, np.arange(m), np.zeros((0, 2)), np.zeros((0, 2)),
                    np.zeros((0, 3)), np.zeros((0, 2)))
    p = Params(r_on=4.0, r_off=6.0, r_cut=math.inf, lj_sigma=np.zeros((2, 2)), lj_eps=np.zeros((2, 2)))
    rows = [np.arange(1, m)] + [np.zeros(0, np.int64)] * n
    return q, topo, p, rows


def test_typed_thinning_matches_exact_jump_chain():
    q, topo, p, rows = _star2(24, seed=7)
    L, Ls = bound_table(topo.charge, topo.type, 2, p.lj_sigma, p.lj_eps, p)
    assert L[0, 1] < 0.5 * L[0, 0]
    pb = pair_weights(L, Ls)
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
        thin[r] = jump_half(q, v, rows, topo, p, Ls, beta, 1.0, 5, r, 1, pair_bounds=pb)[0][0]
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


def test_typed_proposals_follow_the_weighted_mean():
    q, topo, p, rows = _star2(24, seed=7)
    L, Ls = bound_table(topo.charge, topo.type, 2, p.lj_sigma, p.lj_eps, p)
    pb = pair_weights(L, Ls)
    beta = 1.0 / (KB * 300.0)
    v = np.zeros((len(q), 3))
    v[0] = [0.05, -0.02, 0.03]
    M_plain = np.array([jump_half(q, v, rows, topo, p, Ls, beta, 1.0, 5, r, 1, record=True)[1]["M"][0]
                        for r in range(3000)])
    M_typed = np.array([jump_half(q, v, rows, topo, p, Ls, beta, 1.0, 5, r, 1, record=True, pair_bounds=pb)[1]["M"][0]
                        for r in range(3000)])
    n0 = 12
    ratio = (n0 * pb[1][0, 0] + n0 * pb[1][0, 1]) / (24 * Ls[0])
    assert abs(M_typed.mean() / M_plain.mean() - ratio) < 0.05
    assert ratio < 0.8
