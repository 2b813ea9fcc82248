"""GPU parity of the variant in which only the Lennard-Jones part is split by
chi and carried by the jumps, while the whole Coulomb interaction stays in the
short-range force F_0 (the first example of Sec. IV.A).  The CUDA library with
jump_coulomb = 0 against the oracle with coulomb_jumps = False on the same
seeded inputs: per-type bounds, the three gradient parts, one jump half-step
and one BOUNCE step.  Tolerances and tie handling follow test_gpu_parity.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.forcefield import ACCEL, Params
from oracle.integrate import OracleMD, Topology, jump_half
from paper_2002_07109_gb300.water import water_box, water_droplet_molecules

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

TOL = 1e-5

CASES = {
    # a 1000-molecule droplet gives over a hundred LJ proposals per half-step
    "droplet": (lambda: water_droplet_molecules(1000, seed=5), dict(r_on=4.0, r_off=5.0, r_cut=12.0, skin=1.0)),
    "box_ewald": (lambda: water_box(8, seed=6), dict(r_on=4.0, r_off=5.0, r_cut=9.0, skin=1.0, ewald_beta=0.3)),
}


def _topo(s):
    return Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)


def _setup(name, seed=21, perturb=0.0):
    build, cfg = CASES[name]
    s = build()
    rng = np.random.default_rng(7)
    q = s.q + (rng.normal(scale=perturb, size=s.q.shape) if perturb else 0.0)
    ctx = bounce.from_system(s, seed=seed, jump_coulomb=False, **cfg)
    ctx.set_state(q, s.v, step=3)
    p = Params(r_on=cfg["r_on"], r_off=cfg["r_off"], r_cut=cfg["r_cut"], ewald_beta=cfg.get("ewald_beta", 0.0),
               box=s.box, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps, coulomb_jumps=False)
    md = OracleMD(q, s.v, _topo(s), p, seed=seed, skin=cfg.get("skin", 1.0), step=3)
    md.ensure_rows()
    return s, ctx, md


def _check_sum(g, ref, scale):
    d = np.linalg.norm(g - ref, axis=1)
    cond = d / np.maximum(scale, 1e-30)
    plain = d / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)
    assert cond.max() < TOL, ("conditioned", cond.max(), int(cond.argmax()))
    assert np.percentile(plain, 99) < 2 * TOL, ("plain p99", np.percentile(plain, 99))


def _rel_err(a, ref):
    scale = np.maximum(np.linalg.norm(ref, axis=1), 1e-3 * math.sqrt((ref ** 2).sum(1).mean()))
    return np.linalg.norm(a - ref, axis=1) / scale


@pytest.mark.parametrize("name", list(CASES))
def test_bounds_lj_only(name):
    s, ctx, md = _setup(name)
    L, Ls = ctx.bounds()
    assert np.allclose(L, md.L, rtol=1e-9, atol=0)
    assert np.allclose(Ls, md.Lstar, rtol=1e-9, atol=0)
    # water's hydrogens carry no LJ: nothing of theirs is on the jumps
    assert Ls[1] == 0.0 and Ls[0] > 0.0
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("part", ["full", "short", "long"])
def test_split_gradients(name, part):
    s, ctx, md = _setup(name, perturb=0.05)
    code = {"full": bounce.GRAD_FULL, "short": bounce.GRAD_SHORT, "long": bounce.GRAD_LONG}[part]
    g = ctx.gradient(code)
    ref = {"full": md.grad_full, "short": md.grad_short, "long": md.grad_long}[part]()
    _check_sum(g, ref, md.grad_scale(part))
    if part == "long":
        # the long part is pure LJ: zero on every hydrogen
        assert np.all(g[s.type == 1] == 0.0)
    ctx.close()


@pytest.mark.parametrize("stream_id", [1, 2])
def test_jump_half_lj_only(stream_id):
    s, ctx, md = _setup("droplet", perturb=0.05)
    step = 4242
    M, A = ctx.jump_half(step, stream_id)
    _, v = ctx.get_state()
    v_ref, rec = jump_half(md.q, md.v, md.row_list, md.topo, md.p, md.Lstar, md.beta, md.dt, md.seed, step,
                           stream_id, record=True)
    assert np.array_equal(M, rec["M"])
    assert M.sum() > 50 and M[s.type == 1].sum() == 0
    tie = np.zeros(len(M), bool)
    tie[rec["atom"][np.abs(rec["U"] - rec["ratio"]) < 1e-6]] = True
    acc_ref = np.bincount(rec["atom"][rec["accepted"].astype(bool)], minlength=len(M))
    assert np.array_equal(A[~tie], acc_ref[~tie])
    err = _rel_err(v, v_ref)
    assert err[~tie].max() < TOL, err[~tie].max()
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
def test_one_bounce_step_lj_only(name):
    s, ctx, md = _setup(name)
    q0 = md.q.copy()
    ctx.run(1, bounce.BOUNCE)
    tie = np.zeros(s.n_atoms, bool)
    for r in md.step_bounce(record=True):
        tie[r["atom"][np.abs(r["U"] - r["ratio"]) < 1e-6]] = True
    q, v = ctx.get_state()
    dq = np.linalg.norm(q - md.q, axis=1) / np.maximum(np.linalg.norm(md.q - q0, axis=1), 1e-6)
    assert dq[~tie].max() < TOL, dq[~tie].max()
    # F_0 now holds the whole Coulomb sum, with heavy cancellation: the kick's
    # error scale is dt 4.184e-4 / m times the summed magnitudes of its terms
    kscale = md.dt * ACCEL / md.topo.mass * md.grad_scale("short")
    dv = np.linalg.norm(v - md.v, axis=1)
    assert (dv / (np.linalg.norm(md.v, axis=1) + kscale))[~tie].max() < TOL
    assert np.percentile((dv / np.linalg.norm(md.v, axis=1))[~tie], 99) < 2 * TOL
    e = ctx.energies()
    assert e["proposals"] > 0
    ctx.close()


def test_jump_rows_keep_the_lj_partners_over_rebuilds():
    """LJ alone on the jumps with one bound per type: the jump rows keep only
    the O partners of O atoms and are rebuilt when an O atom has moved half
    the skin (H atoms neither propose nor are drawn).  Ten BOUNCE steps of the
    droplet with a 0.2 A row skin, so that the jump rows are rebuilt within
    them, against the oracle's ten steps: the same rebuilds and proposals,
    and positions within the several-step bound (1e-4, as for the 20-step
    trajectory test) relative to the length of the path travelled (atoms
    with a near tie, and their row partners, left out)."""
    build, cfg = CASES["droplet"]
    s = build()
    cfg = dict(cfg, skin=0.2)
    ctx = bounce.from_system(s, seed=21, jump_coulomb=False, **cfg)
    ctx.set_state(s.q, s.v, step=3)
    p = Params(r_on=cfg["r_on"], r_off=cfg["r_off"], r_cut=cfg["r_cut"], box=s.box, lj_sigma=s.lj_sigma,
               lj_eps=s.lj_eps, coulomb_jumps=False)
    md = OracleMD(s.q, s.v, _topo(s), p, seed=21, skin=0.2, step=3)
    assert md.jp is not None
    ctx.run(10, bounce.BOUNCE)
    tie = np.zeros(s.n_atoms, bool)
    path = np.zeros(s.n_atoms)
    for _ in range(10):
        qp = md.q.copy()
        recs = md.step_bounce(record=True)
        path += np.linalg.norm(md.q - qp, axis=1)
        for r in recs:
            t = r["atom"][np.abs(r["U"] - r["ratio"]) < 1e-6]
            tie[t] = True
            for i in t:
                tie[md.jrows[i]] = True
    e = ctx.energies()
    assert md.rebuilds >= 2, md.rebuilds
    assert e["rebuilds"] == md.rebuilds
    assert e["proposals"] == md.proposals and md.proposals > 0
    q, v = ctx.get_state()
    dq = np.linalg.norm(q - md.q, axis=1) / np.maximum(path, 1e-6)
    assert dq[~tie].max() < 10 * TOL, dq[~tie].max()
    # the readers got full rows; the run's jump rows hold O partners only
    rows = ctx.rows()
    o = int(np.nonzero(s.type == 0)[0][0])
    assert np.any(s.type[rows[o]] == 1)
    assert all(np.all(s.type[md.jrows[i]] == 0) for i in range(s.n_atoms) if s.type[i] == 0)
    ctx.close()


def test_idle_rows_completed_for_readers():
    """With LJ alone on the jumps, H atoms have L* = 0 and never propose, so a
    run on clusters builds no rows for them.  Entry points that read every
    row (energies, pair histogram) complete them first: their results at the
    run's final state match the oracle's, and calling them between two runs
    leaves the trajectory (rebuild steps included) bit for bit unchanged."""
    s, ctx, md = _setup("box_ewald")
    assert ctx.bounds()[1][1] == 0.0           # H: no LJ, no jump bound
    ctx.run(30, bounce.BOUNCE)
    q, v = ctx.get_state()
    e = ctx.energies()
    ref = OracleMD(q, v, md.topo, md.p, seed=21, skin=1.0, step=33)
    er = ref.energies()
    sc, sl = ref.energy_scale()
    for k_gpu, k_ref, scale in (("coulomb", "coul", sc), ("lj", "lj", sl)):
        assert abs(e[k_gpu] - er[k_ref]) < 1e-6 * scale + 1e-9, (k_gpu, e[k_gpu], er[k_ref])
    from oracle.observables import pair_histogram
    h = ctx.pair_histogram(0, 1, 8.0, 32)
    assert np.array_equal(h, pair_histogram(q, s.type, s.molecule, 0, 1, 8.0, 32, s.box))
    # the same 60 steps with and without readers in between
    out = []
    for readers in (True, False):
        c2 = bounce.from_system(s, seed=21, jump_coulomb=False, **CASES["box_ewald"][1])
        c2.set_state(s.q, s.v, step=3)
        for _ in range(3):
            c2.run(20, bounce.BOUNCE)
            if readers:
                c2.energies()
                c2.pair_histogram(0, 0, 8.0, 32)
        e2 = c2.energies()
        out.append((c2.get_state(), e2["rebuilds"], e2["proposals"]))
        c2.close()
    (q1, v1), *c1 = out[0]
    (q2, v2), *c2_ = out[1]
    assert np.array_equal(q1, q2) and np.array_equal(v1, v2) and c1 == c2_
    ctx.close()
