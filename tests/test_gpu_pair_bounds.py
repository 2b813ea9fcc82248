"""GPU parity of the per-type-pair bounds with the two-stage partner choice
(pair_bounds = 1): the bound may depend on the types of both particles
(Sec. V).  The CUDA library against the oracle's jump_half / OracleMD with
pair_bounds on the same seeded inputs: type-grouped rows bit-exact, Poisson
counts bit-exact, decisions identical outside near ties, velocities within
1e-5; batches of replicas reproduce the independent runs bit for bit.
Tolerances and tie handling follow test_gpu_parity.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.forcefield import Params
from oracle.integrate import OracleMD, Topology, jump_half, typed_rows
from paper_2002_07109_gb300.water import concat_systems, water_box, water_droplet, water_droplet_molecules

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

TOL = 1e-5

CASES = {
    "droplet_all_pairs": (lambda: water_droplet(4, seed=0), dict(r_on=4.0, r_off=5.0, r_cut=math.inf)),
    "droplet_cutoff": (lambda: water_droplet_molecules(300, seed=2), dict(r_on=4.0, r_off=5.0, r_cut=9.0, skin=1.0)),
    "box_ewald": (lambda: water_box(6, seed=3), dict(r_on=4.0, r_off=5.0, r_cut=8.0, skin=1.0, ewald_beta=0.35)),
}


def _topo(s):
    return Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)


def _setup(name, seed=11, perturb=0.0):
    build, cfg = CASES[name]
    s = build()
    rng = np.random.default_rng(99)
    q = s.q + (rng.normal(scale=perturb, size=s.q.shape) if perturb else 0.0)
    ctx = bounce.from_system(s, seed=seed, pair_bounds=True, **cfg)
    ctx.set_state(q, s.v, step=7)
    p = Params(r_on=cfg["r_on"], r_off=cfg["r_off"], r_cut=cfg["r_cut"], ewald_beta=cfg.get("ewald_beta", 0.0),
               box=s.box, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    md = OracleMD(q, s.v, _topo(s), p, seed=seed, skin=cfg.get("skin", 1.0), step=7, pair_bounds=True)
    md.ensure_rows()
    return s, ctx, md


def _rel_err(a, ref):
    scale = np.maximum(np.linalg.norm(ref, axis=1), 1e-3 * math.sqrt((ref ** 2).sum(1).mean()))
    return np.linalg.norm(a - ref, axis=1) / scale


@pytest.mark.parametrize("name", list(CASES))
def test_typed_rows_bit_exact(name):
    s, ctx, md = _setup(name, perturb=0.05)
    got = ctx.rows()
    ref, _ = typed_rows(md.row_list, md.topo.type, md.L.shape[0])
    assert len(got) == len(ref)
    for i, (a, b) in enumerate(zip(got, ref)):
        assert np.array_equal(a, b), i
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("stream_id", [1, 2])
def test_typed_jump_half(name, stream_id):
    s, ctx, md = _setup(name, perturb=0.05)
    step = 12345
    M, A = ctx.jump_half(step, stream_id)
    _, v = ctx.get_state()
    v_ref, rec = jump_half(md.q, md.v, md.row_list, md.topo, md.p, md.Lstar, md.beta, md.dt, md.seed, step,
                           stream_id, record=True, pair_bounds=md.pair_bounds)
    assert np.array_equal(M, rec["M"])
    assert M.sum() > 100
    tie = np.zeros(len(M), bool)
    tie[rec["atom"][np.abs(rec["U"] - rec["ratio"]) < 1e-6]] = True
    acc_ref = np.bincount(rec["atom"][rec["accepted"].astype(bool)], minlength=len(M))
    assert np.array_equal(A[~tie], acc_ref[~tie])
    assert A.sum() > 10
    assert _rel_err(v, v_ref)[~tie].max() < TOL
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
def test_typed_one_step(name):
    s, ctx, md = _setup(name)
    q0 = md.q.copy()
    ctx.run(1, bounce.BOUNCE)
    tie = np.zeros(s.n_atoms, bool)
    for r in md.step_bounce(record=True):
        tie[r["atom"][np.abs(r["U"] - r["ratio"]) < 1e-6]] = True
    q, v = ctx.get_state()
    dq = np.linalg.norm(q - md.q, axis=1) / np.maximum(np.linalg.norm(md.q - q0, axis=1), 1e-6)
    assert dq[~tie].max() < TOL, dq[~tie].max()
    assert _rel_err(v, md.v)[~tie].max() < TOL
    assert ctx.energies()["proposals"] == md.proposals
    ctx.close()


def test_typed_bounds_propose_less():
    """Same state and seed: the two-stage choice proposes fewer jumps (water's
    O-H and H-H bounds are below the row maxima)."""
    build, cfg = CASES["droplet_cutoff"]
    s = build()
    props = []
    for pb in (False, True):
        ctx = bounce.from_system(s, seed=3, pair_bounds=pb, **cfg)
        ctx.set_state(s.q, s.v, step=0)
        ctx.run(4, bounce.BOUNCE)
        props.append(ctx.energies()["proposals"])
        ctx.close()
    assert props[1] < 0.8 * props[0], props


def test_typed_batch_equals_independent_runs():
    reps = [water_droplet_molecules(n, seed=k) for k, n in enumerate((20, 35, 27))]
    seeds = [11, 22, 33]
    sysb, off = concat_systems(reps)
    cfg = dict(r_on=4.0, r_off=5.0, max_neighbors=256, pair_bounds=True)
    b = bounce.from_system(sysb, seed=999, **cfg)
    b.set_replicas(off, seeds)
    b.set_state(sysb.q, sysb.v, step=3)
    b.run(4, bounce.BOUNCE)
    qb, vb = b.get_state()
    b.close()
    for r, s in enumerate(reps):
        c = bounce.from_system(s, seed=seeds[r], **cfg)
        c.set_state(s.q + np.array([r * 500.0, 0.0, 0.0]), s.v, step=3)
        c.run(4, bounce.BOUNCE)
        q, v = c.get_state()
        c.close()
        assert np.array_equal(qb[off[r]:off[r + 1]], q), r
        assert np.array_equal(vb[off[r]:off[r + 1]], v), r


def test_typed_rows_need_short_enough_rows():
    s = water_droplet(2, seed=0)
    with pytest.raises(bounce.BounceError):
        bounce.from_system(s, pair_bounds=True, max_neighbors=70000)


@pytest.mark.parametrize("n_mol, typed", [(7000, True), (9000, False)])
def test_rows_large_system(n_mol, typed):
    """21,000 / 27,000 atoms: the row builder's CTA-per-atom path (its bitmaps
    over all atoms exceed the warp-per-atom budget), with and without
    per-type-pair bounds; every row bit-exact."""
    from oracle.neighbors import rows_cell_list
    s = water_droplet_molecules(n_mol, seed=3)
    ctx = bounce.from_system(s, seed=2, pair_bounds=typed, r_on=4.0, r_off=5.0, r_cut=9.0, skin=1.0)
    ctx.set_state(s.q, s.v, step=0)
    got = ctx.rows()
    ref = rows_cell_list(s.q, s.molecule, 10.0)
    if typed:
        ref, _ = typed_rows(ref, s.type, 2)
    assert len(got) == len(ref)
    for i, (a, b) in enumerate(zip(got, ref)):
        assert np.array_equal(a, b), i
    ctx.close()
