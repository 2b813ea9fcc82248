"""Edge cases of the GPU path: degenerate and ragged systems against the
oracle, and the error codes for inputs the library must refuse.

  * one molecule: no candidates, no proposals; BOUNCE is BAOAB bit for bit;
  * two molecules (6 atoms, one partial CTA of the 32-atom step kernel):
    one step against the oracle, Poisson counts bit-exact;
  * 1,000 molecules (3,000 atoms, a ragged last CTA) with per-type-pair
    bounds: jump half-step against the oracle;
  * a row longer than max_neighbors: LIST_OVERFLOW, never a silent truncation;
  * non-finite positions, an empty topology, a type outside the table: refused.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.forcefield import Params
from oracle.integrate import OracleMD, Topology, jump_half
from paper_2002_07109_gb300.water import water_droplet, water_droplet_molecules

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

TOL = 1e-5


def _topo(s):
    return Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)


def test_single_molecule_bounce_is_baoab():
    s = water_droplet(1, seed=3)
    out = []
    for integ in (bounce.BOUNCE, bounce.BAOAB):
        ctx = bounce.from_system(s, seed=5, r_on=4.0, r_off=5.0)
        ctx.set_state(s.q, s.v, step=0)
        ctx.run(7, integ)
        out.append(ctx.get_state())
        if integ == bounce.BOUNCE:
            assert ctx.energies()["proposals"] == 0
            assert all(len(r) == 0 for r in ctx.rows())
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_two_molecules_one_step():
    s = water_droplet_molecules(2, seed=4)
    cfg = dict(r_on=1.5, r_off=2.5, r_cut=math.inf)     # a short switch: the pair has jumps
    ctx = bounce.from_system(s, seed=9, **cfg)
    ctx.set_state(s.q, s.v, step=5)
    p = Params(r_on=1.5, r_off=2.5, r_cut=math.inf, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    md = OracleMD(s.q, s.v, _topo(s), p, seed=9, step=5)
    md.ensure_rows()
    M, A = ctx.jump_half(77, 1)
    _, v = ctx.get_state()
    v_ref, rec = jump_half(md.q, md.v, md.row_list, md.topo, md.p, md.Lstar, md.beta, md.dt, md.seed, 77, 1,
                           record=True)
    assert np.array_equal(M, rec["M"]) and M.sum() > 0
    tie = np.zeros(len(M), bool)
    tie[rec["atom"][np.abs(rec["U"] - rec["ratio"]) < 1e-6]] = True
    dv = np.linalg.norm(v - v_ref, axis=1) / np.linalg.norm(v_ref, axis=1)
    assert dv[~tie].max() < TOL
    ctx.close()


def test_ragged_typed_jump_half():
    s = water_droplet_molecules(1000, seed=8)
    assert s.n_atoms % 32 != 0
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=10.0, skin=1.0)
    ctx = bounce.from_system(s, seed=13, pair_bounds=True, **cfg)
    ctx.set_state(s.q, s.v, step=2)
    p = Params(r_on=4.0, r_off=5.0, r_cut=10.0, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    md = OracleMD(s.q, s.v, _topo(s), p, seed=13, skin=1.0, step=2, pair_bounds=True)
    md.ensure_rows()
    M, A = ctx.jump_half(31, 2)
    _, v = ctx.get_state()
    v_ref, rec = jump_half(md.q, md.v, md.row_list, md.topo, md.p, md.Lstar, md.beta, md.dt, md.seed, 31, 2,
                           record=True, pair_bounds=md.pair_bounds)
    assert np.array_equal(M, rec["M"])
    tie = np.zeros(len(M), bool)
    tie[rec["atom"][np.abs(rec["U"] - rec["ratio"]) < 1e-6]] = True
    acc_ref = np.bincount(rec["atom"][rec["accepted"].astype(bool)], minlength=len(M))
    assert np.array_equal(A[~tie], acc_ref[~tie])
    # the last, partial CTA is covered
    assert M[-(s.n_atoms % 32):].sum() > 0
    ctx.close()


def test_row_overflow_is_reported():
    s = water_droplet_molecules(300, seed=2)
    ctx = bounce.from_system(s, seed=1, r_on=4.0, r_off=5.0, r_cut=9.0, skin=1.0, max_neighbors=32)
    ctx.set_state(s.q, s.v, step=0)
    with pytest.raises(bounce.BounceError, match="LIST_OVERFLOW"):
        ctx.run(1, bounce.BOUNCE)
    ctx.close()


def test_bad_inputs_are_refused():
    s = water_droplet(2, seed=0)
    ctx = bounce.from_system(s, r_on=4.0, r_off=5.0)
    q = s.q.copy()
    q[3, 1] = np.nan
    with pytest.raises(bounce.BounceError, match="NONFINITE"):
        ctx.set_state(q, s.v)
    with pytest.raises(bounce.BounceError, match="INVALID_ARG"):
        ctx.set_topology(np.zeros(0, np.int32), np.zeros(0), np.zeros(0), np.zeros(0, np.int32))
    ctx.close()
    ctx = bounce.Context(r_on=4.0, r_off=5.0)
    bad = s.type.copy()
    bad[0] = bounce.MAX_TYPES
    with pytest.raises(bounce.BounceError, match="INVALID_ARG"):
        ctx.set_topology(bad, s.mass, s.charge, s.molecule)
    ctx.close()


def test_set_state_keeps_valid_rows():
    """A new state within skin/2 of the last row build keeps the rows (no
    rebuild counted); one atom moved further forces a rebuild, and the rows
    then match the oracle's rows at the new positions."""
    from oracle.neighbors import rows as oracle_rows
    s = water_droplet_molecules(300, seed=2)
    ctx = bounce.from_system(s, seed=1, r_on=4.0, r_off=5.0, r_cut=9.0, skin=1.0)
    ctx.set_state(s.q, s.v, step=0)
    ctx.rows()
    n0 = ctx.energies()["rebuilds"]
    q1 = s.q + 0.2
    ctx.set_state(q1, s.v, step=0)
    ctx.rows()
    assert ctx.energies()["rebuilds"] == n0
    q2 = q1.copy()
    q2[5] += np.array([0.6, 0.0, 0.0])
    ctx.set_state(q2, s.v, step=0)
    got = ctx.rows()
    assert ctx.energies()["rebuilds"] == n0 + 1
    ref = oracle_rows(q2, s.molecule, 10.0)
    assert all(np.array_equal(a, b) for a, b in zip(got, ref))
    ctx.close()
