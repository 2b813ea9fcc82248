"""GPU parity: the CUDA library against the FP64 oracle on the same seeded
inputs (all calls go through the C ABI via the ctypes binding).

Tolerances.  Candidate rows and Poisson counts: bit-exact.  Thinning
decisions: identical except at atoms where the oracle's |U - lambda/lambda*|
< 1e-6 (counted).  Sums of FP32 pair terms (gradients, energies): the error
of atom i is measured against the sum of the magnitudes of the terms it
adds, c_i = sum_j ||g_ij|| (bonded terms included), which bounds the
rounding error of any floating-point summation; ||dg_i|| <= 1e-5 c_i for
every atom, and the plain relative error ||dg_i|| / ||g_i|| <= 2e-5 at the
99th percentile of the atoms (sums with heavy cancellation have a small
||g_i||, so the plain relative error of those few atoms is not bounded by
the precision).  Velocities after one jump half-step (single pair terms, no
cancellation): ||dv_i|| / ||v_i|| <= 1e-5.  Trajectories over several steps:
the per-step bound, grown by the divergence of nearby trajectories (stated
per test).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import philox
from oracle.forcefield import Params
from oracle.integrate import OracleMD, Topology, jump_half
from oracle.neighbors import rows as oracle_rows
from paper_2002_07109_gb300.water import water_box, water_droplet, water_droplet_molecules

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

TOL = 1e-5


def _topo(s):
    return Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)


def _rel_err(a, ref):
    scale = np.maximum(np.linalg.norm(ref, axis=1), 1e-3 * math.sqrt((ref ** 2).sum(1).mean()))
    return np.linalg.norm(a - ref, axis=1) / scale


CASES = {
    # name: (system builder, config)
    "droplet_all_pairs": (lambda: water_droplet(4, seed=0), dict(r_on=4.0, r_off=5.0, r_cut=math.inf)),
    "droplet_cutoff": (lambda: water_droplet_molecules(300, seed=2), dict(r_on=4.0, r_off=5.0, r_cut=9.0, skin=1.0)),
    "box_ewald": (lambda: water_box(6, seed=3), dict(r_on=4.0, r_off=5.0, r_cut=8.0, skin=1.0, ewald_beta=0.35)),
}
PME_CASE = (lambda: water_box(6, seed=3), dict(r_on=7.0, r_off=8.0, r_cut=9.0, skin=1.0, ewald_beta=0.35,
                                              pme_grid=(20, 20, 20), pme_order=5, max_short=640))


def _setup(name, seed=11, perturb=0.0):
    build, cfg = CASES[name]
    s = build()
    rng = np.random.default_rng(99)
    q = s.q + (rng.normal(scale=perturb, size=s.q.shape) if perturb else 0.0)
    ctx = bounce.from_system(s, seed=seed, **cfg)
    ctx.set_state(q, s.v, step=7)
    p = Params(r_on=cfg["r_on"], r_off=cfg["r_off"], r_cut=cfg["r_cut"], ewald_beta=cfg.get("ewald_beta", 0.0),
               box=s.box, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps, pme_grid=cfg.get("pme_grid"),
               pme_order=cfg.get("pme_order", 5))
    md = OracleMD(q, s.v, _topo(s), p, seed=seed, skin=cfg.get("skin", 1.0), step=7)
    md.ensure_rows()
    return s, ctx, md


CASES_ROWS = dict(CASES, box_large=(lambda: water_box(10, seed=4),
                                     dict(r_on=4.0, r_off=5.0, r_cut=8.0, skin=1.0, ewald_beta=0.35)))


@pytest.mark.parametrize("name", list(CASES_ROWS))
def test_rows_bit_exact(name):
    CASES.setdefault(name, CASES_ROWS[name])
    s, ctx, md = _setup(name, perturb=0.05)
    got = ctx.rows()
    assert len(got) == len(md.row_list)
    for i, (a, b) in enumerate(zip(got, md.row_list)):
        assert np.array_equal(a, b), i
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
def test_bounds_match(name):
    s, ctx, md = _setup(name)
    L, Ls = ctx.bounds()
    assert np.allclose(L, md.L, rtol=1e-9, atol=0)
    assert np.allclose(Ls, md.Lstar, rtol=1e-9, atol=0)
    ctx.close()


def _check_sum(g, ref, scale):
    d = np.linalg.norm(g - ref, axis=1)
    cond = d / np.maximum(scale, 1e-30)
    plain = d / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)
    assert cond.max() < TOL, ("conditioned", cond.max(), int(cond.argmax()))
    assert np.percentile(plain, 99) < 2 * TOL, ("plain p99", np.percentile(plain, 99))
    return cond.max(), np.percentile(plain, 99), plain.max()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("part", ["full", "short", "long"])
def test_gradients(name, part):
    s, ctx, md = _setup(name, perturb=0.05)
    code = {"full": bounce.GRAD_FULL, "short": bounce.GRAD_SHORT, "long": bounce.GRAD_LONG}[part]
    g = ctx.gradient(code)
    ref = {"full": md.grad_full, "short": md.grad_short, "long": md.grad_long}[part]()
    _check_sum(g, ref, md.grad_scale(part))
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
def test_energies(name):
    s, ctx, md = _setup(name, perturb=0.05)
    e = ctx.energies()
    ref = md.energies()
    sc, sl = md.energy_scale()
    scales = {"coulomb": sc, "lj": sl, "bond": abs(ref["bond"]), "angle": abs(ref["angle"]), "kinetic": ref["kin"]}
    for k_gpu, k_ref in (("coulomb", "coul"), ("lj", "lj"), ("bond", "bond"), ("angle", "angle"), ("kinetic", "kin")):
        # pair energies: against the sum of |terms|; bonded and kinetic: plain relative
        assert abs(e[k_gpu] - ref[k_ref]) < 1e-6 * scales[k_gpu] + 1e-9, (k_gpu, e[k_gpu], ref[k_ref])
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("stream_id", [1, 2])
def test_jump_half(name, stream_id):
    s, ctx, md = _setup(name, perturb=0.05)
    step = 12345
    M, A = ctx.jump_half(step, stream_id)
    _, v = ctx.get_state()
    v_ref, rec = jump_half(md.q, md.v, md.row_list, md.topo, md.p, md.Lstar, md.beta, md.dt, md.seed, step,
                           stream_id, record=True)
    # Poisson counts: bit-exact
    assert np.array_equal(M, rec["M"])
    assert M.sum() > 100
    # decisions: identical except at atoms with a near tie in the oracle
    tie = np.zeros(len(M), bool)
    close = np.abs(rec["U"] - rec["ratio"]) < 1e-6
    tie[rec["atom"][close]] = True
    acc_ref = np.bincount(rec["atom"][rec["accepted"].astype(bool)], minlength=len(M))
    assert np.array_equal(A[~tie], acc_ref[~tie])
    assert A.sum() > 10
    err = _rel_err(v, v_ref)
    assert err[~tie].max() < TOL, err[~tie].max()
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("integrator", ["baoab", "bounce"])
def test_one_step(name, integrator):
    s, ctx, md = _setup(name)
    q0 = md.q.copy()
    # velocity error scale: |v| plus the kicks' own error scale (an atom
    # nearly at rest carries the FP32 error of its kicks, not of |v|)
    kscale = _kick_scale(md, "full" if integrator == "baoab" else "short", False)
    code = bounce.BOUNCE if integrator == "bounce" else bounce.BAOAB
    ctx.run(1, code)
    if integrator == "bounce":
        r1, r2 = md.step_bounce(record=True)
        tie = np.zeros(s.n_atoms, bool)
        for r in (r1, r2):
            tie[r["atom"][np.abs(r["U"] - r["ratio"]) < 1e-6]] = True
    else:
        md.step_baoab()
        tie = np.zeros(s.n_atoms, bool)
    q, v = ctx.get_state()
    dq = np.linalg.norm(q - md.q, axis=1) / np.maximum(np.linalg.norm(md.q - q0, axis=1), 1e-6)
    assert dq[~tie].max() < TOL, dq[~tie].max()
    dv = np.linalg.norm(v - md.v, axis=1)
    assert (dv / (np.linalg.norm(md.v, axis=1) + kscale))[~tie].max() < TOL
    assert np.percentile((dv / np.linalg.norm(md.v, axis=1))[~tie], 99) < 2 * TOL
    ctx.close()


def test_run_is_deterministic():
    s, ctx, md = _setup("droplet_cutoff")
    ctx.run(12, bounce.BOUNCE)
    q1, v1 = ctx.get_state()
    ctx.set_state(md.q, md.v, step=7)
    ctx.run(12, bounce.BOUNCE)
    q2, v2 = ctx.get_state()
    assert np.array_equal(q1, q2) and np.array_equal(v1, v2)
    ctx.close()


def test_chunked_runs_equal_one_run():
    """Graph-replayed chunks and direct launches follow one trajectory bit
    for bit: run(70) replays two captured 32-step chunks, the profiling
    entry point launches the same 70 steps one boundary at a time.  A run
    split at other boundaries (1 + 33 + 36 steps) differs first by the
    rounding of two half kicks against one kick; with FP32 pair terms such
    differences occasionally move a term by one unit in the last place and
    then grow with the divergence of nearby trajectories, so that comparison
    takes a bound of 1e-5 A on positions and 1e-5 A/fs on velocities (the
    rms speed is ~1e-2 A/fs) after 70 steps."""
    s, ctx, md = _setup("droplet_cutoff")
    ctx.run(70, bounce.BAOAB)
    q1, v1 = ctx.get_state()
    ctx.set_state(md.q, md.v, step=7)
    ctx.profile_steps(70, bounce.BAOAB)
    q3, v3 = ctx.get_state()
    assert np.array_equal(q1, q3) and np.array_equal(v1, v3)
    ctx.set_state(md.q, md.v, step=7)
    for n in (1, 33, 36):
        ctx.run(n, bounce.BAOAB)
    q2, v2 = ctx.get_state()
    dq, dv = np.abs(q1 - q2).max(), np.abs(v1 - v2).max()
    assert dq < 1e-5 and dv < 1e-5, (dq, dv)
    ctx.close()


def test_no_long_range_bounce_is_baoab():
    s = water_droplet(3, seed=4)
    cfg = dict(r_on=math.inf, r_off=math.inf, r_cut=math.inf)
    outs = []
    for integ in (bounce.BAOAB, bounce.BOUNCE):
        ctx = bounce.from_system(s, seed=3, **cfg)
        ctx.set_state(s.q, s.v)
        ctx.run(10, integ)
        outs.append(ctx.get_state())
        e = ctx.energies()
        ctx.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_multi_step_trajectory_tracks_oracle():
    """20 BOUNCE steps: GPU and oracle stay together until a near tie flips a
    decision (then they may separate); the counted proposals agree.  The
    bound, 1e-4 after up to 20 steps, is the one-step bound of 1e-5 grown by
    the divergence of nearby trajectories of liquid water (a factor of a few
    per ps, here over a few tens of fs, plus the sum of 20 steps' errors)."""
    s, ctx, md = _setup("droplet_all_pairs", seed=21)
    for k in range(20):
        ctx.run(1, bounce.BOUNCE)
        r1, r2 = md.step_bounce(record=True)
        ties = sum(int((np.abs(r["U"] - r["ratio"]) < 1e-6).sum()) for r in (r1, r2))
        q, v = ctx.get_state()
        if ties:
            break
        assert _rel_err(v, md.v).max() < 1e-4, k
    e = ctx.energies()
    assert e["proposals"] > 0
    ctx.close()


def test_full_size_droplet_sampled():
    """4096-molecule droplet with a 12 A cutoff (the benchmark workload):
    rows and full gradients on a sample of atoms (the whole step is in
    test_full_size_droplet_steps)."""
    s = water_droplet(16, seed=0)
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=12.0, skin=1.0)
    ctx = bounce.from_system(s, seed=1, **cfg)
    ctx.set_state(s.q, s.v, step=3)
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(s.n_atoms, 150, replace=False))
    p = Params(r_on=4.0, r_off=5.0, r_cut=12.0, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    ref_rows = oracle_rows(s.q, s.molecule, 13.0, None, atoms=sample)
    got_rows = ctx.rows()
    for a, i in enumerate(sample):
        assert np.array_equal(got_rows[i], ref_rows[a])
    from oracle.forcefield import (pair_gradients, bonded_gradients, pair_gradient_magnitudes,
                                   bonded_gradient_magnitudes)
    from oracle.neighbors import to_pairs
    g = ctx.gradient(bounce.GRAD_FULL)
    ii, jj = to_pairs(ref_rows, sample)
    ref = pair_gradients(s.q, s.charge, s.type, ii, jj, p, "full") + bonded_gradients(
        s.q, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    scale = pair_gradient_magnitudes(s.q, s.charge, s.type, ii, jj, p, "full") + bonded_gradient_magnitudes(
        s.q, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    _check_sum(g[sample], ref[sample], scale[sample])
    ctx.close()


@pytest.mark.parametrize("split, n_steps", [("lj_jumps_rowmax", 3), ("coulomb_jumps_typed", 1)])
def test_full_size_droplet_steps(split, n_steps):
    """The benchmark workload at full size (4096-molecule droplet, r_c 12 A)
    through the launches the benchmark times: run(n) is the step kernel's
    head, body and tail launches.  Every atom against the oracle's n
    B J A O A J B steps.  lj_jumps_rowmax is the benchmark's split (LJ on the
    jumps, Coulomb in F_0, one bound per atom type); coulomb_jumps_typed the
    paper's droplet split with per-type-pair bounds (~1 M proposals per
    step).  Atoms with a near tie, and every atom of their rows, are left out
    of the comparison (a tie may flip one decision).  Positions are compared
    per distance travelled, velocities per their magnitude (at least a tenth
    of the rms speed) and per step (the per-step errors of the n steps add
    up), both at 1e-5."""
    s = water_droplet(16, seed=0)
    lj_only = split == "lj_jumps_rowmax"
    typed = not lj_only
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=12.0, skin=1.0, jump_coulomb=not lj_only, pair_bounds=typed)
    ctx = bounce.from_system(s, seed=7, **cfg)
    ctx.set_state(s.q, s.v, step=11)
    p = Params(r_on=4.0, r_off=5.0, r_cut=12.0, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps, coulomb_jumps=not lj_only)
    md = OracleMD(s.q, s.v, _topo(s), p, seed=7, skin=1.0, step=11, pair_bounds=typed)
    ctx.run(n_steps, bounce.BOUNCE)
    tie_atoms = set()
    path = np.zeros(s.n_atoms)  # distance each atom travels, step by step
    for _ in range(n_steps):
        md.ensure_rows()
        q_prev = md.q.copy()
        for r in md.step_bounce(record=True):
            tie_atoms.update(r["atom"][np.abs(r["U"] - r["ratio"]) < 1e-6].tolist())
        path += np.linalg.norm(md.q - q_prev, axis=1)
    keep = np.ones(s.n_atoms, bool)
    for i in tie_atoms:
        keep[i] = False
        keep[md.row_list[i]] = False
    q, v = ctx.get_state()
    # position error per distance travelled (the per-step relative error does not grow with the steps)
    dq = np.linalg.norm(q - md.q, axis=1) / np.maximum(path, 1e-6)
    assert keep.sum() > 0.75 * s.n_atoms
    assert dq[keep].max() < TOL, dq[keep].max()
    # velocity error per step (the per-step errors add up over the n steps),
    # relative to |v| or a tenth of the rms speed: among 12,288 atoms some are
    # nearly at rest, where the ~1e-8 A/fs absolute error of the FP32 kicks
    # would dominate any relative measure
    rms = math.sqrt((md.v ** 2).sum(1).mean())
    dv = (np.linalg.norm(v - md.v, axis=1) / np.maximum(np.linalg.norm(md.v, axis=1), 0.1 * rms))[keep].max()
    dv /= n_steps
    assert dv < TOL, dv
    if not tie_atoms:
        assert ctx.energies()["proposals"] == md.proposals
    assert md.proposals > (1000 if lj_only else 500000)
    ctx.close()


@pytest.mark.parametrize("name", ["droplet_all_pairs", "box_ewald"])
def test_observables(name):
    from oracle.observables import pair_histogram, msd
    s, ctx, md = _setup(name, perturb=0.05)
    r_max = 8.0
    for ta, tb in ((0, 0), (0, 1), (1, 1)):
        h = ctx.pair_histogram(ta, tb, r_max, 160)
        ref = pair_histogram(md.q, s.type, s.molecule, ta, tb, r_max, 160, s.box)
        assert np.array_equal(h, ref), (ta, tb)
    ctx.set_msd_reference()
    q0 = md.q.copy()
    ctx.run(5, bounce.BAOAB)
    md.run(5, "baoab")
    q, _ = ctx.get_state()
    assert abs(ctx.msd(0) - msd(q, q0, s.type, 0)) < 1e-12 * max(1.0, msd(q, q0, s.type, 0))
    ctx.close()


def _setup_pme(seed=11, perturb=0.05):
    CASES.setdefault("box_pme", PME_CASE)
    return _setup("box_pme", seed=seed, perturb=perturb)


def test_recip_gradient_and_energy():
    from oracle import ewald
    s, ctx, md = _setup_pme()
    g = ctx.gradient(bounce.GRAD_RECIP)
    er, gr = ewald.spme_recip(md.q, s.charge, s.box, 0.35, (20, 20, 20), 5)
    ex, gx = ewald.exclusion(md.q, s.charge, ewald.molecule_pairs(s.molecule), 0.35, s.box)
    # error scale: the magnitudes of the two summed parts
    scale = np.linalg.norm(gr, axis=1) + np.linalg.norm(gx, axis=1)
    _check_sum(g, gr + gx, scale)
    e = ctx.energies()
    ref = md.energies()
    es = ewald.self_energy(s.charge, 0.35)
    assert abs(e["recip"] - ref["recip"]) < 1e-6 * (abs(er) + abs(ex) + abs(es)), (e["recip"], ref["recip"])
    ctx.close()


def _tie_mask(md, n):
    """Atoms to leave out after a run with near ties: each tie atom (one
    decision may flip), its molecule (bonded partners feel its changed
    position through stiff bonds) and its candidate row (pair partners)."""
    keep = np.ones(n, bool)
    mol = md.topo.mol
    for i in md.tie_atoms:
        keep[i] = False
        keep[mol == mol[i]] = False
        if md.row_list is not None:
            keep[md.row_list[i]] = False
    return ~keep


def _kick_scale(md, part, with_recip):
    """||v_i|| error scale of one step: the summed magnitudes of the gradient
    terms an atom is kicked with, times dt 4.184e-4 / m."""
    from oracle import ewald
    from oracle.forcefield import ACCEL
    c = md.grad_scale(part)
    if with_recip:
        t = md.topo
        _, gr = ewald.spme_recip(md.q, t.charge, md.p.box, md.p.ewald_beta, md.p.pme_grid, md.p.pme_order)
        _, gx = ewald.exclusion(md.q, t.charge, ewald.molecule_pairs(t.mol), md.p.ewald_beta, md.p.box)
        c = c + np.linalg.norm(gr, axis=1) + np.linalg.norm(gx, axis=1)
    return md.dt * ACCEL / t_mass(md) * c


def t_mass(md):
    return md.topo.mass


@pytest.mark.parametrize("integrator", ["baoab", "bounce", "bounce_respa", "bounce_respa_ext"])
def test_one_step_with_recip(integrator):
    s, ctx, md = _setup_pme(perturb=0.0)
    q0 = md.q.copy()
    kscale = _kick_scale(md, "full" if integrator == "baoab" else "short", True)
    tie = np.zeros(s.n_atoms, bool)
    if integrator == "baoab":
        ctx.run(1, bounce.BAOAB)
        md.step_baoab()
    elif integrator == "bounce":
        ctx.run(1, bounce.BOUNCE)
        for r in md.step_bounce(record=True):
            tie[r["atom"][np.abs(r["U"] - r["ratio"]) < 1e-6]] = True
    else:
        ctx.set_state(md.q, md.v, step=8)        # RESPA blocks start at multiples of m
        md.step_index = 8
        ctx.run(2, bounce.BOUNCE_RESPA if integrator == "bounce_respa" else bounce.BOUNCE_RESPA_EXT)
        md.run(2, integrator, respa_m=2)
    q, v = ctx.get_state()
    dq = np.linalg.norm(q - md.q, axis=1) / np.maximum(np.linalg.norm(md.q - q0, axis=1), 1e-6)
    assert dq[~tie].max() < TOL, dq[~tie].max()
    dv = np.linalg.norm(v - md.v, axis=1)
    assert (dv / (np.linalg.norm(md.v, axis=1) + kscale))[~tie].max() < TOL
    assert np.percentile((dv / np.linalg.norm(md.v, axis=1))[~tie], 99) < 2 * TOL
    e = ctx.energies()
    assert e["recip"] != 0.0
    ctx.close()


def test_respa_rejects_partial_blocks():
    s, ctx, md = _setup_pme(perturb=0.0)
    ctx.set_state(md.q, md.v, step=8)
    with pytest.raises(bounce.BounceError):
        ctx.run(3, bounce.BOUNCE_RESPA)
    ctx.close()


def test_extended_respa_droplet_block():
    """Extended split without a reciprocal part (droplet): outer kicks carry
    the short-range pair gradient, inner steps only the bonded terms."""
    s, ctx, md = _setup("droplet_cutoff")
    kscale = _kick_scale(md, "short", False)
    ctx.set_state(md.q, md.v, step=10)
    md.step_index = 10
    ctx.run(4, bounce.BOUNCE_RESPA_EXT)
    tie = np.zeros(s.n_atoms, bool)
    for _ in range(2):
        md.block_bounce_respa(2, extended=True)
    q, v = ctx.get_state()
    dv = np.linalg.norm(v - md.v, axis=1)
    # a near tie in any of the 8 jump half-steps may flip one decision: those
    # atoms and their partners are left out, every other atom must agree
    tie = _tie_mask(md, s.n_atoms)
    assert tie.mean() < 0.25, tie.mean()
    err = dv / (np.linalg.norm(md.v, axis=1) + 4 * kscale)
    assert err[~tie].max() < TOL, (err[~tie].max(), len(md.tie_atoms))
    ctx.close()


@pytest.mark.parametrize("case", ["box_pme", "droplet_cutoff"])
def test_respa1_outer_step(case):
    """BOUNCE-RESPA1 (m = 2 inner, m2 = 3 intermediate steps): one outer step
    of 6 BJAOAJB steps against the oracle; the droplet has no reciprocal part."""
    if case == "box_pme":
        s, ctx, md = _setup_pme(perturb=0.0)
        kscale = _kick_scale(md, "short", True)
    else:
        s, ctx, md = _setup(case)
        kscale = _kick_scale(md, "short", False)
    ctx.set_state(md.q, md.v, step=12)
    md.step_index = 12
    ctx.run(6, bounce.BOUNCE_RESPA1)
    md.run(6, "bounce_respa1", respa_m=2, respa_m2=3)
    q, v = ctx.get_state()
    dv = np.linalg.norm(v - md.v, axis=1)
    # a near tie in any of the 12 jump half-steps may flip one decision: those
    # atoms and their partners are left out, every other atom must agree
    tie = _tie_mask(md, s.n_atoms)
    assert tie.mean() < 0.25, tie.mean()
    err = dv / (np.linalg.norm(md.v, axis=1) + 6 * kscale)
    assert err[~tie].max() < TOL, (err[~tie].max(), len(md.tie_atoms))
    ctx.close()


def test_respa1_rejects_partial_outer_steps():
    s, ctx, md = _setup("droplet_cutoff")
    ctx.set_state(md.q, md.v, step=12)
    with pytest.raises(bounce.BounceError):
        ctx.run(4, bounce.BOUNCE_RESPA1)
    ctx.set_state(md.q, md.v, step=8)
    with pytest.raises(bounce.BounceError):
        ctx.run(6, bounce.BOUNCE_RESPA1)
    ctx.close()


def test_full_size_box_pme_sampled():
    """The 32,768-molecule periodic box (98,304 atoms, edge 99.3 A): Ewald
    direct erfc (beta 0.35) within 9 A, SPME 96^3 of order 5, per-type-pair
    bounds.  Rows, the F_0 gradient and the reciprocal gradient (SPME plus the
    same-molecule removal) on a sample of atoms against the oracle."""
    from oracle import ewald
    from oracle.forcefield import (pair_gradients, bonded_gradients, pair_gradient_magnitudes,
                                   bonded_gradient_magnitudes)
    from oracle.neighbors import to_pairs
    s = water_box(32, seed=0)
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=9.0, skin=1.0, ewald_beta=0.35, pme_grid=(96, 96, 96), pme_order=5,
               max_neighbors=1024, pair_bounds=True)
    ctx = bounce.from_system(s, seed=1, **cfg)
    ctx.set_state(s.q, s.v, step=0)
    rng = np.random.default_rng(1)
    sample = np.sort(rng.choice(s.n_atoms, 120, replace=False))
    ref_rows = oracle_rows(s.q, s.molecule, 10.0, s.box, atoms=sample)
    got = ctx.rows()
    from oracle.integrate import typed_rows
    ref_typed, _ = typed_rows(ref_rows, s.type, 2)
    for a, i in enumerate(sample):
        assert np.array_equal(got[i], ref_typed[a]), i
    p = Params(r_on=4.0, r_off=5.0, r_cut=9.0, ewald_beta=0.35, box=s.box, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps,
               pme_grid=(96, 96, 96), pme_order=5)
    ii, jj = to_pairs(ref_rows, sample)
    g = ctx.gradient(bounce.GRAD_SHORT)
    ref = pair_gradients(s.q, s.charge, s.type, ii, jj, p, "short") + bonded_gradients(
        s.q, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0, s.box)
    scale = pair_gradient_magnitudes(s.q, s.charge, s.type, ii, jj, p, "short") + bonded_gradient_magnitudes(
        s.q, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0, s.box)
    _check_sum(g[sample], ref[sample], scale[sample])
    gr = ctx.gradient(bounce.GRAD_RECIP)
    _, g_rec = ewald.spme_recip(s.q, s.charge, s.box, 0.35, (96, 96, 96), 5)
    _, g_exc = ewald.exclusion(s.q, s.charge, ewald.molecule_pairs(s.molecule), 0.35, s.box)
    sc = np.linalg.norm(g_rec, axis=1) + np.linalg.norm(g_exc, axis=1)
    _check_sum(gr[sample], (g_rec + g_exc)[sample], sc[sample])
    ctx.close()


def _shuffled(s, seed):
    """The same system with its molecules renumbered in random order, so that
    atom indices carry no spatial order."""
    import dataclasses
    nm = len(s.molecule) // 3
    perm = np.random.default_rng(seed).permutation(nm)          # new molecule k is old molecule perm[k]
    old_of_new = (3 * perm[:, None] + np.arange(3)).ravel()
    new_of_old = np.empty_like(old_of_new)
    new_of_old[old_of_new] = np.arange(len(old_of_new))
    return dataclasses.replace(
        s, q=s.q[old_of_new], v=s.v[old_of_new], type=s.type[old_of_new], mass=s.mass[old_of_new],
        charge=s.charge[old_of_new], molecule=np.repeat(np.arange(nm, dtype=np.int32), 3),
        bonds=new_of_old[s.bonds].astype(np.int32), angles=new_of_old[s.angles].astype(np.int32))


@pytest.mark.parametrize("typed", [False, True])
def test_rows_windowed_random_order(typed):
    """Rows of a 41,472-atom box whose molecules are numbered in random order:
    the row builder's index window does not span every atom, so members
    outside it take further passes; sampled rows against the oracle's brute
    force, bit for bit (typed: grouped by partner type)."""
    s = _shuffled(water_box(24, seed=8), seed=2)
    ctx = bounce.from_system(s, seed=1, r_on=4.0, r_off=5.0, r_cut=8.0, skin=1.0, ewald_beta=0.35,
                             max_neighbors=1024, pair_bounds=typed)
    ctx.set_state(s.q, s.v, step=0)
    sample = np.sort(np.random.default_rng(3).choice(s.n_atoms, 200, replace=False))
    ref = oracle_rows(s.q, s.molecule, 9.0, s.box, atoms=sample)
    if typed:
        from oracle.integrate import typed_rows
        ref, _ = typed_rows(ref, s.type, 2)
    got = ctx.rows()
    for a, i in enumerate(sample):
        assert np.array_equal(got[i], ref[a]), i
    ctx.close()


@pytest.mark.parametrize("coulomb_jumps", [False, True])
def test_full_size_box_first_step_sampled(coulomb_jumps):
    """The 98,304-atom box in the split and launch configuration the
    benchmark times (Ewald erfc beta 0.35 and LJ within 9 A, SPME 96^3 of
    order 5, jumps beyond a 7.5-8.5 A switch with one bound per atom type,
    row skin 2.5 A, cluster skin 2 A, thread-per-atom step kernel): one BOUNCE
    step through run().  The positions after it depend only on the starting
    state (B with F_0 and the reciprocal gradient, the first jump half-step,
    A O A), so the oracle's first half-step is computed for 3,000 sampled
    atoms from their own rows and pairs and compared atom by atom, relative
    to the distance travelled; near-tie atoms are left out."""
    from oracle import ewald
    from oracle.bounds import bound_table
    from oracle.forcefield import ACCEL, KB, bonded_gradients, pair_gradients
    from oracle.integrate import filter_rows, jump_partners, o_step
    from oracle.neighbors import to_pairs
    s = water_box(32, seed=0)
    rng = np.random.default_rng(8)
    q0 = s.q + rng.normal(scale=0.05, size=s.q.shape)
    cfg = dict(r_on=7.5, r_off=8.5, r_cut=9.0, skin=2.5, pair_skin=3.0, ewald_beta=0.35, pme_grid=(96, 96, 96),
               pme_order=5, max_neighbors=2048, jump_coulomb=coulomb_jumps)
    ctx = bounce.from_system(s, seed=13, **cfg)
    ctx.set_state(q0, s.v, step=0)
    ctx.run(1, bounce.BOUNCE)
    q1, _ = ctx.get_state()
    ctx.close()
    p = Params(r_on=7.5, r_off=8.5, r_cut=9.0, ewald_beta=0.35, box=s.box, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps,
               pme_grid=(96, 96, 96), pme_order=5, coulomb_jumps=coulomb_jumps)
    topo = Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    sample = np.sort(rng.choice(s.n_atoms, 3000, replace=False))
    rows_s = oracle_rows(q0, s.molecule, 11.5, s.box, atoms=sample)
    row_list = [np.zeros(0, np.int64)] * s.n_atoms
    for a, i in enumerate(sample):
        row_list[i] = rows_s[a]
    # B: F_0 (bonded + the (1 - chi) share of the pairs) and the reciprocal gradient at q_0
    ii, jj = to_pairs(rows_s, sample)
    G = pair_gradients(q0, s.charge, s.type, ii, jj, p, "short") + bonded_gradients(
        q0, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0, s.box)
    _, g_rec = ewald.spme_recip(q0, s.charge, s.box, 0.35, (96, 96, 96), 5)
    _, g_exc = ewald.exclusion(q0, s.charge, ewald.molecule_pairs(s.molecule), 0.35, s.box)
    G = G + g_rec + g_exc
    h = 0.5
    v = s.v - ((h * ACCEL) / s.mass)[:, None] * G
    # J over dt/2 (stream 1) with the sampled atoms' rows; the others have none
    # (LJ alone on the jumps: the rows keep only the partners a jump can draw)
    _, Lstar = bound_table(s.charge, s.type, 2, s.lj_sigma, s.lj_eps, p)
    jp = jump_partners(s.type, Lstar, p)
    assert (jp is None) == coulomb_jumps
    jrows = row_list if jp is None else filter_rows(row_list, s.type, jp[0])
    v, rec = jump_half(q0, v, jrows, topo, p, Lstar, 1.0 / (KB * 300.0), 1.0, 13, 0, philox.STREAM_J1,
                       record=True)
    tie = np.zeros(s.n_atoms, bool)
    tie[rec["atom"][np.abs(rec["U"] - rec["ratio"]) < 1e-6]] = True
    q = q0 + h * v
    v = o_step(v, s.mass, 300.0, 0.001, 1.0, 13, 0)
    q = q + h * v
    keep = sample[~tie[sample]]
    dq = np.linalg.norm(q1[keep] - q[keep], axis=1) / np.maximum(np.linalg.norm(q[keep] - q0[keep], axis=1), 1e-6)
    assert dq.max() < TOL, (dq.max(), int(rec["M"].sum()))
    if coulomb_jumps:
        assert rec["M"][sample].sum() > 20         # the jump step ran on the sample


@pytest.mark.parametrize("grid", [(32, 64, 96), (40, 128, 160)])
def test_recip_fft_line_lengths(grid):
    """SPME with grid lines of every kind the FFT takes: lengths 32 M
    (M = 1..5) go to the warp-shuffle transform, others (40) to the batched
    Stockham transform; the reciprocal gradient and energy against the
    oracle's FFT on the same grid."""
    from oracle import ewald
    s = water_box(6, seed=3)
    cfg = dict(r_on=7.0, r_off=8.0, r_cut=9.0, skin=1.0, ewald_beta=0.35, pme_grid=grid, pme_order=5)
    ctx = bounce.from_system(s, seed=1, **cfg)
    ctx.set_state(s.q, s.v, step=0)
    g = ctx.gradient(bounce.GRAD_RECIP)
    er, gr = ewald.spme_recip(s.q, s.charge, s.box, 0.35, grid, 5)
    ex, gx = ewald.exclusion(s.q, s.charge, ewald.molecule_pairs(s.molecule), 0.35, s.box)
    scale = np.linalg.norm(gr, axis=1) + np.linalg.norm(gx, axis=1)
    _check_sum(g, gr + gx, scale)
    e = ctx.energies()
    es = ewald.self_energy(s.charge, 0.35)
    assert abs(e["recip"] - (er + ex + es)) < 1e-6 * (abs(er) + abs(ex) + abs(es)), (e["recip"], er + ex + es)
    ctx.close()
