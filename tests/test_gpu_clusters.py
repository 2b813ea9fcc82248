"""The cluster-pair path of the pair sums (systems with a cutoff) against the
FP64 oracle, through the C ABI.

The pair sums of BAOAB's full gradient and of F_0 run over clusters of 8
atoms with a half list of cluster pairs (each pair evaluated once, both sides
accumulated in int64 fixed point).  Checked here, beyond the small cases of
test_gpu_parity.py:
  * a periodic box large enough that most cluster pairs take one periodic
    image for all their atom pairs while the pairs near half a box edge take
    the minimum image per atom pair; Ewald erfc; both the F_0 share with
    Coulomb on the jumps (short-range list) and with Coulomb in F_0;
  * a droplet with the 12 A cutoff of the benchmark workload;
  * the sums are the same on every call and on a second context (fixed-point
    accumulation: the result does not depend on the order of the atomics);
  * Newton's third law: the pair part of the full gradient sums to zero.
Tolerance as for every FP32 pair sum: the error of atom i against the sum of
the magnitudes of its terms, ||dg_i|| <= 1e-5 sum_j ||g_ij||, and the plain
relative error ||dg_i|| / ||g_i|| at the 99th percentile, 2e-5 (the atoms
whose terms cancel most cannot carry a plain relative bound).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.forcefield import Params
from oracle.integrate import OracleMD, Topology
from paper_2002_07109_gb300.water import water_box, water_droplet_molecules

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

TOL = 1e-5


def _topo(s):
    return Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)


CASES = {
    "box_14_coulomb_jumps": (lambda: water_box(14, seed=6),
                             dict(r_on=7.5, r_off=8.5, r_cut=9.0, skin=1.0, ewald_beta=0.35, max_neighbors=1024)),
    "box_14_vdw_jumps": (lambda: water_box(14, seed=6),
                         dict(r_on=4.0, r_off=5.0, r_cut=9.0, skin=1.0, ewald_beta=0.35, max_neighbors=1024,
                              jump_coulomb=False)),
    "droplet_rc12": (lambda: water_droplet_molecules(1000, seed=3),
                     dict(r_on=4.0, r_off=5.0, r_cut=12.0, skin=1.0, max_neighbors=2048)),
}


def _setup(name):
    build, cfg = CASES[name]
    s = build()
    rng = np.random.default_rng(5)
    q = s.q + rng.normal(scale=0.05, size=s.q.shape)
    ctx = bounce.from_system(s, seed=3, **cfg)
    ctx.set_state(q, s.v, step=3)
    p = Params(r_on=cfg["r_on"], r_off=cfg["r_off"], r_cut=cfg["r_cut"], ewald_beta=cfg.get("ewald_beta", 0.0),
               box=s.box, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps, coulomb_jumps=cfg.get("jump_coulomb", True))
    md = OracleMD(q, s.v, _topo(s), p, seed=3, skin=cfg["skin"], step=3)
    md.ensure_rows()
    return s, ctx, md, cfg


@pytest.mark.parametrize("name", list(CASES))
def test_cluster_gradients_match_oracle(name):
    s, ctx, md, cfg = _setup(name)
    for part, code in (("full", bounce.GRAD_FULL), ("short", bounce.GRAD_SHORT)):
        g = ctx.gradient(code)
        ref = md.grad_full() if part == "full" else md.grad_short()
        d = np.linalg.norm(g - ref, axis=1)
        cond = d / np.maximum(md.grad_scale(part), 1e-30)
        plain = d / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)
        assert cond.max() < TOL, (part, cond.max(), int(cond.argmax()))
        assert np.percentile(plain, 99) < 2 * TOL, (part, np.percentile(plain, 99))
    ctx.close()


def test_cluster_sums_are_deterministic_and_newton3():
    s, ctx, md, cfg = _setup("box_14_coulomb_jumps")
    g1 = ctx.gradient(bounce.GRAD_FULL)
    g2 = ctx.gradient(bounce.GRAD_FULL)
    assert np.array_equal(g1, g2)
    ctx2 = bounce.from_system(s, seed=3, **cfg)
    q, v = ctx.get_state()
    ctx2.set_state(q, v, step=3)
    assert np.array_equal(ctx2.gradient(bounce.GRAD_FULL), g1)
    # pairs only (no bonded terms, no reciprocal part): the sum over atoms vanishes
    ref = md.grad_full()
    bonded = md.grad_bonded()
    pair = g1 - bonded
    assert np.abs(pair.sum(0)).max() < 1e-6 * np.abs(ref).sum(0).max()
    ctx.close()
    ctx2.close()


@pytest.mark.parametrize("integrator", ["baoab", "bounce"])
def test_cluster_runs_repeat_bit_for_bit(integrator):
    """Two contexts on one state give the same trajectory bit for bit over
    steps that rebuild the clusters (fixed-point sums, deterministic
    clusters)."""
    build, cfg = CASES["box_14_coulomb_jumps"]
    s = build()
    code = bounce.BOUNCE if integrator == "bounce" else bounce.BAOAB
    out = []
    for _ in range(2):
        ctx = bounce.from_system(s, seed=9, **cfg)
        ctx.set_state(s.q, s.v, step=0)
        ctx.run(40, code)
        out.append(ctx.get_state())
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("integrator, split", [("bounce", "coulomb_jumps"), ("bounce", "typed"),
                                                ("bounce_respa1", "coulomb_jumps"), ("baoab", "-")])
def test_thread_per_atom_step_kernel_is_bitwise(integrator, split):
    """The thread-per-atom step kernel (rare proposals) and the cooperative
    32-atom kernel follow the same trajectory bit for bit, counters
    included, over steps with jump proposals, reflections and rebuilds."""
    build, cfg = CASES["box_14_coulomb_jumps"]
    s = build()
    extra = dict(r_on=5.0, r_off=6.0, pair_bounds=split == "typed")   # a closer switch: more proposals
    if integrator == "bounce_respa1":
        extra.update(respa_m=2, respa_m2=2)
    code = {"bounce": bounce.BOUNCE, "bounce_respa1": bounce.BOUNCE_RESPA1, "baoab": bounce.BAOAB}[integrator]
    out = []
    for sk in (1, 2):
        ctx = bounce.from_system(s, seed=5, **dict(cfg, **extra), step_kernel=sk)
        ctx.set_state(s.q, s.v, step=0)
        ctx.run(40, code)
        e = ctx.energies()
        out.append((ctx.get_state(), e["proposals"], e["accepts"], e["near_ties"]))
        ctx.close()
    (q1, v1), *c1 = out[0]
    (q2, v2), *c2 = out[1]
    assert np.array_equal(q1, q2) and np.array_equal(v1, v2)
    assert c1 == c2
    if integrator != "baoab":
        assert c1[0] > 100 and c1[1] > 0


@pytest.mark.parametrize("pair_skin", [1.0, 2.0])
def test_pruned_lists_after_a_run(pair_skin):
    """After steps that moved the atoms (cluster lists built once or twice,
    pruned again several times), the pair sums read the current pruned lists
    and still hold every pair inside the cutoff: the full gradient at the
    run's final state against the oracle's."""
    build, cfg = CASES["box_14_coulomb_jumps"]
    s = build()
    cfg = dict(cfg, pair_skin=pair_skin)
    ctx = bounce.from_system(s, seed=3, **cfg)
    ctx.set_state(s.q, s.v, step=0)
    ctx.run(60, bounce.BAOAB)
    q, v = ctx.get_state()
    p = Params(r_on=cfg["r_on"], r_off=cfg["r_off"], r_cut=cfg["r_cut"], ewald_beta=cfg["ewald_beta"], box=s.box,
               lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    md = OracleMD(q, v, _topo(s), p, seed=3, skin=cfg["skin"], step=60)
    md.ensure_rows()
    g = ctx.gradient(bounce.GRAD_FULL)
    ref = md.grad_full()
    d = np.linalg.norm(g - ref, axis=1)
    assert (d / md.grad_scale("full")).max() < TOL
    assert np.percentile(d / np.linalg.norm(ref, axis=1), 99) < 2 * TOL
    e = ctx.energies()
    assert e["full_pairs"] > 0
    ctx.close()


@pytest.mark.parametrize("name", ["box_14_coulomb_jumps", "droplet_rc12"])
def test_reused_context_repeats_a_fresh_one(name):
    """set_state resets everything a run leaves behind (cluster lists and
    their pruned copies, slot copies in both position buffers): a context
    that ran 70 steps and is set back to the start follows the fresh
    context's next 70 steps bit for bit."""
    build, cfg = CASES[name]
    s = build()
    out = []
    for warm in (0, 70):
        ctx = bounce.from_system(s, seed=11, **cfg)
        ctx.set_state(s.q, s.v, step=7)
        if warm:
            ctx.run(warm, bounce.BAOAB)
            ctx.set_state(s.q, s.v, step=7)
        ctx.run(70, bounce.BAOAB)
        out.append(ctx.get_state())
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
