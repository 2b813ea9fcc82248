"""The all-pairs tile path of the pair sums (droplets and replica batches
without a cutoff) and the autotuner, against the FP64 oracle through the C
ABI.

The pair sums of BAOAB's full gradient and of F_0 (with Coulomb wholly in
F_0, so that F_0 spans every pair) run over static items of 32-atom i-tiles
against j-blocks, each pair once, both sides in int64 fixed point.  Checked:
a droplet whose atom count is not a multiple of 32 (ragged last tile and
j-block) for every j-block length the autotuner may choose, repeatability,
and the autotuner on a droplet (tiles) and on a box (cluster columns).
Tolerance: the error of atom i against the sum of the magnitudes of its
FP32 terms, 1e-5, and the plain relative error at the 99th percentile, 2e-5
(the atoms whose terms cancel most cannot carry a plain relative bound).
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


def _setup(coulomb_jumps):
    s = water_droplet_molecules(215, seed=4)          # 645 atoms: 20 full tiles and a ragged one
    rng = np.random.default_rng(2)
    q = s.q + rng.normal(scale=0.05, size=s.q.shape)
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=math.inf, jump_coulomb=coulomb_jumps)
    ctx = bounce.from_system(s, seed=3, **cfg)
    ctx.set_state(q, s.v, step=2)
    p = Params(r_on=4.0, r_off=5.0, r_cut=math.inf, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps,
               coulomb_jumps=coulomb_jumps)
    md = OracleMD(q, s.v, Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles,
                                   s.angle_k_t0), p, seed=3, step=2)
    md.ensure_rows()
    return s, ctx, md


def _check(g, ref, scale):
    d = np.linalg.norm(g - ref, axis=1)
    assert (d / scale).max() < TOL, (d / scale).max()
    assert np.percentile(d / np.linalg.norm(ref, axis=1), 99) < 2 * TOL


def test_tile_gradients_match_oracle():
    s, ctx, md = _setup(coulomb_jumps=False)
    full, short = md.grad_full(), md.grad_short()
    for _ in range(2):
        _check(ctx.gradient(bounce.GRAD_FULL), full, md.grad_scale("full"))
        _check(ctx.gradient(bounce.GRAD_SHORT), short, md.grad_scale("short"))
    g1 = ctx.gradient(bounce.GRAD_FULL)
    assert np.array_equal(g1, ctx.gradient(bounce.GRAD_FULL))
    ctx.close()


@pytest.mark.parametrize("integrator", ["baoab", "bounce"])
def test_autotune_keeps_parity(integrator):
    """The autotuner picks a j-block length and grid; the pair sums of the
    chosen shape still match the oracle, and a run continues normally."""
    s, ctx, md = _setup(coulomb_jumps=False)
    code = bounce.BOUNCE if integrator == "bounce" else bounce.BAOAB
    t = ctx.autotune(code)
    assert t["tile_j"] in (32, 64, 128, 256) and t["candidates"] == 12 and t["pair_ms"] > 0
    _check(ctx.gradient(bounce.GRAD_FULL), md.grad_full(), md.grad_scale("full"))
    ctx.run(10, code)
    assert math.isfinite(ctx.energies()["potential"])
    ctx.close()


def test_autotune_cluster_columns():
    s = water_box(10, seed=5)
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=8.0, skin=1.0, ewald_beta=0.35, max_neighbors=1024)
    ctx = bounce.from_system(s, seed=3, **cfg)
    ctx.set_state(s.q, s.v)
    p = Params(r_on=4.0, r_off=5.0, r_cut=8.0, ewald_beta=0.35, box=s.box, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    md = OracleMD(s.q, s.v, Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles,
                                     s.angle_k_t0), p, seed=3)
    md.ensure_rows()
    t = ctx.autotune(bounce.BAOAB)
    assert t["column_edge"] > 2.0 and t["candidates"] == 5
    _check(ctx.gradient(bounce.GRAD_FULL), md.grad_full(), md.grad_scale("full"))
    ctx.run(8, bounce.BAOAB)
    assert math.isfinite(ctx.energies()["potential"])
    ctx.close()
