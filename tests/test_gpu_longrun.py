"""Long-run observables of the GPU path against the oracle, statistically.

Two independent realisations of the same process (the GPU library and the
FP64 oracle, same equilibrated start, different Philox seeds), 20,000 BOUNCE
steps each of the 64-molecule droplet (all pairs, LJ on jumps beyond a 4-5 A
switch, Coulomb wholly in F_0, per-type-pair bounds, 1 fs, friction 10/ps so
that blocks of 2 ps are independent):
the mean potential energy per molecule, the kinetic temperature and the O-O
coordination number within 3.5 A (the first shell of the O-O pair-distance
histogram, the droplet's RDF observable) must agree within three combined
standard errors of their block means (10 blocks of 100 samples, 20 steps
apart).  The printed z values are the per-observable agreement in standard
errors.  This split keeps reflections rare, so the trajectories stay at the
equilibrium temperature; with Coulomb on the jumps at this switch BOUNCE
heats flexible water at 1 fs on both sides alike.
"""
import math

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from oracle.forcefield import KB, Params
from oracle.integrate import OracleMD, Topology
from oracle.observables import pair_histogram
from paper_2002_07109_gb300.water import water_droplet

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

N_STEPS, EVERY, BLOCKS = 20000, 20, 10
R_SHELL = 3.5


def _block_stats(x):
    b = np.asarray(x).reshape(BLOCKS, -1).mean(1)
    return b.mean(), b.std(ddof=1) / math.sqrt(BLOCKS)


def test_long_run_observables_match_oracle():
    s = water_droplet(4, seed=0)
    n_mol = int(s.molecule.max()) + 1
    n_o = int((s.type == 0).sum())
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=math.inf, jump_coulomb=False, pair_bounds=True)
    eq = bounce.from_system(s, seed=100, gamma=0.05, **cfg)
    eq.set_state(s.q, s.v)
    eq.run(3000, bounce.BAOAB)
    q0, v0 = eq.get_state()
    eq.close()

    gpu = {"pe": [], "T": [], "coord": []}
    ctx = bounce.from_system(s, seed=1, gamma=0.01, **cfg)
    ctx.set_state(q0, v0, step=0)
    for _ in range(N_STEPS // EVERY):
        ctx.run(EVERY, bounce.BOUNCE)
        e = ctx.energies()
        gpu["pe"].append(e["potential"] / n_mol)
        gpu["T"].append(e["temperature"])
        gpu["coord"].append(2.0 * ctx.pair_histogram(0, 0, R_SHELL, 1)[0] / n_o)
    ctx.close()

    topo = Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    p = Params(r_on=4.0, r_off=5.0, r_cut=math.inf, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps, coulomb_jumps=False)
    md = OracleMD(q0, v0, topo, p, seed=2, gamma=0.01, pair_bounds=True)
    ora = {"pe": [], "T": [], "coord": []}
    for _ in range(N_STEPS // EVERY):
        md.run(EVERY, "bounce")
        e = md.energies()
        ora["pe"].append(e["pot"] / n_mol)
        ora["T"].append(2.0 * e["kin"] / (3.0 * s.n_atoms * KB))
        h = pair_histogram(md.q, topo.type, topo.mol, 0, 0, R_SHELL, 1)
        ora["coord"].append(2.0 * h[0] / n_o)

    z = {}
    for k in gpu:
        m1, e1 = _block_stats(gpu[k])
        m2, e2 = _block_stats(ora[k])
        z[k] = abs(m1 - m2) / math.sqrt(e1 * e1 + e2 * e2)
        print(k, "gpu %.4f +- %.4f  oracle %.4f +- %.4f  z %.2f" % (m1, e1, m2, e2, z[k]))
    assert all(v < 3.0 for v in z.values()), z
    # the run stays at equilibrium (no jump heating at this split)
    assert abs(np.mean(gpu["T"]) - 300.0) < 15.0
