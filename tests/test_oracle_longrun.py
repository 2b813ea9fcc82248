"""The oracle's block runner of the long-run comparison (oracle/longrun.py):
with one sample per half block, each block's observables equal what the
oracle's own step and observable functions give along the same trajectory."""
import math

import numpy as np

from oracle.forcefield import KB, Params
from oracle.integrate import OracleMD, Topology
from oracle.longrun import run_blocks
from oracle.observables import msd, pair_histogram
from paper_2002_07109_gb300.water import water_droplet

KEYS = ("type", "mass", "charge", "molecule", "bonds", "bond_k_r0", "angles", "angle_k_t0", "lj_sigma", "lj_eps")


def test_blocks_follow_the_trajectory():
    s = water_droplet(2, seed=1)                  # 8 molecules, 24 atoms
    sysd = {k: getattr(s, k) for k in KEYS}
    every, block, n_blocks = 5, 10, 2
    out = run_blocks(sysd, s.q, s.v, 3, n_blocks=n_blocks, block=block, every=every, gamma=0.01, r_on=4.0,
                     r_off=5.0, hist_rmax=8.0, hist_bins=16)
    assert {k: v.shape for k, v in out.items()} == {"pe": (2,), "T": (2,), "hist": (2, 16), "D": (2,)}

    # the same trajectory by hand: two samples per block, at its middle and end
    topo = Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    p = Params(r_on=4.0, r_off=5.0, r_cut=math.inf, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps, coulomb_jumps=False)
    md = OracleMD(s.q, s.v, topo, p, seed=3, gamma=0.01, pair_bounds=True)
    n_mol = int(s.molecule.max()) + 1
    for b in range(n_blocks):
        q_ref = md.q.copy()
        pe, T, h, m = [], [], np.zeros(16), []
        for _ in range(block // every):
            md.run(every, "bounce")
            e = md.energies()
            pe.append(e["pot"] / n_mol)
            T.append(2.0 * e["kin"] / (3.0 * s.n_atoms * KB))
            h += pair_histogram(md.q, topo.type, topo.mol, 0, 0, 8.0, 16)
            m.append(msd(md.q, q_ref, topo.type, 0))
        assert out["pe"][b] == np.mean(pe)
        assert out["T"][b] == np.mean(T)
        assert np.array_equal(out["hist"][b], h / 2)
        # D from the growth of the MSD over the block's second half (A^2/ps)
        assert out["D"][b] == (m[1] - m[0]) / (6.0 * every * 1e-3)
    # a histogram block mean counts O-O pairs of different molecules: at most n_O (n_O - 1) / 2
    n_o = int((s.type == 0).sum())
    assert np.all(out["hist"].sum(1) <= n_o * (n_o - 1) / 2)
