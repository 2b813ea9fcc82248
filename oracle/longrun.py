"""Long-run observables of the FP64 oracle, block by block (test
infrastructure: only tests/ may import this module).

One independent BOUNCE run (Sec. IV.B, the B J A O A J B step of OracleMD)
from a given state, reduced to block means of the observables that the
long-run comparison with the GPU library uses: the potential energy per
molecule, the kinetic temperature, the O-O pair-distance histogram (the
droplet's RDF observable) and the self-diffusion coefficient of O from the
growth of the mean squared displacement over the second half of each block.
A module-level function so that a `spawn` process pool can run several
seeds at once.
"""
import numpy as np

from oracle.forcefield import KB, Params
from oracle.integrate import OracleMD, Topology
from oracle.observables import msd, pair_histogram


def run_blocks(sysd, q0, v0, seed, *, n_blocks, block, every, gamma, r_on, r_off, hist_rmax, hist_bins,
               coulomb_jumps=False, pair_bounds=True):
    """sysd: dict of the system arrays (type, mass, charge, molecule, bonds,
    bond_k_r0, angles, angle_k_t0, lj_sigma, lj_eps).  Returns a dict of
    per-block arrays: pe (kcal/mol per molecule), T (K), hist (O-O pairs per
    bin, averaged over the block's samples), D (A^2/ps)."""
    topo = Topology(sysd["type"], sysd["mass"], sysd["charge"], sysd["molecule"], sysd["bonds"],
                    sysd["bond_k_r0"], sysd["angles"], sysd["angle_k_t0"])
    p = Params(r_on=r_on, r_off=r_off, r_cut=np.inf, lj_sigma=sysd["lj_sigma"], lj_eps=sysd["lj_eps"],
               coulomb_jumps=coulomb_jumps)
    md = OracleMD(q0, v0, topo, p, seed=seed, gamma=gamma, pair_bounds=pair_bounds)
    n = len(topo.type)
    n_mol = int(topo.mol.max()) + 1
    half = block // 2
    out = {"pe": [], "T": [], "hist": [], "D": []}
    for _ in range(n_blocks):
        q_ref = md.q.copy()
        pe, T, hist, m = [], [], np.zeros(hist_bins), []
        for k in range(block // every):
            md.run(every, "bounce")
            e = md.energies()
            pe.append(e["pot"] / n_mol)
            T.append(2.0 * e["kin"] / (3.0 * n * KB))
            hist += pair_histogram(md.q, topo.type, topo.mol, 0, 0, hist_rmax, hist_bins)
            if (k + 1) * every in (half, block):
                m.append(msd(md.q, q_ref, topo.type, 0))
        out["pe"].append(np.mean(pe))
        out["T"].append(np.mean(T))
        out["hist"].append(hist / (block // every))
        out["D"].append((m[1] - m[0]) / (6.0 * half * md.dt * 1e-3))
    return {k: np.asarray(v) for k, v in out.items()}
