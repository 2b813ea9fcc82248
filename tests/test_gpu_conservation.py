"""Energy conservation on the GPU (no friction): a physics check of the whole
pair path over many steps, which single-step parity cannot see.

Without friction BAOAB is velocity Verlet, whose shadow energy is conserved:
the total energy (kinetic + every potential term, reciprocal Ewald included)
fluctuates but does not drift.  A pair the pair sums drop or misplace for
some steps (for instance an atom crossing a periodic face between two builds
of the pair lists) injects energy every time, and the drift shows it.  Runs
of 2,000 steps at 0.5 fs (1 ps) from a state relaxed with strong friction;
the bound, 0.02 kcal/mol per molecule over the run, is a fraction of the
energy of one degree of freedom (k_B T / 2 = 0.3) and far below the drift a
missing-pair error produces (over 1 kcal/mol per molecule per ps).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2002_07109_gb300.water import water_box, water_droplet_molecules

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

CASES = {
    "box_pme": (lambda: water_box(10, seed=2),
                dict(r_on=7.5, r_off=8.5, r_cut=9.0, skin=1.0, ewald_beta=0.35, pme_grid=(32, 32, 32), pme_order=5,
                     max_neighbors=1024)),
    "box_ewald_direct": (lambda: water_box(10, seed=2),
                         dict(r_on=7.5, r_off=8.5, r_cut=9.0, skin=1.0, ewald_beta=0.35, max_neighbors=1024)),
    # a cutoff beyond the droplet's diameter: the cluster path, with no pair
    # crossing the cutoff (plain truncation of Coulomb at a cutoff inside the
    # droplet changes the energy by W(r_c) at every crossing without any
    # force, a random walk of several kcal/mol per molecule per ps)
    "droplet_clusters": (lambda: water_droplet_molecules(300, seed=1),
                         dict(r_on=4.0, r_off=5.0, r_cut=40.0, skin=1.0, max_neighbors=2048)),
    "droplet_all_pairs": (lambda: water_droplet_molecules(300, seed=1), dict(r_on=4.0, r_off=5.0)),
}


def _total(e):
    return e["kinetic"] + e["potential"] + e["recip"]


@pytest.mark.parametrize("name", list(CASES))
def test_baoab_without_friction_conserves_energy(name):
    build, cfg = CASES[name]
    s = build()
    n_mol = s.n_atoms // 3
    eq = bounce.from_system(s, seed=4, gamma=0.05, dt=0.5, **cfg)
    eq.set_state(s.q, s.v)
    eq.run(1000, bounce.BAOAB)
    q, v = eq.get_state()
    eq.close()
    ctx = bounce.from_system(s, seed=4, gamma=0.0, dt=0.5, **cfg)
    ctx.set_state(q, v)
    e0 = _total(ctx.energies())
    trace = []
    for _ in range(10):
        ctx.run(200, bounce.BAOAB)
        trace.append(_total(ctx.energies()))
    drift = (trace[-1] - e0) / n_mol
    assert abs(drift) < 0.02, (drift, [(t - e0) / n_mol for t in trace])
    if s.box is not None:
        # atoms crossed the box faces between list builds (the case the check is for)
        q1, _ = ctx.get_state()
        assert np.any(np.floor(q1 / s.box) != np.floor(q / s.box))
    ctx.close()
