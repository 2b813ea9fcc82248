"""Batched independent replicas: one context advancing several droplets in
the same launches must reproduce, bit for bit, each replica run alone with
its own seed (per-replica Philox keys, indices inside the replica, candidate
rows confined to the replica)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

from paper_2002_07109_gb300.water import concat_systems, water_droplet_molecules


@pytest.mark.parametrize("integrator", ["bounce", "baoab"])
def test_batch_equals_independent_runs(integrator):
    code = bounce.BOUNCE if integrator == "bounce" else bounce.BAOAB
    reps = [water_droplet_molecules(n, seed=k) for k, n in enumerate((20, 35, 27))]
    seeds = [11, 22, (1 << 40) + 33]
    sysb, off = concat_systems(reps)
    cfg = dict(r_on=4.0, r_off=5.0, max_neighbors=256)
    b = bounce.from_system(sysb, seed=999, **cfg)
    b.set_replicas(off, seeds)
    b.set_state(sysb.q, sysb.v, step=3)
    b.run(6, code)
    qb, vb = b.get_state()
    eb = b.energies()
    b.close()
    tot_prop = 0
    for r, s in enumerate(reps):
        c = bounce.from_system(s, seed=seeds[r], **cfg)
        c.set_state(s.q + np.array([r * 500.0, 0.0, 0.0]), s.v, step=3)
        c.run(6, code)
        q, v = c.get_state()
        tot_prop += c.energies()["proposals"]
        c.close()
        assert np.array_equal(qb[off[r]:off[r + 1]], q), r
        assert np.array_equal(vb[off[r]:off[r + 1]], v), r
    assert eb["proposals"] == tot_prop


def test_replica_arguments_are_checked():
    reps = [water_droplet_molecules(n, seed=k) for k, n in enumerate((10, 12))]
    sysb, off = concat_systems(reps)
    b = bounce.from_system(sysb, r_on=4.0, r_off=5.0)
    with pytest.raises(bounce.BounceError):
        b.set_replicas(np.array([0, 7, sysb.n_atoms]), [1, 2])      # splits a molecule
    with pytest.raises(bounce.BounceError):
        b.set_replicas(np.array([0, sysb.n_atoms - 3]), [1])          # does not cover all atoms
    b.close()
