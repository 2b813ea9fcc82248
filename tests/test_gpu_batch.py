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


def test_full_size_batch_sampled():
    """The 256-replica batch (64-1,024 molecules each, seeded sizes, one seed
    per replica) at full size: one BOUNCE step of the whole batch in shared
    launches; three sampled replicas run alone reproduce their part bit for
    bit."""
    from paper_2002_07109_gb300.water import replica_sizes
    sizes = replica_sizes(256, 64, 1024, seed=0)
    reps = [water_droplet_molecules(int(n), seed=r) for r, n in enumerate(sizes)]
    seeds = [1000 + r for r in range(len(reps))]
    sysb, off = concat_systems(reps)
    cfg = dict(r_on=4.0, r_off=5.0, max_neighbors=3 * int(sizes.max()), pair_bounds=True)
    b = bounce.from_system(sysb, seed=1, **cfg)
    b.set_replicas(off, seeds)
    b.set_state(sysb.q, sysb.v, step=0)
    b.run(1, bounce.BOUNCE)
    qb, vb = b.get_state()
    eb = b.energies()
    b.close()
    assert eb["proposals"] > 100 * sysb.n_atoms
    for r in (0, int(np.argmax(sizes)), len(reps) - 1):
        s = reps[r]
        c = bounce.from_system(s, seed=seeds[r], **cfg)
        c.set_state(s.q + np.array([r * 500.0, 0.0, 0.0]), s.v, step=0)
        c.run(1, bounce.BOUNCE)
        q, v = c.get_state()
        c.close()
        assert np.array_equal(qb[off[r]:off[r + 1]], q), r
        assert np.array_equal(vb[off[r]:off[r + 1]], v), r
