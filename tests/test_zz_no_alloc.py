"""The allocation-free pair-energy entry point, through the C ABI, on two
calls in a row: against the context's energy entry point
(bounce_get_energies) and against the FP64 oracle's pair energies.

Some callers cannot allocate device memory: code inside an allocator that
owns the whole device pool, or hosts that forbid allocation after start-up.
They use bounce_pair_energy_noalloc; its results must equal the regular
path's and the oracle's within the tolerance of the other energy tests:
|dE| <= 1e-6 * sum |terms|.  Collected last on purpose (file name), and
self-contained so it also passes alone in a fresh process.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

from oracle.forcefield import Params, pair_energies, pair_energy_magnitudes
from oracle.neighbors import rows, to_pairs
from paper_2002_07109_gb300.water import water_box, water_droplet_molecules

CASES = {
    "droplet_cutoff": (lambda: water_droplet_molecules(300, seed=2), dict(r_cut=9.0)),
    "droplet_all_pairs": (lambda: water_droplet_molecules(120, seed=5), dict(r_cut=math.inf)),
    "box_ewald": (lambda: water_box(6, seed=3), dict(r_cut=8.0, ewald_beta=0.35)),
}


def _device_state(s, q):
    dev = torch.device("cuda", 0)
    return (torch.tensor(q, dtype=torch.float64, device=dev), torch.tensor(s.charge, dtype=torch.float64, device=dev),
            torch.tensor(s.type, dtype=torch.int32, device=dev), torch.tensor(s.molecule, dtype=torch.int32, device=dev))


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_context_and_oracle(name):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build, cfg = CASES[name]
    s = build()
    rng = np.random.default_rng(4)
    q = s.q + rng.normal(scale=0.05, size=s.q.shape)
    ctx = bounce.from_system(s, seed=1, r_on=4.0, r_off=5.0, skin=1.0, **cfg)
    ctx.set_state(q, s.v)
    e = ctx.energies()
    ctx.close()
    p = Params(r_cut=cfg["r_cut"], ewald_beta=cfg.get("ewald_beta", 0.0), box=s.box, lj_sigma=s.lj_sigma,
               lj_eps=s.lj_eps)
    ii, jj = to_pairs(rows(q, s.molecule, math.inf, s.box))
    sc, sl = pair_energy_magnitudes(q, s.charge, s.type, ii, jj, p)
    oc, ol = pair_energies(q, s.charge, s.type, ii, jj, p)
    tq, tc, tt, tm = _device_state(s, q)
    dev = tq.device
    stream = torch.cuda.current_stream(dev).cuda_stream
    free = []
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        f0 = torch.cuda.mem_get_info(dev)[0]
        r = bounce.pair_energy_noalloc(tq, tc, tt, tm, s.lj_sigma, s.lj_eps, cfg["r_cut"], cfg.get("ewald_beta", 0.0),
                                       s.box, out, stream)
        assert r == 0, r
        torch.cuda.synchronize()
        free.append((f0, torch.cuda.mem_get_info(dev)[0]))
        coul, lj = out.cpu().numpy()
        assert abs(coul - e["coulomb"]) < 1e-6 * sc + 1e-9, (call, coul, e["coulomb"])
        assert abs(lj - e["lj"]) < 1e-6 * sl + 1e-9, (call, lj, e["lj"])
        assert abs(coul - oc) < 1e-6 * sc + 1e-9, (call, coul, oc)
        assert abs(lj - ol) < 1e-6 * sl + 1e-9, (call, lj, ol)
    # the second call (set-up done by the first) leaves the device's free memory as it found it
    assert free[1][0] == free[1][1], free


def test_noalloc_flags_types_outside_the_table():
    """A type >= n_types is not read from the LJ tables: both totals are NaN,
    and the next call with valid types is correct again (status cleared)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    s = water_droplet_molecules(40, seed=1)
    tq, tc, tt, tm = _device_state(s, s.q)
    out = torch.zeros(2, dtype=torch.float64, device=tq.device)
    bad = tt.clone()
    bad[5] = 3
    assert bounce.pair_energy_noalloc(tq, tc, bad, tm, s.lj_sigma, s.lj_eps, math.inf, 0.0, None, out, None) == 0
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    assert bounce.pair_energy_noalloc(tq, tc, tt, tm, s.lj_sigma, s.lj_eps, math.inf, 0.0, None, out, None) == 0
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()


def test_noalloc_rejects_bad_sizes_and_cutoffs():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda", 0)
    n = bounce.NOALLOC_MAX_ATOMS + 1
    z = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    zi = torch.zeros(n, dtype=torch.int32, device=dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    r = bounce.pair_energy_noalloc(z, z[:, 0].contiguous(), zi, zi, np.ones((1, 1)), np.zeros((1, 1)), math.inf, 0.0,
                                   None, out, None)
    assert r == -1
    # periodic box: the minimum image is the pair sum only for r_cut <= L/2
    s = water_box(3, seed=0)
    tq, tc, tt, tm = _device_state(s, s.q)
    for r_cut in (math.inf, 0.6 * s.box[0]):
        assert bounce.pair_energy_noalloc(tq, tc, tt, tm, s.lj_sigma, s.lj_eps, r_cut, 0.35, s.box, out, None) == -1
    # the binding refuses tensors the entry point would misread
    with pytest.raises(ValueError):
        bounce.pair_energy_noalloc(tq.float(), tc, tt, tm, s.lj_sigma, s.lj_eps, 4.0, 0.35, s.box, out, None)
    with pytest.raises(ValueError):
        bounce.pair_energy_noalloc(tq, tc[:-1], tt, tm, s.lj_sigma, s.lj_eps, 4.0, 0.35, s.box, out, None)
    with pytest.raises(ValueError):
        bounce.pair_energy_noalloc(tq.t().contiguous().t(), tc, tt, tm, s.lj_sigma, s.lj_eps, 4.0, 0.35, s.box, out,
                                   None)
