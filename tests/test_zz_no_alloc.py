"""The allocation-free pair-energy entry point against the context's energy
entry point (bounce_get_energies), through the C ABI, on two calls in a row.

Callers that cannot allocate device memory (code running under another
framework's CUDA-graph capture, inside a caching allocator that owns the
pool, or on hosts that forbid allocation after start-up) use
bounce_pair_energy_noalloc; its results must equal the regular path's within
the tolerance of the other energy tests: |dE| <= 1e-6 * sum |terms|.
Collected last on purpose (file name), and self-contained so it also passes
alone in a fresh process.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

from oracle.forcefield import Params, pair_energy_magnitudes
from oracle.neighbors import rows, to_pairs
from paper_2002_07109_gb300.water import water_box, water_droplet_molecules

CASES = {
    "droplet_cutoff": (lambda: water_droplet_molecules(300, seed=2), dict(r_cut=9.0)),
    "droplet_all_pairs": (lambda: water_droplet_molecules(120, seed=5), dict(r_cut=math.inf)),
    "box_ewald": (lambda: water_box(6, seed=3), dict(r_cut=8.0, ewald_beta=0.35)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_context_energies(name):
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
    dev = torch.device("cuda", 0)
    tq = torch.tensor(q, dtype=torch.float64, device=dev)
    tc = torch.tensor(s.charge, dtype=torch.float64, device=dev)
    tt = torch.tensor(s.type, dtype=torch.int32, device=dev)
    tm = torch.tensor(s.molecule, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
        r = bounce.pair_energy_noalloc(tq, tc, tt, tm, s.lj_sigma, s.lj_eps, cfg["r_cut"], cfg.get("ewald_beta", 0.0),
                                       s.box, out, stream)
        assert r == 0, r
        torch.cuda.synchronize()
        coul, lj = out.cpu().numpy()
        assert abs(coul - e["coulomb"]) < 1e-6 * sc + 1e-9, (call, coul, e["coulomb"])
        assert abs(lj - e["lj"]) < 1e-6 * sl + 1e-9, (call, lj, e["lj"])


def test_noalloc_rejects_oversized_systems():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    n = bounce.NOALLOC_MAX_ATOMS + 1
    dev = torch.device("cuda", 0)
    z = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    zi = torch.zeros(n, dtype=torch.int32, device=dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    r = bounce.pair_energy_noalloc(z, z[:, 0].contiguous(), zi, zi, np.ones((1, 1)), np.zeros((1, 1)), math.inf, 0.0,
                                   None, out, None)
    assert r == -1
