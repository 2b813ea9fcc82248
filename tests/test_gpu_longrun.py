"""Long-run observables of the GPU path against the oracle, statistically.

Independent realisations of the same process on both sides (the GPU library
and the FP64 oracle, same equilibrated start, different Philox seeds): four
runs of 20,000 BOUNCE steps each of the 64-molecule droplet (all pairs, LJ
on jumps beyond a 4-5 A switch, Coulomb wholly in F_0, per-type-pair bounds,
1 fs, the workloads' friction of 1/ps), the oracle's four runs in a spawn
process pool beside the GPU runs.  Observables per block of 4 ps (four
times the thermostat's relaxation time 1/gamma, so that the block means are
nearly independent): the mean potential energy per molecule, the kinetic
temperature, the O-O coordination number within 3.5 A (the first shell of
the O-O pair-distance histogram, the droplet's RDF observable) and the O
self-diffusion coefficient from the growth of the mean squared displacement
over the block's second half.  Each must agree within three combined
standard errors (of the 20 block means per side; of the four run means for
the coordination number, a histogram observable; for four independent
scalars, two standard errors would fail a correct program about one time in
six; three, about one time in a hundred); the whole O-O histogram (0-8 A,
0.25 A bins) is compared by its chi^2 per bin, with standard errors from the
spread of the runs.  The printed z values are the
per-observable agreement in standard errors.  This split keeps reflections
rare, so the trajectories stay at the equilibrium temperature; with Coulomb
on the jumps at this switch BOUNCE heats flexible water at 1 fs on both
sides alike.
"""
import math
import multiprocessing as mp

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from oracle.longrun import run_blocks
from paper_2002_07109_gb300.water import water_droplet

bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

RUNS, BLOCKS, BLOCK, EVERY = 4, 5, 4000, 20
R_SHELL, H_RMAX, H_BINS = 3.5, 8.0, 32
GAMMA = 0.001


def _stats(x):
    x = np.asarray(x, dtype=np.float64)
    return x.mean(0), x.std(0, ddof=1) / math.sqrt(len(x))


def _gpu_blocks(s, q0, v0, seed, cfg):
    n_mol = int(s.molecule.max()) + 1
    ctx = bounce.from_system(s, seed=seed, gamma=GAMMA, **cfg)
    ctx.set_state(q0, v0, step=0)
    out = {"pe": [], "T": [], "hist": [], "D": []}
    for _ in range(BLOCKS):
        ctx.set_msd_reference()
        pe, T, hist, m = [], [], np.zeros(H_BINS), []
        for k in range(BLOCK // EVERY):
            ctx.run(EVERY, bounce.BOUNCE)
            e = ctx.energies()
            pe.append(e["potential"] / n_mol)
            T.append(e["temperature"])
            hist += ctx.pair_histogram(0, 0, H_RMAX, H_BINS)
            if (k + 1) * EVERY in (BLOCK // 2, BLOCK):
                m.append(ctx.msd(0))
        out["pe"].append(np.mean(pe))
        out["T"].append(np.mean(T))
        out["hist"].append(hist / (BLOCK // EVERY))
        out["D"].append((m[1] - m[0]) / (6.0 * (BLOCK // 2) * 1e-3))
    ctx.close()
    return {k: np.asarray(v) for k, v in out.items()}


def test_long_run_observables_match_oracle():
    s = water_droplet(4, seed=0)
    n_o = int((s.type == 0).sum())
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=math.inf, jump_coulomb=False, pair_bounds=True)
    eq = bounce.from_system(s, seed=100, gamma=0.05, **cfg)
    eq.set_state(s.q, s.v)
    eq.run(3000, bounce.BAOAB)
    q0, v0 = eq.get_state()
    eq.close()

    sysd = {k: getattr(s, k) for k in ("type", "mass", "charge", "molecule", "bonds", "bond_k_r0", "angles",
                                       "angle_k_t0", "lj_sigma", "lj_eps")}
    kw = dict(n_blocks=BLOCKS, block=BLOCK, every=EVERY, gamma=GAMMA, r_on=4.0, r_off=5.0, hist_rmax=H_RMAX,
              hist_bins=H_BINS)
    with mp.get_context("spawn").Pool(RUNS) as pool:
        jobs = [pool.apply_async(run_blocks, (sysd, q0, v0, 2 + 17 * r), kw) for r in range(RUNS)]
        gpu = [_gpu_blocks(s, q0, v0, 1 + 17 * r, cfg) for r in range(RUNS)]
        ora = [j.get() for j in jobs]

    def pooled(runs, key):
        return np.concatenate([r[key] for r in runs])

    # coordination number within R_SHELL: pairs per O in the histogram bins below it
    n_shell = int(round(R_SHELL / (H_RMAX / H_BINS)))
    z = {}
    for key in ("pe", "T", "D", "coord"):
        if key == "coord":
            # a histogram observable: standard errors from the spread of the
            # runs' means, as for the histogram below
            a = [r["hist"][:, :n_shell].sum(1).mean() * 2.0 / n_o for r in gpu]
            b = [r["hist"][:, :n_shell].sum(1).mean() * 2.0 / n_o for r in ora]
        else:
            a, b = pooled(gpu, key), pooled(ora, key)
        m1, e1 = _stats(a)
        m2, e2 = _stats(b)
        z[key] = abs(m1 - m2) / math.hypot(e1, e2)
        print(key, "gpu %.4f +- %.4f  oracle %.4f +- %.4f  z %.2f" % (m1, e1, m2, e2, z[key]))
    # the histogram's slow parts (the droplet's shape) correlate the blocks of
    # one run: its bins (and the coordination number above) take their
    # standard errors from the spread of the independent runs' means (t with
    # 2 (RUNS - 1) degrees of freedom, whose z^2 has mean 1.5 for four runs
    # per side)
    h1, s1 = _stats([r["hist"].mean(0) for r in gpu])
    h2, s2 = _stats([r["hist"].mean(0) for r in ora])
    ok = (s1 + s2) > 0
    zb = np.abs(h1 - h2)[ok] / np.hypot(s1, s2)[ok]
    chi2 = float((zb ** 2).mean())
    print("O-O histogram: chi^2 per bin %.2f, largest bin z %.2f, over %d bins" % (chi2, zb.max(), int(ok.sum())))
    assert all(v < 3.0 for v in z.values()), z
    assert chi2 < 3.0, chi2
    # the runs stay at equilibrium (no jump heating at this split)
    assert abs(np.mean(pooled(gpu, "T")) - 300.0) < 15.0
