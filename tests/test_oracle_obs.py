"""Pins for the oracle's observables (no GPU)."""
import itertools
import math

import numpy as np

from oracle.observables import bin_edges_sq, msd, pair_histogram
from paper_2002_07109_gb300.water import water_box, water_droplet


def test_histogram_matches_direct_loop():
    s = water_droplet(2, seed=1)
    r_max, nb = 8.0, 40
    h = pair_histogram(s.q, s.type, s.molecule, 0, 1, r_max, nb)
    want = np.zeros(nb, np.int64)
    for i, j in itertools.combinations(range(s.n_atoms), 2):
        if s.molecule[i] == s.molecule[j] or {int(s.type[i]), int(s.type[j])} != {0, 1}:
            continue
        r = math.sqrt(float(((s.q[i] - s.q[j]) ** 2).sum()))
        k = int(r // (r_max / nb))
        if k < nb:
            want[k] += 1
    assert np.array_equal(h, want)


def test_histogram_total_counts_pairs_in_range():
    s = water_box(4, seed=2)
    h = pair_histogram(s.q, s.type, s.molecule, 0, 0, 6.0, 60, s.box)
    o = np.nonzero(s.type == 0)[0]
    d = s.q[o][:, None, :] - s.q[o][None, :, :]
    d -= s.box * np.rint(d / s.box)
    r = np.sqrt((d ** 2).sum(-1))
    iu = np.triu_indices(len(o), 1)
    assert h.sum() == int((r[iu] < 6.0).sum())
    E = bin_edges_sq(6.0, 60)
    assert E[0] == 0.0 and abs(E[-1] - 36.0) < 1e-12


def test_msd_of_a_translation():
    s = water_droplet(2, seed=0)
    q = s.q + np.array([0.3, -0.4, 1.2])
    assert abs(msd(q, s.q, s.type, 0) - (0.09 + 0.16 + 1.44)) < 1e-12
