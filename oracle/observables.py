"""Observables of the paper's accuracy study (Sec. VI: potential energy,
radial distribution functions, self-diffusion by the Einstein relation).

  pair_histogram  counts of unordered pairs (i < j, different molecules) of
                  the type pair {ta, tb} by distance, bins of width
                  w = r_max / n_bins; pair (i, j) falls in bin k when
                  (k w)^2 <= r_ij^2 < ((k+1) w)^2, all in FP64 with
                  r^2 = (dx dx + dy dy) + dz dz (minimum image when periodic).
                  A droplet has no volume to normalise by, so the counts
                  themselves are the observable (this project's reading).
  msd             mean over atoms of one type of |q_i(t) - q_i(0)|^2
                  (unwrapped positions).

Pins: the histogram against a direct loop over pairs on a tiny system and
its total against the number of pairs in range; the MSD against a uniform
translation (tests/test_oracle_obs.py).
"""
import numpy as np

from .forcefield import displacement, r2_of


def bin_edges_sq(r_max, n_bins):
    w = r_max / n_bins
    k = np.arange(n_bins + 1, dtype=np.float64)
    return (k * w) * (k * w)


def pair_histogram(q, typ, mol, ta, tb, r_max, n_bins, box=None):
    q = np.asarray(q, dtype=np.float64)
    n = q.shape[0]
    E = bin_edges_sq(r_max, n_bins)
    hist = np.zeros(n_bins, dtype=np.int64)
    ii, jj = np.triu_indices(n, k=1)
    sel = (mol[ii] != mol[jj]) & (((typ[ii] == ta) & (typ[jj] == tb)) | ((typ[ii] == tb) & (typ[jj] == ta)))
    ii, jj = ii[sel], jj[sel]
    r2 = r2_of(displacement(q[ii], q[jj], box))
    k = np.searchsorted(E, r2, side="right") - 1
    ok = (k >= 0) & (k < n_bins)
    np.add.at(hist, k[ok], 1)
    return hist


def msd(q, q_ref, typ, t):
    d = np.asarray(q, dtype=np.float64) - np.asarray(q_ref, dtype=np.float64)
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    return float(d2[np.asarray(typ) == t].mean())
