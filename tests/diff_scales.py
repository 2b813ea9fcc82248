"""Error scales of the force-matching results: per result, the sum of the
magnitudes of the FP32 terms a floating-point evaluation adds up (the scale
that bounds its rounding error, as for every FP32 sum in these tests).

For directed pairs (i, j) with d = q_i - q_j, r = |d| and g = W'(r)/r the
forces are F_i = -sum_j g d.  With u = dL/dF (the upstream gradient):
  * forces:        sum_j |g| r, with |g| the magnitudes of g's Coulomb and
                   LJ terms added (and likewise for g');
  * dL/dq_i:       sum_j (sqrt(3) |g| + |g'| r) (|u_i| + |u_j|) + w_E sum_j |g| r
                   (the pair Hessian g I + (g'/r) d d^T, bounded in norm, on
                   u_i - u_j formed from the two upstream values rounded to
                   FP32, whose errors follow |u_i| + |u_j|);
  * dL/d(param):   sum_pairs (|u_i| + |u_j|) |d(g d)/d(param)| + w_E |dW/d(param)|.
Written here from the pair terms for the test's tolerances only; the values
themselves come from the oracle (oracle/diff.py).
"""
import math

import numpy as np
from scipy.special import erfc

K_COUL = 332.063713


def _terms(q, typ, qt, sig, eps, ii, jj, beta, box):
    d = q[ii] - q[jj]
    if box is not None:
        d = d - box * np.rint(d / box)
    r = np.sqrt((d * d).sum(1))
    ti, tj = typ[ii], typ[jj]
    qq = K_COUL * qt[ti] * qt[tj]
    s = 0.5 * (sig + sig.T)[ti, tj]
    e = 0.5 * (eps + eps.T)[ti, tj]
    s6 = s ** 6
    c12, c6 = 4 * e * s6 * s6, 4 * e * s6
    ex = np.exp(-beta * beta * r * r)
    ec = erfc(beta * r)
    k2 = 2 * beta / math.sqrt(math.pi)
    # Coulomb / Ewald direct: W = qq f, f = erfc(b r)/r
    f = ec / r
    f1 = -ec / r ** 2 - k2 * ex / r
    f2 = 2 * ec / r ** 3 + 2 * k2 * ex / r ** 2 + 2 * k2 * beta * beta * ex
    W = qq * f + (c12 / r ** 12 - c6 / r ** 6)
    W1 = qq * f1 + (-12 * c12 / r ** 13 + 6 * c6 / r ** 7)
    # magnitudes of the terms: W' and W'' add Coulomb and LJ terms of either
    # sign, whose cancellation does not cancel their rounding errors
    A1 = np.abs(qq) * (ec / r ** 2 + k2 * ex / r) + 12 * c12 / r ** 13 + 6 * c6 / r ** 7
    A2 = np.abs(qq) * f2 + 156 * c12 / r ** 14 + 42 * c6 / r ** 8
    g = W1 / r
    g1 = A2 / r + A1 / r ** 2
    return d, r, g, g1, qq, f1, c12, c6, s, e, ti, tj, A1


def scales(q, typ, qt, sig, eps, ii, jj, beta, box, u, w_energy, du_in=None):
    """(force scale [n], dL/dq scale [n], qt scale [T], sig scale [T, T],
    eps scale [T, T]).  du_in (per atom, optional): a bound on the error of
    the upstream gradient u itself (when u is formed from FP32 forces); its
    propagation through the pair Hessian and the parameter derivatives is
    added to the scales."""
    n, T = len(q), len(qt)
    d, r, g, g1, qq, f1, c12, c6, s, e, ti, tj, A1 = _terms(q, typ, qt, sig, eps, ii, jj, beta, box)
    ga = A1 / r
    fs = np.bincount(ii, ga * r, minlength=n)
    nu = np.linalg.norm(u, axis=1)
    du = nu[ii] + nu[jj]
    if du_in is not None:
        # errors of u follow |u| (FP32 rounding of the inputs) plus the given bound
        du = du + (du_in[ii] + du_in[jj]) / 1e-5
    qs = np.bincount(ii, (math.sqrt(3) * ga + g1 * r) * du + w_energy * ga * r, minlength=n)
    # parameter derivatives of g r (the size of d(g d)) and of W, per directed pair
    sq, ss, se = np.zeros(T), np.zeros((T, T)), np.zeros((T, T))
    for a in range(T):
        na = (ti == a).astype(float) + (tj == a).astype(float)
        if qt[a] == 0:
            continue
        dgc = np.abs(qq * f1) * na / abs(qt[a])                 # |d(g d)/d qt_a| of the Coulomb part
        dWc = np.abs(qq * erfc(beta * r) / r) * na / abs(qt[a])  # |dW/d qt_a|
        sq[a] = (dgc * du).sum() + w_energy * 0.5 * dWc.sum()
    for a in range(T):
        for b in range(T):
            m = ((ti == a) & (tj == b)) | ((ti == b) & (tj == a))
            if not m.any():
                continue
            with np.errstate(divide="ignore", invalid="ignore"):
                dg_de = np.where(e[m] != 0, np.abs(-12 * c12[m] / r[m] ** 13 + 6 * c6[m] / r[m] ** 7) / e[m], 0.0)
                dg_ds = np.abs(-144 * c12[m] / r[m] ** 13 + 36 * c6[m] / r[m] ** 7) / np.maximum(s[m], 1e-30)
                dW_de = np.where(e[m] != 0, np.abs(c12[m] / r[m] ** 12 - c6[m] / r[m] ** 6) / e[m], 0.0)
                dW_ds = np.abs(12 * c12[m] / r[m] ** 12 - 6 * c6[m] / r[m] ** 6) / np.maximum(s[m], 1e-30)
            se[a, b] = (dg_de * du[m]).sum() + w_energy * 0.5 * dW_de.sum()
            ss[a, b] = (dg_ds * du[m]).sum() + w_energy * 0.5 * dW_ds.sum()
    return fs, qs, sq, ss, se
