"""Jump-rate bounds (paper Sec. IV.A, last paragraphs; Sec. V first paragraph).

For a pair of types (a, b) the long-range gradient term is
F_ij = chi(r) W'_ab(r) (q_i - q_j)/r, so ||F_ij|| <= L_ab := sup_r |chi W'_ab|,
and the rate lambda_ij = beta max(0, v_i . F_ij) is bounded by
beta ||v_i|| L_ab.  The paper computes the sup numerically once (a 1-D
maximisation).  This project's reading (jump partners drawn uniformly over
all candidates of atom i, whatever their type) uses the row maximum
L*_a = max_b L_ab, which bounds every candidate of an atom of type a.

Method: a dense grid of 10^6 points on [r', R] (R = r_c, or r'' + 60 A with no
cutoff), then a bounded scalar refinement around the best grid point, then a
relative pad of 1e-6 so that round-off never makes the bound too small.

Per-type-pair bounds (Sec. V: the bound L may depend on the types of the two
particles).  pair_weights turns the table into the two-stage partner choice:
the type b of the partner is drawn with probability proportional to
n_ib Lq_ab, then the partner uniformly among the n_ib candidates of that
type.  Lq_ab = ceil(2^16 L_ab / L*_a) + 1 is an integer weight (0 where
L_ab = 0) so that the choice is exact integer arithmetic, and the bound it
stands for, Lt_ab = (Lq_ab L*_a) 2^-16 >= L_ab, is used in the acceptance.

Pins: closed form k |q_a q_b| / r''^2 for an indicator chi and bare Coulomb,
and a brute-force check that lambda <= lambda* on random pairs
(tests/test_oracle_bounds.py).
"""
import math
import numpy as np
from scipy.optimize import minimize_scalar

from .forcefield import chi, pair_dW

PAD = 1e-6


def sup_chi_dW(qa, qb, sig, eps, p, n_grid=1_000_000):
    """sup over r >= r' (r < r_c) of |chi(r) W'(r)| for one type pair."""
    lo = p.r_on if p.r_off > p.r_on else p.r_off
    hi = p.r_cut if math.isfinite(p.r_cut) else p.r_off + 60.0
    if not hi > lo:
        return 0.0
    r = np.linspace(lo, hi, n_grid)
    r = r[r < p.r_cut] if math.isfinite(p.r_cut) else r

    def f(x):
        return abs(float(chi(x, p.r_on, p.r_off) * pair_dW(x, qa, qb, sig, eps, p)))

    vals = np.abs(chi(r, p.r_on, p.r_off) * pair_dW(r, qa, qb, sig, eps, p))
    k = int(np.argmax(vals))
    best = float(vals[k])
    a = float(r[max(k - 2, 0)])
    b = float(r[min(k + 2, len(r) - 1)])
    if b > a:
        res = minimize_scalar(lambda x: -f(x), bounds=(a, b), method='bounded', options={'xatol': 1e-12})
        best = max(best, -float(res.fun))
    return best


def bound_table(charge, typ, n_types, lj_sigma, lj_eps, p):
    """L_ab (padded) for every type pair, and the row maxima L*_a.

    W'_ab is linear in the charge product, so with per-atom charges the sup
    over a type pair is reached at one of the four products of the types'
    extreme charges; all four are tried."""
    charge = np.asarray(charge, dtype=np.float64)
    typ = np.asarray(typ)
    T = int(n_types)
    L = np.zeros((T, T))
    ext = []
    for a in range(T):
        qa = charge[typ == a]
        ext.append((float(qa.min()), float(qa.max())) if len(qa) else (0.0, 0.0))
    for a in range(T):
        for b in range(T):
            best = 0.0
            charged = getattr(p, "coulomb_jumps", True)
            for qa in (set(ext[a]) if charged else {0.0}):
                for qb in (set(ext[b]) if charged else {0.0}):
                    best = max(best, sup_chi_dW(qa, qb, lj_sigma[a, b], lj_eps[a, b], p))
            L[a, b] = best * (1.0 + PAD)
    return L, L.max(axis=1)


QBITS = 16


def pair_weights(L, Lstar):
    """(Lq, Lt): integer weights of the two-stage partner choice and the
    bounds they stand for, Lt_ab = (Lq_ab L*_a) 2^-16 >= L_ab."""
    L = np.asarray(L, dtype=np.float64)
    T = L.shape[0]
    Lq = np.zeros((T, T), dtype=np.int64)
    Lt = np.zeros((T, T))
    for a in range(T):
        for b in range(T):
            if L[a, b] > 0.0:
                Lq[a, b] = int(math.ceil(L[a, b] / Lstar[a] * float(1 << QBITS))) + 1
                Lt[a, b] = (float(Lq[a, b]) * Lstar[a]) * 2.0 ** -QBITS
    return Lq, Lt
