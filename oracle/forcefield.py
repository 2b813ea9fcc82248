"""Force field and the short/long split of the paper, in FP64.

Sign convention (paper Sec. II.A and Eq. Lambda_i): the vector fields F_i the
paper splits are terms of the GRADIENT of E_pot, grad E_pot = sum_i F_i, not
physical forces.  Everything here returns gradients; the B step subtracts
them.  Functions:

  pair_dW        W'(r) of one pair: Coulomb k qa qb / r (droplets, Sec. V) or
                 the Ewald direct part k qa qb erfc(beta r) / r (periodic
                 boxes, Sec. V), plus 4 eps ((sigma/r)^12 - (sigma/r)^6).
                 Truncated at r_c (W = W' = 0 for r >= r_c).
  chi            smooth switching function, 0 below r', 1 above r''
                 (Sec. IV.A); this project's reading: quintic smoothstep.
  pair_gradients per-atom sum over directed pairs of
                 part="full": W'(r) d/r, part="short": (1 - chi) W'(r) d/r
                 (F_shortVdW and F_shortdir of Sec. IV.A / V),
                 part="long": chi W'(r) d/r (the F_ij of Sec. IV.A).
  bonded_*       harmonic bonds k (r - r0)^2 and angles k (theta - theta0)^2.
  energies       E_coul, E_lj, E_bond, E_angle over unordered pairs i < j.

Pins: finite differences of the energies, Newton's third law, the identity
full = short + long, closed-form single-pair values (tests/test_oracle_ff.py).
"""
from dataclasses import dataclass
import math
import numpy as np
from scipy.special import erfc

K_COUL = 332.063713        # kcal A / (mol e^2)
KB = 0.0019872041          # kcal / (mol K)
ACCEL = 4.184e-4           # (kcal/mol/A)/(g/mol) -> A/fs^2


@dataclass
class Params:
    r_on: float = 4.0          # r'  (chi = 0 below)
    r_off: float = 5.0         # r'' (chi = 1 above)
    r_cut: float = math.inf    # pair cutoff, inf = none (droplets)
    ewald_beta: float = 0.0    # 0 = bare Coulomb; > 0 = Ewald direct erfc
    box: np.ndarray = None     # periodic edges (3,), None = open
    lj_sigma: np.ndarray = None
    lj_eps: np.ndarray = None
    pme_grid: tuple = None     # SPME grid (K1, K2, K3) for periodic Ewald, None = no reciprocal part
    pme_order: int = 5         # B-spline order
    coulomb_jumps: bool = True # False: Coulomb wholly in F_0, only the LJ part is split (Sec. IV.A first example)


def chi(r, r_on, r_off):
    """Switching function chi(r) with chi = 0 for r <= r', 1 for r >= r''.

    Reading of the paper (its form is given in a supplement that is not
    available): chi(s) = 10 s^3 - 15 s^4 + 6 s^5 with s = (r - r')/(r'' - r').
    With r' = r'' it is the indicator of [r'', inf)."""
    r = np.asarray(r, dtype=np.float64)
    if not r_off > r_on:
        return (r >= r_off).astype(np.float64)
    s = np.clip((r - r_on) / (r_off - r_on), 0.0, 1.0)
    return s * s * s * (10.0 + s * (-15.0 + 6.0 * s))


def pair_W(r, qa, qb, sig, eps, p):
    """Pair energy W(r) (unsplit), truncated at r_cut."""
    r = np.asarray(r, dtype=np.float64)
    if p.ewald_beta > 0:
        coul = K_COUL * qa * qb * erfc(p.ewald_beta * r) / r
    else:
        coul = K_COUL * qa * qb / r
    with np.errstate(divide='ignore', invalid='ignore'):
        sr6 = np.where(eps != 0, (sig / r) ** 6, 0.0)
    lj = 4.0 * eps * (sr6 * sr6 - sr6)
    return np.where(r < p.r_cut, coul + lj, 0.0)


def pair_dW(r, qa, qb, sig, eps, p):
    """dW/dr of one pair, truncated at r_cut."""
    r = np.asarray(r, dtype=np.float64)
    if p.ewald_beta > 0:
        b = p.ewald_beta
        coul = -K_COUL * qa * qb * (erfc(b * r) / (r * r) + 2.0 * b / math.sqrt(math.pi) * np.exp(-b * b * r * r) / r)
    else:
        coul = -K_COUL * qa * qb / (r * r)
    with np.errstate(divide='ignore', invalid='ignore'):
        sr6 = np.where(eps != 0, (sig / r) ** 6, 0.0)
    lj = -24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r
    return np.where(r < p.r_cut, coul + lj, 0.0)


def displacement(qi, qj, box):
    """q_i - q_j, minimum image when box is given: d - L rint(d / L)."""
    d = qi - qj
    if box is not None:
        L = np.asarray(box, dtype=np.float64)
        d = d - L * np.rint(d / L)
    return d


def _uncut(p):
    """The same parameters without the cutoff (callers apply inside_cut)."""
    return Params(r_on=p.r_on, r_off=p.r_off, r_cut=math.inf, ewald_beta=p.ewald_beta, box=p.box,
                  lj_sigma=p.lj_sigma, lj_eps=p.lj_eps, pme_grid=p.pme_grid, pme_order=p.pme_order,
                  coulomb_jumps=p.coulomb_jumps)


def split_dW(r, qa, qb, sig, eps, p):
    """(part of W' switched by chi, part always in F_0): the whole W' and 0,
    or the LJ part and the Coulomb part when Coulomb stays in F_0."""
    if p.coulomb_jumps:
        return pair_dW(r, qa, qb, sig, eps, p), 0.0
    lj_only = pair_dW(r, 0.0, 0.0, sig, eps, p)
    return lj_only, pair_dW(r, qa, qb, sig, eps, p) - lj_only


def all_pairs(mol):
    """Directed pairs (i, j), j != i, different molecules, ascending i then j."""
    n = len(mol)
    ii, jj = np.nonzero(mol[:, None] != mol[None, :])
    return ii.astype(np.int64), jj.astype(np.int64)


def r2_of(d):
    """(dx*dx + dy*dy) + dz*dz in FP64 round-to-nearest."""
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def inside_cut(r2, p):
    """Pair cutoff test r^2 < r_c^2 (every pair sum uses this exact form)."""
    return r2 < p.r_cut * p.r_cut if math.isfinite(p.r_cut) else np.ones(np.shape(r2), dtype=bool)


def pair_terms(q, charge, typ, ii, jj, p):
    """r, d and the pair parameters for directed pairs (ii, jj)."""
    d = displacement(q[ii], q[jj], p.box)
    r = np.sqrt(r2_of(d))
    ti, tj = typ[ii], typ[jj]
    sig = p.lj_sigma[ti, tj]
    eps = p.lj_eps[ti, tj]
    return d, r, charge[ii], charge[jj], sig, eps


def pair_gradients(q, charge, typ, ii, jj, p, part="full"):
    """Sum over the directed pairs (i, j) in (ii, jj) of the gradient of
    W(|q_i - q_j|) with respect to q_i, times 1 (full), 1 - chi (short) or
    chi (long).  Returns (N, 3)."""
    n = q.shape[0]
    g = np.zeros((n, 3))
    if len(ii) == 0:
        return g
    d, r, qa, qb, sig, eps = pair_terms(q, charge, typ, ii, jj, p)
    inside = inside_cut(r2_of(d), p)
    sw, fixed = split_dW(r, qa, qb, sig, eps, _uncut(p))
    if part == "short":
        w = sw * (1.0 - chi(r, p.r_on, p.r_off)) + fixed
    elif part == "long":
        w = sw * chi(r, p.r_on, p.r_off)
    else:
        w = sw + fixed
    w = np.where(inside, w, 0.0)
    contrib = (w / r)[:, None] * d
    np.add.at(g, ii, contrib)
    return g


def pair_gradient_magnitudes(q, charge, typ, ii, jj, p, part="full"):
    """Per-atom sum over the directed pairs of the magnitude of each pair's
    gradient term: the scale of the rounding error of any floating-point
    evaluation of the sum (forward error bound of summation)."""
    n = q.shape[0]
    m = np.zeros(n)
    if len(ii) == 0:
        return m
    d, r, qa, qb, sig, eps = pair_terms(q, charge, typ, ii, jj, p)
    inside = inside_cut(r2_of(d), p)
    sw, fixed = split_dW(r, qa, qb, sig, eps, _uncut(p))
    c = chi(r, p.r_on, p.r_off)
    if part == "short":
        w = np.abs(sw * (1.0 - c)) + np.abs(fixed)
    elif part == "long":
        w = np.abs(sw * c)
    else:
        w = np.abs(sw) + np.abs(fixed)
    np.add.at(m, ii, np.where(inside, w, 0.0))
    return m


def pair_gradient_one(qi, qj, qa, qb, sig, eps, p, part="long"):
    """Gradient of one pair with respect to q_i (vectorised over rows)."""
    d = displacement(qi, qj, p.box)
    r2 = r2_of(d)
    r = np.sqrt(r2)
    with np.errstate(divide='ignore', invalid='ignore'):
        sw, fixed = split_dW(r, qa, qb, sig, eps, _uncut(p))
        c = chi(r, p.r_on, p.r_off)
        if part == "long":
            w = sw * c
        elif part == "short":
            w = sw * (1.0 - c) + fixed
        else:
            w = sw + fixed
        w = np.where(inside_cut(r2, p), w, 0.0)
    with np.errstate(divide='ignore', invalid='ignore'):
        f = np.where(r > 0, w / r, 0.0)
    return f[..., None] * d


def bonded_gradients(q, bonds, bond_k_r0, angles, angle_k_t0, box=None):
    """Gradient of sum k_b (r - r0)^2 + sum k_t (theta - theta0)^2."""
    g = np.zeros_like(q)
    if len(bonds):
        a, b = bonds[:, 0], bonds[:, 1]
        d = displacement(q[a], q[b], box)
        r = np.sqrt((d * d).sum(1))
        k, r0 = bond_k_r0[:, 0], bond_k_r0[:, 1]
        c = (2.0 * k * (r - r0) / r)[:, None] * d
        np.add.at(g, a, c)
        np.add.at(g, b, -c)
    if len(angles):
        a, b, c = angles[:, 0], angles[:, 1], angles[:, 2]
        u = displacement(q[a], q[b], box)
        w = displacement(q[c], q[b], box)
        nu = np.sqrt((u * u).sum(1))
        nw = np.sqrt((w * w).sum(1))
        cos = (u * w).sum(1) / (nu * nw)
        cos = np.clip(cos, -1.0, 1.0)
        th = np.arccos(cos)
        sin = np.sqrt(1.0 - cos * cos)
        k, t0 = angle_k_t0[:, 0], angle_k_t0[:, 1]
        dE = 2.0 * k * (th - t0)
        # d theta / d u = -(w/(|u||w|) - cos u/|u|^2) / sin
        du = -(w / (nu * nw)[:, None] - (cos / (nu * nu))[:, None] * u) / sin[:, None]
        dw = -(u / (nu * nw)[:, None] - (cos / (nw * nw))[:, None] * w) / sin[:, None]
        ga = dE[:, None] * du
        gc = dE[:, None] * dw
        np.add.at(g, a, ga)
        np.add.at(g, c, gc)
        np.add.at(g, b, -(ga + gc))
    return g


def bonded_gradient_magnitudes(q, bonds, bond_k_r0, angles, angle_k_t0, box=None):
    """Per-atom sum of the magnitudes of the bonded gradient terms."""
    m = np.zeros(q.shape[0])
    if len(bonds):
        a, b = bonds[:, 0], bonds[:, 1]
        d = displacement(q[a], q[b], box)
        r = np.sqrt((d * d).sum(1))
        c = np.abs(2.0 * bond_k_r0[:, 0] * (r - bond_k_r0[:, 1]))
        np.add.at(m, a, c)
        np.add.at(m, b, c)
    if len(angles):
        a, b, c = angles[:, 0], angles[:, 1], angles[:, 2]
        u = displacement(q[a], q[b], box)
        w = displacement(q[c], q[b], box)
        nu = np.sqrt((u * u).sum(1))
        nw = np.sqrt((w * w).sum(1))
        cos = np.clip((u * w).sum(1) / (nu * nw), -1.0, 1.0)
        sin = np.sqrt(1.0 - cos * cos)
        dE = 2.0 * angle_k_t0[:, 0] * (np.arccos(cos) - angle_k_t0[:, 1])
        du = -(w / (nu * nw)[:, None] - (cos / (nu * nu))[:, None] * u) / sin[:, None]
        dw = -(u / (nu * nw)[:, None] - (cos / (nw * nw))[:, None] * w) / sin[:, None]
        ga = dE[:, None] * du
        gc = dE[:, None] * dw
        np.add.at(m, a, np.linalg.norm(ga, axis=1))
        np.add.at(m, c, np.linalg.norm(gc, axis=1))
        np.add.at(m, b, np.linalg.norm(ga + gc, axis=1))
    return m


def bonded_energies(q, bonds, bond_k_r0, angles, angle_k_t0, box=None):
    eb = 0.0
    ea = 0.0
    if len(bonds):
        d = displacement(q[bonds[:, 0]], q[bonds[:, 1]], box)
        r = np.sqrt((d * d).sum(1))
        eb = float((bond_k_r0[:, 0] * (r - bond_k_r0[:, 1]) ** 2).sum())
    if len(angles):
        u = displacement(q[angles[:, 0]], q[angles[:, 1]], box)
        w = displacement(q[angles[:, 2]], q[angles[:, 1]], box)
        cos = (u * w).sum(1) / np.sqrt((u * u).sum(1) * (w * w).sum(1))
        th = np.arccos(np.clip(cos, -1.0, 1.0))
        ea = float((angle_k_t0[:, 0] * (th - angle_k_t0[:, 1]) ** 2).sum())
    return eb, ea


def pair_energies(q, charge, typ, ii, jj, p):
    """(E_coul, E_lj) over the unordered pairs i < j among (ii, jj)."""
    keep = ii < jj
    ii, jj = ii[keep], jj[keep]
    if len(ii) == 0:
        return 0.0, 0.0
    d, r, qa, qb, sig, eps = pair_terms(q, charge, typ, ii, jj, p)
    inside = inside_cut(r2_of(d), p)
    if p.ewald_beta > 0:
        coul = K_COUL * qa * qb * erfc(p.ewald_beta * r) / r
    else:
        coul = K_COUL * qa * qb / r
    sr6 = np.where(eps != 0, (sig / r) ** 6, 0.0)
    lj = 4.0 * eps * (sr6 * sr6 - sr6)
    return float(np.where(inside, coul, 0.0).sum()), float(np.where(inside, lj, 0.0).sum())


def pair_energy_magnitudes(q, charge, typ, ii, jj, p):
    """(sum |Coulomb term|, sum |LJ term|) over the unordered pairs i < j."""
    keep = ii < jj
    ii, jj = ii[keep], jj[keep]
    if len(ii) == 0:
        return 0.0, 0.0
    d, r, qa, qb, sig, eps = pair_terms(q, charge, typ, ii, jj, p)
    inside = inside_cut(r2_of(d), p)
    if p.ewald_beta > 0:
        coul = K_COUL * qa * qb * erfc(p.ewald_beta * r) / r
    else:
        coul = K_COUL * qa * qb / r
    sr6 = np.where(eps != 0, (sig / r) ** 6, 0.0)
    lj = 4.0 * eps * (sr6 * sr6 - sr6)
    return float(np.abs(np.where(inside, coul, 0.0)).sum()), float(np.abs(np.where(inside, lj, 0.0)).sum())


def kinetic_energy(v, mass):
    """sum 1/2 m v^2 in kcal/mol (v in A/fs, m in g/mol)."""
    return float(0.5 * (mass[:, None] * v * v).sum() / ACCEL)
