"""Pins for the oracle's force field, bounds and neighbour rows (no GPU)."""
import math

import numpy as np
import pytest
from scipy.special import erfc

from oracle import forcefield as ff
from oracle.bounds import bound_table
from oracle.neighbors import rows, rows_cell_list, needs_rebuild, to_pairs
from paper_2002_07109_gb300.water import water_droplet, water_box


def _params(s, **kw):
    return ff.Params(lj_sigma=s.lj_sigma, lj_eps=s.lj_eps, box=s.box, **kw)


def _total_energy(s, q, p, ii, jj):
    ec, el = ff.pair_energies(q, s.charge, s.type, ii, jj, p)
    eb, ea = ff.bonded_energies(q, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0, p.box)
    return ec + el + eb + ea


@pytest.mark.parametrize("kind", ["droplet", "box"])
def test_full_gradient_is_energy_derivative(kind):
    """Central finite differences (h = 1e-4 A) of E_pot match the analytic
    full gradient (pairs + bonds + angles)."""
    if kind == "droplet":
        s = water_droplet(3, seed=2)
        p = _params(s, r_on=4.0, r_off=5.0, r_cut=math.inf)
    else:
        s = water_box(4, seed=2)
        p = _params(s, r_on=4.0, r_off=5.0, r_cut=6.0, ewald_beta=0.35)
    rng = np.random.default_rng(0)
    q = s.q + rng.normal(scale=0.05, size=s.q.shape)
    ii, jj = ff.all_pairs(s.molecule)
    g = (ff.pair_gradients(q, s.charge, s.type, ii, jj, p, "full")
         + ff.bonded_gradients(q, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0, p.box))
    h = 1e-4
    # the truncated energy jumps at r_c: skip atoms with a pair within 2h of it
    d = ff.displacement(q[ii], q[jj], p.box)
    r = np.sqrt((d * d).sum(1))
    near = np.unique(ii[np.abs(r - p.r_cut) < 2 * h]) if math.isfinite(p.r_cut) else []
    pool = np.setdiff1d(np.arange(s.n_atoms), near)
    for a in rng.choice(pool, 12, replace=False):
        for c in range(3):
            qp = q.copy(); qp[a, c] += h
            qm = q.copy(); qm[a, c] -= h
            fd = (_total_energy(s, qp, p, ii, jj) - _total_energy(s, qm, p, ii, jj)) / (2 * h)
            assert abs(fd - g[a, c]) < 1e-6 * max(1.0, abs(g[a, c])) + 2e-6, (a, c, fd, g[a, c])


def test_short_plus_long_is_full_and_newton3():
    s = water_droplet(3, seed=4)
    p = _params(s, r_on=4.0, r_off=5.0, r_cut=math.inf)
    ii, jj = ff.all_pairs(s.molecule)
    full = ff.pair_gradients(s.q, s.charge, s.type, ii, jj, p, "full")
    short = ff.pair_gradients(s.q, s.charge, s.type, ii, jj, p, "short")
    long = ff.pair_gradients(s.q, s.charge, s.type, ii, jj, p, "long")
    assert np.allclose(short + long, full, rtol=1e-12, atol=1e-12)
    # translation invariance: the gradient sums to zero
    assert np.abs(full.sum(0)).max() < 1e-9
    b = ff.bonded_gradients(s.q, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    assert np.abs(b.sum(0)).max() < 1e-9


def test_single_pair_closed_forms():
    p = ff.Params(r_on=4.0, r_off=5.0, lj_sigma=np.array([[3.15]]), lj_eps=np.array([[0.152]]))
    r = 3.7
    # Coulomb + LJ derivative written out by hand
    sr6 = (3.15 / r) ** 6
    want = -332.063713 * 0.834 * 0.834 / r ** 2 + 4 * 0.152 * (-12 * sr6 * sr6 + 6 * sr6) / r
    assert abs(ff.pair_dW(r, -0.834, -0.834, 3.15, 0.152, p) - want) < 1e-12
    pe = ff.Params(r_on=4.0, r_off=5.0, ewald_beta=0.35, r_cut=9.0)
    b = 0.35
    want = -332.063713 * (erfc(b * r) / r ** 2 + 2 * b / math.sqrt(math.pi) * math.exp(-(b * r) ** 2) / r)
    assert abs(ff.pair_dW(r, 1.0, 1.0, 0.0, 0.0, pe) - want) < 1e-12
    assert ff.pair_dW(9.0, 1.0, 1.0, 0.0, 0.0, pe) == 0.0        # truncated at r_c (strict)
    # switching function: endpoints, midpoint, monotone
    assert ff.chi(4.0, 4.0, 5.0) == 0.0 and ff.chi(5.0, 4.0, 5.0) == 1.0
    assert abs(ff.chi(4.5, 4.0, 5.0) - 0.5) < 1e-15
    x = np.linspace(3, 6, 1001)
    assert np.all(np.diff(ff.chi(x, 4.0, 5.0)) >= 0)
    assert ff.chi(4.99, 5.0, 5.0) == 0.0 and ff.chi(5.0, 5.0, 5.0) == 1.0


def test_bound_indicator_closed_form():
    """For an indicator switch at r'' and bare Coulomb, sup |chi W'| is
    k |q_a q_b| / r''^2 (Sec. IV.A bounds chi by that indicator)."""
    typ = np.array([0, 1])
    charge = np.array([-0.834, 0.417])
    z = np.zeros((2, 2))
    p = ff.Params(r_on=5.0, r_off=5.0, lj_sigma=z, lj_eps=z)
    L, Ls = bound_table(charge, typ, 2, z, z, p)
    k = 332.063713
    want = np.array([[k * 0.834 ** 2, k * 0.834 * 0.417], [k * 0.834 * 0.417, k * 0.417 ** 2]]) / 25.0
    assert np.allclose(L, want * (1 + 1e-6), rtol=1e-9)
    assert np.allclose(Ls, L.max(1))


@pytest.mark.parametrize("ewald", [0.0, 0.35])
def test_bound_covers_every_pair(ewald):
    """lambda <= lambda*: ||F_ij|| <= L*_{t_i} for random pair geometries."""
    s = water_droplet(2, seed=1)
    p = _params(s, r_on=4.0, r_off=5.0, r_cut=9.0 if ewald else math.inf, ewald_beta=ewald)
    L, Ls = bound_table(s.charge, s.type, 2, s.lj_sigma, s.lj_eps, p)
    rng = np.random.default_rng(5)
    r = rng.uniform(0.5, 20.0, 200000)
    for a in (0, 1):
        for b in (0, 1):
            qa = s.charge[s.type == a][0]
            qb = s.charge[s.type == b][0]
            g = np.abs(ff.chi(r, p.r_on, p.r_off) * ff.pair_dW(r, qa, qb, s.lj_sigma[a, b], s.lj_eps[a, b], p))
            assert g.max() <= L[a, b] <= Ls[a]
            # and the bound is tight (within the pad plus grid resolution)
            assert g.max() > L[a, b] * (1 - 1e-3)


@pytest.mark.parametrize("kind", ["droplet", "box"])
def test_rows_brute_force_equals_cell_list(kind):
    rng = np.random.default_rng(3)
    if kind == "droplet":
        s = water_droplet(5, seed=3)
        box = None
    else:
        s = water_box(6, seed=3)
        box = s.box
    q = s.q + rng.normal(scale=0.3, size=s.q.shape)
    a = rows(q, s.molecule, 6.5, box)
    b = rows_cell_list(q, s.molecule, 6.5, box)
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
        assert np.all(np.diff(x) > 0)


def test_rows_no_cutoff_and_exclusions():
    s = water_droplet(2, seed=0)
    r = rows(s.q, s.molecule, math.inf)
    for i, row in enumerate(r):
        assert len(row) == s.n_atoms - 3
        assert np.all(s.molecule[row] != s.molecule[i])
    ii, jj = to_pairs(r)
    assert len(ii) == s.n_atoms * (s.n_atoms - 3)


def test_rebuild_rule():
    q = np.zeros((4, 3))
    q2 = q.copy()
    q2[2, 0] = 0.5
    assert not needs_rebuild(q2, q, 1.0)          # exactly skin/2 does not trigger
    q2[2, 0] = 0.5000001
    assert needs_rebuild(q2, q, 1.0)
    assert needs_rebuild(q, None, 1.0)
