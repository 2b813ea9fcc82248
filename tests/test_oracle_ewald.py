"""Pins for the oracle's Ewald / SPME reciprocal space (no GPU)."""
import math

import numpy as np
from scipy.special import erfc

from oracle import ewald
from oracle.forcefield import K_COUL
from paper_2002_07109_gb300.water import water_box


def _nacl(d=2.82, nc=2):
    pts, ch = [], []
    for i in range(2 * nc):
        for j in range(2 * nc):
            for k in range(2 * nc):
                pts.append([i * d, j * d, k * d])
                ch.append(1.0 if (i + j + k) % 2 == 0 else -1.0)
    L = 2 * nc * d
    return np.array(pts), np.array(ch), np.array([L, L, L])


def test_madelung_constant_of_rock_salt():
    """Direct (erfc) + reciprocal + self Ewald energy of a NaCl crystal equals
    -N/2 k M q^2 / d with the Madelung constant M = 1.747565 (textbook)."""
    d = 2.82
    q, ch, box = _nacl(d)
    beta, L = 0.9, box[0]
    dd = q[:, None, :] - q[None, :, :]
    dd -= L * np.rint(dd / L)
    r = np.sqrt((dd ** 2).sum(-1))
    iu = np.triu_indices(len(q), 1)
    rr, qq = r[iu], (ch[:, None] * ch[None, :])[iu]
    rc = L / 2 - 1e-9
    Ed = K_COUL * np.sum(np.where(rr < rc, qq * erfc(beta * rr) / rr, 0.0))
    Er, _ = ewald.recip_plain(q, ch, box, beta, 14)
    E = Ed + Er + ewald.self_energy(ch, beta)
    M = -E / (len(q) / 2) / (K_COUL / d)
    assert abs(M - 1.747565) < 2e-6


def test_spme_converges_to_plain_ewald():
    s = water_box(3, seed=1)
    beta = 0.35
    Ep, Gp = ewald.recip_plain(s.q, s.charge, s.box, beta, 12)
    Es, Gs = ewald.spme_recip(s.q, s.charge, s.box, beta, (48, 48, 48), 8)
    assert abs(Es - Ep) < 1e-7 * abs(Ep)
    assert np.abs(Gs - Gp).max() < 1e-6 * np.abs(Gp).max()
    # the production order (5) on a coarser grid stays close
    E5, G5 = ewald.spme_recip(s.q, s.charge, s.box, beta, (16, 16, 16), 5)
    assert abs(E5 - Ep) < 1e-3 * abs(Ep)
    assert np.abs(G5 - Gp).max() < 1e-2 * np.abs(Gp).max()


def test_recip_and_exclusion_gradients_by_finite_differences():
    s = water_box(2, seed=3)
    beta = 0.35
    pairs = ewald.molecule_pairs(s.molecule)
    rng = np.random.default_rng(0)
    h = 1e-5
    for fn in (lambda q: ewald.spme_recip(q, s.charge, s.box, beta, (20, 20, 20), 5),
               lambda q: ewald.recip_plain(q, s.charge, s.box, beta, 6),
               lambda q: ewald.exclusion(q, s.charge, pairs, beta, s.box)):
        E, G = fn(s.q)
        for a in rng.choice(s.n_atoms, 5, replace=False):
            for c in range(3):
                qp = s.q.copy(); qp[a, c] += h
                qm = s.q.copy(); qm[a, c] -= h
                fd = (fn(qp)[0] - fn(qm)[0]) / (2 * h)
                assert abs(fd - G[a, c]) < 1e-5 * max(1.0, abs(G[a, c])), (a, c, fd, G[a, c])


def test_bspline_partition_of_unity():
    x = np.linspace(0, 1, 101)
    for n in (4, 5, 6):
        tot = sum(ewald.bspline(x + t, n) for t in range(n))
        assert np.allclose(tot, 1.0, atol=1e-14)
        dtot = sum(ewald.bspline_deriv(x + t, n) for t in range(n))
        assert np.allclose(dtot, 0.0, atol=1e-13)


def _respa_setup(dt):
    from oracle.forcefield import Params
    from oracle.integrate import OracleMD, Topology
    s = water_box(3, seed=2)
    topo = Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    # no long-range jump part (chi = 0 inside r_c), no LJ, erfc(beta r_c) ~ 4e-7, no friction
    p = Params(r_on=100.0, r_off=100.0, r_cut=4.5, ewald_beta=0.8, box=s.box, lj_sigma=s.lj_sigma,
               lj_eps=0.0 * s.lj_eps, pme_grid=(16, 16, 16), pme_order=5)
    return OracleMD(s.q, s.v * 0.3, topo, p, seed=1, gamma=0.0, dt=dt, skin=0.5)


def test_bounce_respa_reduces_to_baoab_and_is_second_order():
    """BOUNCE-RESPA with m = 1 and no jump part is BAOAB with the reciprocal
    gradient in the kicks; with m = 2 its energy error is O(delta^2)."""
    a = _respa_setup(0.25)
    b = _respa_setup(0.25)
    a.run(20, "baoab")
    b.run(20, "bounce_respa", respa_m=1)
    assert np.allclose(a.q, b.q, rtol=0, atol=1e-10) and np.allclose(a.v, b.v, rtol=0, atol=1e-12)
    dev = []
    for dt in (0.25, 0.125):
        md = _respa_setup(dt)
        e0 = md.energies()
        t0 = e0["pot"] + e0["kin"]
        worst = 0.0
        for _ in range(6):
            md.run(int(round(2.5 / dt)) * 2, "bounce_respa", respa_m=2)
            e = md.energies()
            worst = max(worst, abs(e["pot"] + e["kin"] - t0))
        dev.append(worst)
    assert 2.5 < dev[0] / dev[1] < 6.0, dev
    assert md.proposals == 0


def test_extended_respa_with_one_inner_step_is_baoab():
    """With m = 1 and no jump part, the extended split kicks the same total
    gradient as BAOAB at the same positions."""
    a = _respa_setup(0.25)
    b = _respa_setup(0.25)
    a.run(12, "baoab")
    b.run(12, "bounce_respa_ext", respa_m=1)
    assert np.allclose(a.q, b.q, rtol=0, atol=1e-10) and np.allclose(a.v, b.v, rtol=0, atol=1e-12)


def test_respa1_with_one_intermediate_step_is_extended_respa():
    """With m2 = 1 the intermediate and outer kicks act at the same positions,
    so BOUNCE-RESPA1 is the extended BOUNCE-RESPA (up to the rounding of
    adding two kicks instead of their sum); with m = m2 = 1 it is BAOAB."""
    a = _respa_setup(0.25)
    b = _respa_setup(0.25)
    a.run(12, "bounce_respa_ext", respa_m=2)
    b.run(12, "bounce_respa1", respa_m=2, respa_m2=1)
    assert np.allclose(a.q, b.q, rtol=0, atol=1e-10) and np.allclose(a.v, b.v, rtol=0, atol=1e-12)
    c = _respa_setup(0.25)
    d = _respa_setup(0.25)
    c.run(8, "baoab")
    d.run(8, "bounce_respa1", respa_m=1, respa_m2=1)
    assert np.allclose(c.q, d.q, rtol=0, atol=1e-10) and np.allclose(c.v, d.v, rtol=0, atol=1e-12)


def test_respa1_is_second_order():
    """Energy error of BOUNCE-RESPA1 (m = 2, m2 = 2, no jump part, no
    friction) falls by about 4 when delta halves."""
    dev = []
    for dt in (0.25, 0.125):
        md = _respa_setup(dt)
        e0 = md.energies()
        t0 = e0["pot"] + e0["kin"]
        worst = 0.0
        for _ in range(4):
            md.run(int(round(2.0 / dt)) * 4, "bounce_respa1", respa_m=2, respa_m2=2)
            e = md.energies()
            worst = max(worst, abs(e["pot"] + e["kin"] - t0))
        dev.append(worst)
    assert 2.5 < dev[0] / dev[1] < 6.0, dev
