"""Pins for the oracle's force-matching gradients (no GPU): central finite
differences (h = 1e-4) of the loss with respect to positions, per-type
charges, sigma and eps."""
import math

import numpy as np

from oracle.diff import force_matching_loss
from paper_2002_07109_gb300.water import water_box


def _setup():
    s = water_box(3, seed=5)
    qt = np.array([-0.834, 0.417])
    sig = np.array([[3.15, 1.8], [1.8, 1.2]])        # nonzero H terms exercise every table entry
    eps = np.array([[0.152, 0.05], [0.05, 0.02]])
    F_t = np.random.default_rng(0).normal(scale=5.0, size=s.q.shape)
    return s, qt, sig, eps, F_t


def _L(s, q, qt, sig, eps, F_t):
    return force_matching_loss(q, s.type, s.molecule, qt, sig, eps, F_t, 4.5, 0.35, s.box, w_energy=0.3)[0]


def test_gradients_match_central_differences():
    s, qt, sig, eps, F_t = _setup()
    L, F, E, gq, gqt, gs, ge = force_matching_loss(s.q, s.type, s.molecule, qt, sig, eps, F_t, 4.5, 0.35, s.box,
                                                   w_energy=0.3)
    h = 1e-4
    for a in (0, 5, 17):
        for c in range(3):
            qp = s.q.copy(); qp[a, c] += h
            qm = s.q.copy(); qm[a, c] -= h
            fd = (_L(s, qp, qt, sig, eps, F_t) - _L(s, qm, qt, sig, eps, F_t)) / (2 * h)
            assert abs(fd - gq[a, c]) < 1e-5 * max(1.0, abs(gq[a, c])), (a, c, fd, gq[a, c])
    for t in range(2):
        p = qt.copy(); p[t] += h
        m = qt.copy(); m[t] -= h
        fd = (_L(s, s.q, p, sig, eps, F_t) - _L(s, s.q, m, sig, eps, F_t)) / (2 * h)
        assert abs(fd - gqt[t]) < 1e-5 * max(1.0, abs(gqt[t]))
    for (a, b) in ((0, 0), (0, 1), (1, 1)):
        for tab, g in ((sig, gs), (eps, ge)):
            p = tab.copy(); p[a, b] += h; p[b, a] = p[a, b]
            m = tab.copy(); m[a, b] -= h; m[b, a] = m[a, b]
            args_p = (p, eps) if tab is sig else (sig, p)
            args_m = (m, eps) if tab is sig else (sig, m)
            fd = (_L(s, s.q, qt, *args_p, F_t) - _L(s, s.q, qt, *args_m, F_t)) / (2 * h)
            assert abs(fd - g[a, b]) < 2e-5 * max(1.0, abs(g[a, b])), (a, b, fd, g[a, b])
            assert g[a, b] == g[b, a]


def test_forces_are_minus_energy_gradient():
    s, qt, sig, eps, F_t = _setup()
    _, F, E, *_ = force_matching_loss(s.q, s.type, s.molecule, qt, sig, eps, F_t, 4.5, 0.35, s.box)
    h = 1e-5
    for a in (1, 9):
        for c in range(3):
            qp = s.q.copy(); qp[a, c] += h
            qm = s.q.copy(); qm[a, c] -= h
            Ep = force_matching_loss(qp, s.type, s.molecule, qt, sig, eps, F_t, 4.5, 0.35, s.box)[2]
            Em = force_matching_loss(qm, s.type, s.molecule, qt, sig, eps, F_t, 4.5, 0.35, s.box)[2]
            assert abs(-(Ep - Em) / (2 * h) - F[a, c]) < 1e-5 * max(1.0, abs(F[a, c]))
