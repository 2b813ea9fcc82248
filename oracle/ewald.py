"""Ewald electrostatics for periodic boxes (paper Sec. V: the Coulomb energy
is split into a reciprocal part, computed in Fourier space, and a direct
part k q_i q_j erfc(beta r)/r that BOUNCE splits again into F_0 and jumps).

Functions (FP64, orthorhombic box, kcal/mol, A):
  recip_plain      reciprocal energy and gradient by the textbook k-space sum
                   E = k/(2 pi V) sum_{m != 0} exp(-pi^2 m^2/beta^2)/m^2 |S(m)|^2,
                   S(m) = sum_j q_j exp(2 pi i m.r_j), m = (n1/L1, n2/L2, n3/L3).
  self_energy      -k beta/sqrt(pi) sum_j q_j^2.
  exclusion        -k sum_{excluded i<j} q_i q_j erf(beta r)/r and its gradient:
                   removes the reciprocal-space interaction of pairs (here:
                   atoms of one molecule) that the direct sum skips.
  spme_recip       smooth particle-mesh Ewald reciprocal energy and gradient
                   (Essmann, Perera, Berkowitz, Darden, Lee, Pedersen, J. Chem.
                   Phys. 103, 8577 (1995)): cardinal B-splines of order n spread
                   the charges on a K1 x K2 x K3 grid, E = 1/2 sum_m B(m) C(m)
                   |F(Q)(m)|^2, the gradient from the convolution theta * Q.

Pins: the NaCl Madelung constant 1.747565 from direct + reciprocal + self
(textbook special case); SPME converges to the plain k-space sum; gradients
against central finite differences (tests/test_oracle_ewald.py).
"""
import math

import numpy as np
from scipy.special import erf

from .forcefield import K_COUL


def self_energy(charge, beta):
    return -K_COUL * beta / math.sqrt(math.pi) * float(np.sum(np.asarray(charge) ** 2))


def _mvecs(box, kmax):
    n = np.arange(-kmax, kmax + 1)
    N = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3)
    N = N[np.any(N != 0, axis=1)]
    return N / np.asarray(box, dtype=np.float64)


def recip_plain(q, charge, box, beta, kmax):
    """(energy, gradient (N, 3)) of the reciprocal Ewald part by direct k-sum."""
    q = np.asarray(q, dtype=np.float64)
    charge = np.asarray(charge, dtype=np.float64)
    V = float(np.prod(box))
    M = _mvecs(box, kmax)
    m2 = (M * M).sum(1)
    f = np.exp(-math.pi ** 2 * m2 / beta ** 2) / m2
    E = 0.0
    G = np.zeros_like(q)
    for s in range(0, len(M), 2048):
        Ms, fs = M[s:s + 2048], f[s:s + 2048]
        th = 2.0 * math.pi * q @ Ms.T                      # (N, nm)
        c, sn = np.cos(th), np.sin(th)
        Sre = charge @ c
        Sim = charge @ sn
        E += float((fs * (Sre * Sre + Sim * Sim)).sum())
        # d|S|^2/dr_j = -4 pi q_j m Im(conj(S) e^{i th_j})
        im = Sre[None, :] * sn - Sim[None, :] * c            # Im(conj(S) e^{i th})
        G += -4.0 * math.pi * charge[:, None] * ((fs[None, :] * im) @ Ms)
    pref = K_COUL / (2.0 * math.pi * V)
    return pref * E, pref * G


def exclusion(q, charge, pairs, beta, box=None):
    """-k sum over excluded pairs of q_i q_j erf(beta r)/r, and its gradient."""
    q = np.asarray(q, dtype=np.float64)
    G = np.zeros_like(q)
    if len(pairs) == 0:
        return 0.0, G
    i, j = pairs[:, 0], pairs[:, 1]
    d = q[i] - q[j]
    if box is not None:
        L = np.asarray(box, dtype=np.float64)
        d = d - L * np.rint(d / L)
    r = np.sqrt((d * d).sum(1))
    qq = charge[i] * charge[j]
    E = -K_COUL * float((qq * erf(beta * r) / r).sum())
    # d/dr [erf(b r)/r] = 2b/sqrt(pi) exp(-b^2 r^2)/r - erf(b r)/r^2
    dw = -K_COUL * qq * (2.0 * beta / math.sqrt(math.pi) * np.exp(-beta * beta * r * r) / r - erf(beta * r) / (r * r))
    c = (dw / r)[:, None] * d
    np.add.at(G, i, c)
    np.add.at(G, j, -c)
    return E, G


def molecule_pairs(mol):
    """Unordered pairs of distinct atoms sharing a molecule id."""
    mol = np.asarray(mol)
    out = []
    for m in np.unique(mol):
        idx = np.nonzero(mol == m)[0]
        for a in range(len(idx)):
            for b in range(a + 1, len(idx)):
                out.append((idx[a], idx[b]))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def bspline(x, n):
    """Cardinal B-spline M_n(x) (support [0, n]) by the recursion
    M_n(x) = x/(n-1) M_{n-1}(x) + (n-x)/(n-1) M_{n-1}(x-1), M_2(x) = 1 - |x-1|."""
    x = np.asarray(x, dtype=np.float64)
    if n == 2:
        return np.where((x >= 0) & (x <= 2), 1.0 - np.abs(x - 1.0), 0.0)
    return (x * bspline(x, n - 1) + (n - x) * bspline(x - 1.0, n - 1)) / (n - 1)


def bspline_deriv(x, n):
    """dM_n/dx = M_{n-1}(x) - M_{n-1}(x - 1)."""
    return bspline(x, n - 1) - bspline(np.asarray(x) - 1.0, n - 1)


def _bmod2(K, n):
    """|b(m)|^2 = 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K)|^2.

    For odd n the sum vanishes at the Nyquist index m = K/2; there |b|^2 is
    taken as the mean of its two neighbours (this project's reading; C(m)
    is negligible at that frequency for any usable grid)."""
    m = np.arange(K)
    k = np.arange(n - 1)
    w = bspline(k + 1.0, n)
    s = np.abs((w[None, :] * np.exp(2j * math.pi * np.outer(m, k) / K)).sum(1)) ** 2
    out = np.empty(K)
    ok = s > 1e-7
    out[ok] = 1.0 / s[ok]
    for j in np.nonzero(~ok)[0]:
        out[j] = 0.5 * (1.0 / s[(j - 1) % K] + 1.0 / s[(j + 1) % K])
    return out


def spme_influence(box, beta, grid, order):
    """B(m) C(m) on the grid (m = 0 term zero), C = exp(-pi^2 m^2/beta^2)/(pi V m^2)."""
    K1, K2, K3 = grid
    L = np.asarray(box, dtype=np.float64)
    V = float(np.prod(L))

    def freq(K, Lx):
        m = np.arange(K)
        return np.where(m <= K // 2, m, m - K) / Lx

    f1, f2, f3 = freq(K1, L[0]), freq(K2, L[1]), freq(K3, L[2])
    m2 = f1[:, None, None] ** 2 + f2[None, :, None] ** 2 + f3[None, None, :] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.where(m2 > 0, np.exp(-math.pi ** 2 * m2 / beta ** 2) / (math.pi * V * m2), 0.0)
    B = _bmod2(K1, order)[:, None, None] * _bmod2(K2, order)[None, :, None] * _bmod2(K3, order)[None, None, :]
    return B * C


def spme_recip(q, charge, box, beta, grid, order):
    """(energy, gradient (N, 3)) of the reciprocal Ewald part by SPME."""
    q = np.asarray(q, dtype=np.float64)
    charge = np.asarray(charge, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    K = np.asarray(grid, dtype=np.int64)
    n = order
    u = (q / L - np.floor(q / L)) * K                    # scaled fractional coordinates in [0, K)
    fl = np.floor(u).astype(np.int64)
    fr = u - fl
    t = np.arange(n)
    # grid points k = fl - t with weights M_n(fr + t), derivative M_n'(fr + t)
    idx = [(fl[:, d][:, None] - t[None, :]) % K[d] for d in range(3)]
    w = [bspline(fr[:, d][:, None] + t[None, :], n) for d in range(3)]
    dw = [bspline_deriv(fr[:, d][:, None] + t[None, :], n) for d in range(3)]
    Q = np.zeros(tuple(K))
    for a in range(n):
        for b in range(n):
            wab = charge * w[0][:, a] * w[1][:, b]
            for c in range(n):
                np.add.at(Q, (idx[0][:, a], idx[1][:, b], idx[2][:, c]), wab * w[2][:, c])
    BC = spme_influence(L, beta, tuple(K), n)
    FQ = np.fft.fftn(Q)
    E = 0.5 * float((BC * np.abs(FQ) ** 2).sum())
    conv = np.real(np.fft.ifftn(BC * FQ)) * float(np.prod(K))
    G = np.zeros_like(q)
    for a in range(n):
        for b in range(n):
            for c in range(n):
                cv = conv[idx[0][:, a], idx[1][:, b], idx[2][:, c]]
                G[:, 0] += cv * dw[0][:, a] * w[1][:, b] * w[2][:, c]
                G[:, 1] += cv * w[0][:, a] * dw[1][:, b] * w[2][:, c]
                G[:, 2] += cv * w[0][:, a] * w[1][:, b] * dw[2][:, c]
    G *= (charge[:, None] * (K / L)[None, :])
    return K_COUL * E, K_COUL * G
