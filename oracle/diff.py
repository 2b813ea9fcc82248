"""Force matching on the direct-space pair terms (FP64, PyTorch CPU autograd).

The pair forces of the force field are F_i = -sum_j g(r_ij) (q_i - q_j) with
g = W'(r)/r, W = k q_a q_b / r (or k q_a q_b erfc(beta r)/r under periodic
Ewald) + 4 eps_ab ((sigma_ab/r)^12 - (sigma_ab/r)^6), summed over pairs of
different molecules with r^2 < r_c^2 (paper Sec. IV.A, V).  Parameters are
per atom type: charges q_t and symmetric tables sigma_ab, eps_ab.

force_matching_loss returns L = sum_i |F_i - F_target,i|^2 + w_E E and its
gradients with respect to positions, charges, sigma and eps by reverse-mode
automatic differentiation of this plain formula: an independent route to the
same numbers the GPU's hand-written backward computes.  Pinned by central
finite differences (tests/test_oracle_diff.py).
"""
import math

import numpy as np
import torch

from .forcefield import K_COUL
from .neighbors import rows_cell_list, to_pairs


def _pairs(q, mol, r_cut, box):
    """Directed pairs (i, j) of different molecules with r^2 < r_c^2 (FP64):
    through the oracle's cell list when there is a cutoff (the same set as
    the brute-force rows, which pin it), else every pair."""
    n = len(mol)
    if math.isfinite(r_cut):
        return to_pairs(rows_cell_list(q, mol, r_cut, box))
    ii, jj = np.nonzero(mol[:, None] != mol[None, :])
    d = q[ii] - q[jj]
    if box is not None:
        d = d - box * np.rint(d / box)
    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    keep = r2 < r_cut * r_cut if math.isfinite(r_cut) else np.ones(len(ii), bool)
    return ii[keep], jj[keep]


def forces_energy(q, typ, qt, sig, eps, ii, jj, ewald_beta=0.0, box=None):
    """Torch FP64: (F (N, 3), E) for the directed pairs (ii, jj)."""
    d = q[ii] - q[jj]
    if box is not None:
        L = torch.as_tensor(box, dtype=torch.float64)
        d = d - L * torch.round(d.detach() / L)
    r2 = (d * d).sum(1)
    r = torch.sqrt(r2)
    ti, tj = typ[ii], typ[jj]
    qq = K_COUL * qt[ti] * qt[tj]
    s6 = sig[ti, tj] ** 6
    c12 = 4.0 * eps[ti, tj] * s6 * s6
    c6 = 4.0 * eps[ti, tj] * s6
    ir = 1.0 / r
    ir6 = ir ** 6
    if ewald_beta > 0:
        b = ewald_beta
        W = qq * torch.erfc(b * r) * ir
        dW = -qq * (torch.erfc(b * r) * ir * ir + 2.0 * b / math.sqrt(math.pi) * torch.exp(-b * b * r2) * ir)
    else:
        W = qq * ir
        dW = -qq * ir * ir
    W = W + (c12 * ir6 - c6) * ir6
    dW = dW + (-12.0 * c12 * ir6 + 6.0 * c6) * ir6 * ir
    g = dW * ir
    n = q.shape[0]
    G = torch.zeros((n, 3), dtype=torch.float64).index_add(0, torch.as_tensor(ii), g[:, None] * d)
    E = 0.5 * W.sum()           # every unordered pair appears twice among the directed pairs
    return -G, E


def force_matching_loss(q, typ, mol, qt, sig, eps, F_target, r_cut, ewald_beta=0.0, box=None, w_energy=0.0):
    """L and dL/d(q, qt, sig, eps) (sig, eps gradients symmetrised: entry
    (a, b) is the derivative with respect to the shared table entry)."""
    ii, jj = _pairs(np.asarray(q), np.asarray(mol), r_cut, None if box is None else np.asarray(box))
    tq = torch.tensor(np.asarray(q), dtype=torch.float64, requires_grad=True)
    tqt = torch.tensor(np.asarray(qt), dtype=torch.float64, requires_grad=True)
    tsu = torch.tensor(np.asarray(sig), dtype=torch.float64, requires_grad=True)
    teu = torch.tensor(np.asarray(eps), dtype=torch.float64, requires_grad=True)
    tsig = 0.5 * (tsu + tsu.T)          # one parameter per unordered type pair
    teps = 0.5 * (teu + teu.T)
    typ_t = torch.as_tensor(np.asarray(typ), dtype=torch.long)
    F, E = forces_energy(tq, typ_t, tqt, tsig, teps, ii, jj, ewald_beta, box)
    L = ((F - torch.as_tensor(np.asarray(F_target), dtype=torch.float64)) ** 2).sum() + w_energy * E
    gq, gqt, gs, ge = torch.autograd.grad(L, [tq, tqt, tsu, teu])
    # the symmetrisation halves each off-diagonal derivative: undo it
    gs = gs + gs.T - torch.diag(torch.diagonal(gs))
    ge = ge + ge.T - torch.diag(torch.diagonal(ge))
    return float(L.detach()), F.detach().numpy(), float(E.detach()), gq.numpy(), gqt.numpy(), gs.numpy(), ge.numpy()
