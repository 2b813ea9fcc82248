"""Candidate rows for the jump step and the pair sums.

Paper Sec. V, first paragraph: the Poisson parameter of atom i uses the number
of particles that interact with i, and the partner J is drawn uniformly among
them.  Any superset of the interacting set is exact (extra candidates have
F_ij = 0 and are always rejected).  This project's candidate row of atom i:

    { j : molecule(j) != molecule(i),  r_ij^2 < r_list^2 }   in ascending j,

with r_ij^2 = (dx*dx + dy*dy) + dz*dz in FP64 round-to-nearest (minimum image
d - L rint(d/L) under periodic boundaries), r_list = r_c + skin, or every
other-molecule atom when there is no cutoff.  Rows are rebuilt at a position
set q when max_i |q_i - q_i(ref)|^2 > (skin/2)^2 (unwrapped displacement since
the last build), checked before every evaluation.

``rows`` is the brute-force definition.  ``rows_cell_list`` is an
independent construction through a cell grid, used only to pin ``rows``.
"""
import math
import numpy as np


def _r2(q_i, q_j, box):
    d = q_i - q_j
    if box is not None:
        L = np.asarray(box, dtype=np.float64)
        d = d - L * np.rint(d / L)
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def rows(q, mol, r_list, box=None, atoms=None):
    """Brute-force candidate rows (list of int64 arrays, ascending)."""
    q = np.asarray(q, dtype=np.float64)
    mol = np.asarray(mol)
    n = q.shape[0]
    atoms = np.arange(n) if atoms is None else np.asarray(atoms)
    out = []
    rl2 = r_list * r_list if math.isfinite(r_list) else math.inf
    chunk = max(1, 4_000_000 // max(n, 1))
    for s in range(0, len(atoms), chunk):
        idx = atoms[s:s + chunk]
        r2 = _r2(q[idx][:, None, :], q[None, :, :], box)
        ok = (mol[idx][:, None] != mol[None, :]) & (r2 < rl2)
        for k in range(len(idx)):
            out.append(np.nonzero(ok[k])[0].astype(np.int64))
    return out


def rows_cell_list(q, mol, r_list, box=None):
    """Same rows through a cell grid of edge >= r_list (27-cell stencil).

    Open boundaries: the grid spans the bounding box of q.  Periodic: the box
    is cut into floor(L / r_list) cells per axis (at least 3)."""
    q = np.asarray(q, dtype=np.float64)
    n = q.shape[0]
    if box is not None:
        L = np.asarray(box, dtype=np.float64)
        nc = np.maximum(np.floor(L / r_list).astype(int), 1)
        h = L / nc
        w = q - L * np.floor(q / L)
        c = np.minimum(np.floor(w / h).astype(int), nc - 1)
    else:
        lo = q.min(0)
        span = q.max(0) - lo
        nc = np.maximum(np.floor(span / r_list).astype(int), 1)
        h = np.where(nc > 0, np.maximum(span / nc, r_list), r_list)
        c = np.minimum(np.floor((q - lo) / h).astype(int), nc - 1)
    key = (c[:, 0] * nc[1] + c[:, 1]) * nc[2] + c[:, 2]
    cells = {}
    for a in range(n):
        cells.setdefault(int(key[a]), []).append(a)
    out = []
    rl2 = r_list * r_list
    for i in range(n):
        cand = set()
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    cc = c[i] + np.array([dx, dy, dz])
                    if box is not None:
                        cc = cc % nc
                    elif np.any(cc < 0) or np.any(cc >= nc):
                        continue
                    k = int((cc[0] * nc[1] + cc[1]) * nc[2] + cc[2])
                    cand.update(cells.get(k, []))
        cand = np.array(sorted(cand), dtype=np.int64)
        r2 = _r2(q[i][None, :], q[cand], box)
        ok = (mol[cand] != mol[i]) & (r2 < rl2)
        out.append(cand[ok])
    return out


def needs_rebuild(q, q_ref, skin):
    """max_i |q_i - q_ref_i|^2 > (skin/2)^2 (FP64, unwrapped)."""
    if q_ref is None:
        return True
    d = q - q_ref
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    h = 0.5 * skin
    return bool(np.any(d2 > h * h))


def to_pairs(row_list, atoms=None):
    """Flatten rows into directed pair arrays (ii, jj)."""
    atoms = np.arange(len(row_list)) if atoms is None else np.asarray(atoms)
    ii = np.concatenate([np.full(len(r), a, dtype=np.int64) for a, r in zip(atoms, row_list)]) if len(row_list) else np.zeros(0, np.int64)
    jj = np.concatenate(row_list) if len(row_list) else np.zeros(0, np.int64)
    return ii, jj
