"""BAOAB and BOUNCE (BJAOAJB) steps in FP64, following the paper.

Paper Sec. III.C (splitting): one step of BOUNCE is
    B(delta/2) J(delta/2) A(delta/2) O(delta) A(delta/2) J(delta/2) B(delta/2)
and BAOAB is the same without the J steps.  Sec. IV.B spells the steps out:
    B: p <- p - delta/2 F_0(q)
    J: for each atom i independently (Sec. IV.A: given q, the V_i are
       independent chains), draw M_i ~ Poisson(n_i beta ||v_i|| L delta/2),
       then M_i times: J uniform over the n_i candidates, U uniform on [0,1];
       if U < lambda_iJ / lambda*_iJ then v_i <- R_iJ(v_i)
    A: q <- q + delta/2 M^-1 p
    O: p <- e^{-gamma delta} p + sqrt(beta^-1 (1 - e^{-2 gamma delta}) M) G
with lambda_ij = beta max(0, v_i . F_ij), lambda* = beta ||v_i|| L and
R_ij(v) = v - 2 (v . F_ij)/||F_ij||^2 F_ij (Sec. IV.A).  So the acceptance
test is U ||v_i|| L < v_i . F_ij (beta cancels).

Readings of the paper used here (all listed in the design notes):
  * F_0 = bonded + (1 - chi) part of every pair term; F_ij = chi W' d/r.
  * friction coefficient is mass-independent: c1 = exp(-gamma delta).
  * L is the per-type row maximum L*_{t_i} (oracle.bounds), or, with
    per-type-pair bounds, Lt_{t_i t_j} with the two-stage partner choice
    (jump_half, oracle.bounds.pair_weights).
  * Candidates (Sec. V: J is drawn among the particles interacting with i):
    when the jumps carry only the LJ part (Coulomb wholly in F_0) with one
    bound per type, a pair of types without LJ parameters does not interact
    through the jump part, so the row of an atom keeps only the partners its
    type has LJ with, and the rows are rebuilt on the displacement of the
    atoms that can take part in a jump (jump_partners).
  * Random numbers: Philox4x32-10 keyed by the run seed with counter
    (slot, atom, step, stream); stream 1 for the J after the first B,
    stream 2 for the J before the last B, stream 0 for O.  Proposal k
    (1-based) uses slot k: J = floor(x0 n_i / 2^32), U = 53-bit from x1, x2.
    O uses slot 0: Box-Muller on (x0, x1) and (x2, x3).
  * Units: v in A/fs, gradients in kcal/mol/A; a kick is
    v <- v - (h * 4.184e-4 / m) G.
  * Periodic Ewald (Sec. V): the reciprocal part (SPME) plus the removal of
    excluded (same-molecule) pairs from it is one gradient term G_recip.
    BAOAB adds it to the full gradient; basic BOUNCE adds it to F_0 (every
    step); BOUNCE-RESPA kicks with it over Delta/2 = m delta/2 before and
    after every block of m BJAOAJB steps (the outer splitting of Sec. V).
"""
import math
import numpy as np

from . import philox, poisson
from .forcefield import (ACCEL, KB, Params, bonded_gradients, pair_gradients, pair_gradient_magnitudes,
                         bonded_gradient_magnitudes, pair_gradient_one, kinetic_energy, pair_energies,
                         pair_energy_magnitudes, bonded_energies)
from .neighbors import rows as build_rows, needs_rebuild, to_pairs
from . import ewald


class Topology:
    def __init__(self, typ, mass, charge, mol, bonds, bond_k_r0, angles, angle_k_t0):
        self.type = np.asarray(typ, dtype=np.int64)
        self.mass = np.asarray(mass, dtype=np.float64)
        self.charge = np.asarray(charge, dtype=np.float64)
        self.mol = np.asarray(mol, dtype=np.int64)
        self.bonds = np.asarray(bonds, dtype=np.int64).reshape(-1, 2)
        self.bond_k_r0 = np.asarray(bond_k_r0, dtype=np.float64).reshape(-1, 2)
        self.angles = np.asarray(angles, dtype=np.int64).reshape(-1, 3)
        self.angle_k_t0 = np.asarray(angle_k_t0, dtype=np.float64).reshape(-1, 2)


def o_step(v, mass, temperature, gamma, dt, seed, step, atoms=None):
    """O: v <- c1 v + sqrt((1 - c1^2) k_B T / m) G, c1 = exp(-gamma dt)."""
    n = v.shape[0]
    atoms = np.arange(n) if atoms is None else atoms
    x = philox.draw(seed, 0, atoms, step, philox.STREAM_O)
    ua, ub = philox.u24_open0(x[0]), philox.u24(x[1])
    uc, ud = philox.u24_open0(x[2]), philox.u24(x[3])
    r1 = np.sqrt(-2.0 * np.log(ua))
    r2 = np.sqrt(-2.0 * np.log(uc))
    g = np.stack([r1 * np.cos(2.0 * math.pi * ub), r1 * np.sin(2.0 * math.pi * ub), r2 * np.cos(2.0 * math.pi * ud)], 1)
    c1 = math.exp(-gamma * dt)
    sd = np.sqrt((1.0 - c1 * c1) * KB * temperature * ACCEL / mass)
    return c1 * v + sd[:, None] * g


def typed_rows(row_list, typ, n_types):
    """Candidate rows regrouped by partner type: segment b holds the members of
    type b in ascending index, segments in increasing b; and the counts n_ib."""
    typ = np.asarray(typ)
    out = []
    counts = np.zeros((len(row_list), n_types), dtype=np.int64)
    for i, r in enumerate(row_list):
        r = np.asarray(r, dtype=np.int64)
        segs = [r[typ[r] == b] for b in range(n_types)]
        out.append(np.concatenate(segs) if segs else r)
        counts[i] = [len(x) for x in segs]
    return out, counts


def two_stage_pick(t, C, S, Lq_a):
    """Position in the type-grouped row of the candidate that weight unit t
    (0 <= t < W) falls on: segment b with C_b <= t < C_{b+1}, then
    (t - C_b) // Lq_ab within it.  C: (m, T+1) cumulative weights, S: (m, T+1)
    segment starts, Lq_a: (m, T) weights of the atoms' types."""
    t = np.asarray(t, dtype=np.int64)
    b = (C[:, 1:] <= t[:, None]).sum(1)
    rows = np.arange(len(t))
    return S[rows, b] + (t - C[rows, b]) // Lq_a[rows, b]


def jump_partners(typ, Lstar, p, pair_bounds=None):
    """Which candidates a jump can draw (reading of Sec. V: the partner J of
    atom i is drawn among the particles interacting with i through the jump
    part).  With LJ alone on the jumps (p.coulomb_jumps False) and one bound
    per type, atom i of type a proposes only if L*_a > 0, and only atoms of a
    type b with LJ parameters for (a, b) interact with it through the jump
    part.  Returns None when that keeps every candidate (Coulomb on the jumps,
    per-type-pair bounds, or no pair of present types without LJ), else
    (partner [T, T] bool: type b is a candidate of type a; moving [T] bool:
    types whose displacement can change a row, owners and their partners)."""
    if pair_bounds is not None or p.coulomb_jumps:
        return None
    T = len(Lstar)
    lj = (np.asarray(p.lj_eps)[:T, :T] != 0) & (np.asarray(p.lj_sigma)[:T, :T] != 0)
    present = np.zeros(T, bool)
    present[np.unique(typ)] = True
    owner = (np.asarray(Lstar) > 0) & present
    partner = owner[:, None] & lj
    if not np.any(owner[:, None] & present[None, :] & ~partner):
        return None
    return partner, owner | partner.any(0)


def filter_rows(row_list, typ, partner):
    """Rows restricted to the candidates a jump can draw: member j of atom i
    stays if partner[t_i, t_j] (ascending order kept; atoms whose type has
    no partner get empty rows)."""
    typ = np.asarray(typ)
    return [r[partner[typ[i], typ[r]]] for i, r in enumerate(row_list)]


def jump_half(q, v, row_list, topo, p, Lstar_row, beta, dt, seed, step, stream, record=False, pair_bounds=None):
    """The jump step J over a half step dt/2 for every atom (Sec. IV.B).

    pair_bounds = None: one bound L*_{t_i} for every candidate, J uniform over
    the row.  pair_bounds = (Lq, Lt) (oracle.bounds.pair_weights): two-stage
    choice over the type-grouped row (typed_rows) -- the weight of a candidate
    of type b is Lq_ab, the Poisson mean is beta ||v|| (delta/2) L*_a W_i 2^-16
    with W_i = sum_b n_ib Lq_ab, and the acceptance bound is Lt_ab.
    Proposal k: t = floor(x0 W_i / 2^32); segment b with C_b <= t < C_{b+1}
    (C_b = sum_{c<b} n_ic Lq_ac); J = (start of segment b) + (t - C_b) // Lq_ab.

    Returns the new velocities and, if record, a dict of per-proposal arrays
    (atom, k, J, j, U, ratio = max(0, v.F)/(||v|| L), accepted)."""
    n = q.shape[0]
    v = np.array(v, dtype=np.float64, copy=True)
    if pair_bounds is not None:
        Lq, Lt = pair_bounds
        T = Lq.shape[0]
        row_list, counts = typed_rows(row_list, topo.type, T)
        wq = counts * Lq[topo.type]                      # n_ib Lq_ab
        W = wq.sum(1)
        C = np.concatenate([np.zeros((n, 1), np.int64), np.cumsum(wq, 1)], 1)
        S = np.concatenate([np.zeros((n, 1), np.int64), np.cumsum(counts, 1)], 1)
        assert np.all(W < 2 ** 32)
    nrow = np.array([len(r) for r in row_list], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(nrow)])
    flat = np.concatenate(row_list) if n else np.zeros(0, np.int64)
    s = np.sqrt((v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2])
    Ls = Lstar_row[topo.type]
    if pair_bounds is None:
        mu = ((((beta * s) * Ls) * nrow) * dt) * 0.5
    else:
        mu = ((((beta * s) * Ls) * (W * 2.0 ** -16)) * dt) * 0.5
    atoms = np.arange(n)
    M = poisson.counts(mu, atoms, seed, step, stream)
    rec = {k: [] for k in ('atom', 'k', 'J', 'j', 'U', 'ratio', 'accepted')} if record else None
    kmax = int(M.max()) if n else 0
    for k in range(1, kmax + 1):
        act = np.nonzero(M >= k)[0]
        x = philox.draw(seed, k, act, step, stream)
        if pair_bounds is None:
            J = philox.index_below(x[0], nrow[act])
        else:
            J = two_stage_pick(philox.index_below(x[0], W[act]), C[act], S[act], Lq[topo.type[act]])
        j = flat[offs[act] + J]
        U = philox.u53(x[1], x[2])
        ti, tj = topo.type[act], topo.type[j]
        Lb = Ls[act] if pair_bounds is None else Lt[ti, tj]
        G = pair_gradient_one(q[act], q[j], topo.charge[act], topo.charge[j],
                              p.lj_sigma[ti, tj], p.lj_eps[ti, tj], p, part="long")
        va = v[act]
        a = (va[:, 0] * G[:, 0] + va[:, 1] * G[:, 1]) + va[:, 2] * G[:, 2]
        thr = (U * s[act]) * Lb
        acc = thr < a
        if record:
            with np.errstate(divide='ignore', invalid='ignore'):
                ratio = np.where(s[act] > 0, np.maximum(a, 0.0) / (s[act] * Lb), 0.0)
            for key, val in (('atom', act), ('k', np.full(len(act), k)), ('J', J), ('j', j), ('U', U),
                             ('ratio', ratio), ('accepted', acc)):
                rec[key].append(val)
        if np.any(acc):
            ia = act[acc]
            Ga = G[acc]
            aa = a[acc]
            ff = (Ga[:, 0] * Ga[:, 0] + Ga[:, 1] * Ga[:, 1]) + Ga[:, 2] * Ga[:, 2]
            coef = (aa + aa) / ff
            v[ia] = v[ia] - coef[:, None] * Ga
    if record:
        rec = {key: (np.concatenate(val) if val else np.zeros(0)) for key, val in rec.items()}
        rec['M'] = M
        rec['mu'] = mu
    return v, rec


class OracleMD:
    """Plain FP64 BAOAB / BOUNCE integrator over one system."""

    def __init__(self, q, v, topo, p, *, dt=1.0, gamma=0.001, temperature=300.0, seed=0, skin=1.0, step=0,
                 pair_bounds=False):
        self.q = np.array(q, dtype=np.float64)
        self.v = np.array(v, dtype=np.float64)
        self.topo = topo
        self.p = p
        self.dt = float(dt)
        self.gamma = float(gamma)
        self.T = float(temperature)
        self.beta = 1.0 / (KB * self.T)
        self.seed = int(seed)
        self.skin = float(skin)
        self.step_index = int(step)
        self.q_ref = None
        self.row_list = None
        self._plist = None          # BAOAB's own pair list (see full_pairs)
        self._plist_ref = None
        self.rebuilds = 0
        self.proposals = 0
        self.accepts = 0
        self.tie_atoms = set()      # atoms whose thinning decision was within 1e-6 of a tie
        from .bounds import bound_table, pair_weights
        T = int(max(topo.type.max() + 1, p.lj_sigma.shape[0]))
        self.L, self.Lstar = bound_table(topo.charge, topo.type, T, p.lj_sigma, p.lj_eps, p)
        self.pair_bounds = pair_weights(self.L, self.Lstar) if pair_bounds else None
        # rows of the jump step when they differ from the full rows (jump_partners)
        self.jp = jump_partners(topo.type, self.Lstar, p, self.pair_bounds)
        self.jrows = None
        self.jq_ref = None

    @property
    def r_list(self):
        return self.p.r_cut + self.skin if math.isfinite(self.p.r_cut) else math.inf

    def ensure_rows(self):
        if self.row_list is None or (math.isfinite(self.r_list) and needs_rebuild(self.q, self.q_ref, self.skin)):
            self.row_list = build_rows(self.q, self.topo.mol, self.r_list, self.p.box)
            self.q_ref = self.q.copy()
            if self.jp is None:
                self.rebuilds += 1

    def jump_rows(self):
        """The candidate rows of the jump step at the current positions: the
        full rows, or (jump_partners) the rows restricted to the partners a
        jump can draw, rebuilt when an atom of a moving type has moved half
        the skin since their build (atoms of other types neither propose nor
        are drawn)."""
        if self.jp is None:
            self.ensure_rows()
            return self.row_list
        partner, moving = self.jp
        mv = moving[self.topo.type]
        if self.jrows is None or (math.isfinite(self.r_list) and needs_rebuild(self.q[mv], self.jq_ref[mv], self.skin)):
            full = build_rows(self.q, self.topo.mol, self.r_list, self.p.box)
            self.jrows = filter_rows(full, self.topo.type, partner)
            self.jq_ref = self.q.copy()
            self.rebuilds += 1
        return self.jrows

    def pairs(self):
        return to_pairs(self.row_list)

    def full_pairs(self):
        """Pairs for BAOAB's full gradient from a list of its own, refreshed by
        the same skin rule: BAOAB reads no candidate rows, so its steps leave
        the rows of the jump step (and their rebuild history) untouched.  The
        pairs inside r_c are the same either way."""
        if self._plist is None or (math.isfinite(self.r_list) and needs_rebuild(self.q, self._plist_ref, self.skin)):
            self._plist = to_pairs(build_rows(self.q, self.topo.mol, self.r_list, self.p.box))
            self._plist_ref = self.q.copy()
        return self._plist

    def grad_short(self):
        """F_0: bonded + (1 - chi) pair part."""
        return self.grad_short_pairs() + self.grad_bonded()

    def grad_short_pairs(self):
        ii, jj = self.pairs()
        t = self.topo
        return pair_gradients(self.q, t.charge, t.type, ii, jj, self.p, "short")

    def grad_bonded(self):
        t = self.topo
        return bonded_gradients(self.q, t.bonds, t.bond_k_r0, t.angles, t.angle_k_t0, self.p.box)

    def grad_full(self, pairs=None):
        ii, jj = self.pairs() if pairs is None else pairs
        t = self.topo
        return (pair_gradients(self.q, t.charge, t.type, ii, jj, self.p, "full")
                + bonded_gradients(self.q, t.bonds, t.bond_k_r0, t.angles, t.angle_k_t0, self.p.box))

    def has_recip(self):
        return self.p.box is not None and self.p.ewald_beta > 0 and self.p.pme_grid is not None

    def recip(self):
        """(E_recip + E_self + E_excl, gradient of E_recip + E_excl)."""
        if not self.has_recip():
            return 0.0, np.zeros_like(self.q)
        t = self.topo
        er, gr = ewald.spme_recip(self.q, t.charge, self.p.box, self.p.ewald_beta, self.p.pme_grid, self.p.pme_order)
        if not hasattr(self, "_excl"):
            self._excl = ewald.molecule_pairs(t.mol)
        ex, gx = ewald.exclusion(self.q, t.charge, self._excl, self.p.ewald_beta, self.p.box)
        return er + ex + ewald.self_energy(t.charge, self.p.ewald_beta), gr + gx

    def grad_long(self):
        ii, jj = self.pairs()
        t = self.topo
        return pair_gradients(self.q, t.charge, t.type, ii, jj, self.p, "long")

    def grad_scale(self, part):
        """Per-atom sum of the magnitudes of the terms of the gradient part
        (the forward error scale of a floating-point evaluation)."""
        ii, jj = self.pairs()
        t = self.topo
        m = pair_gradient_magnitudes(self.q, t.charge, t.type, ii, jj, self.p, part)
        if part != "long":
            m = m + bonded_gradient_magnitudes(self.q, t.bonds, t.bond_k_r0, t.angles, t.angle_k_t0, self.p.box)
        return m

    def energy_scale(self):
        ii, jj = self.pairs()
        t = self.topo
        return pair_energy_magnitudes(self.q, t.charge, t.type, ii, jj, self.p)

    def kick(self, G, h):
        self.v = self.v - ((h * ACCEL) / self.topo.mass)[:, None] * G

    def drift(self, h):
        self.q = self.q + h * self.v

    def jump(self, stream, record=False):
        self.v, rec = jump_half(self.q, self.v, self.jump_rows(), self.topo, self.p, self.Lstar, self.beta,
                                self.dt, self.seed, self.step_index, stream, record=True,
                                pair_bounds=self.pair_bounds)
        self.proposals += int(rec['M'].sum())
        self.accepts += int(rec['accepted'].sum()) if len(rec['accepted']) else 0
        if len(rec['U']):
            self.tie_atoms.update(rec['atom'][np.abs(rec['U'] - rec['ratio']) < 1e-6].tolist())
        return rec if record else None

    def step_baoab(self):
        h = 0.5 * self.dt
        self.kick(self.grad_full(self.full_pairs()) + self.recip()[1], h)
        self.drift(h)
        self.v = o_step(self.v, self.topo.mass, self.T, self.gamma, self.dt, self.seed, self.step_index)
        self.drift(h)
        self.kick(self.grad_full(self.full_pairs()) + self.recip()[1], h)
        self.step_index += 1

    def _f0(self, with_recip, bonded_only):
        g = self.grad_bonded() if bonded_only else self.grad_short()
        return g + (self.recip()[1] if with_recip else 0.0)

    def step_bounce(self, record=False, with_recip=True, bonded_only=False):
        """One BJAOAJB step; F_0 includes G_recip unless with_recip is False
        (BOUNCE-RESPA moves it to the outer kicks) and holds only the bonded
        terms when bonded_only (the extended split's inner steps)."""
        h = 0.5 * self.dt
        self.ensure_rows()
        self.kick(self._f0(with_recip, bonded_only), h)
        r1 = self.jump(philox.STREAM_J1, record)
        self.drift(h)
        self.v = o_step(self.v, self.topo.mass, self.T, self.gamma, self.dt, self.seed, self.step_index)
        self.drift(h)
        self.ensure_rows()
        r2 = self.jump(philox.STREAM_J2, record)
        self.kick(self._f0(with_recip, bonded_only), h)
        self.step_index += 1
        return (r1, r2) if record else None

    def block_bounce_respa(self, m=2, extended=False):
        """One outer step Delta = m delta of BOUNCE-RESPA: kick with G_out over
        Delta/2, m BJAOAJB steps without it, kick again over Delta/2.
        G_out = G_recip, or with extended = True (Sec. V, the bonded/non-bonded
        split) G_out = short-range pair part + G_recip and the inner F_0 holds
        only the bonded terms."""
        H = 0.5 * m * self.dt

        def g_out():
            self.ensure_rows()
            return self.recip()[1] + (self.grad_short_pairs() if extended else 0.0)

        self.kick(g_out(), H)
        for _ in range(m):
            self.step_bounce(with_recip=False, bonded_only=extended)
        self.kick(g_out(), H)

    def block_bounce_respa1(self, m=4, m2=3):
        """One outer step Delta_out = m2 m delta of BOUNCE-RESPA1 (Sec. V, the
        RESPA1 splitting): kick with G_recip over Delta_out/2; m2 intermediate
        steps, each a kick with the short-range pair part over m delta/2, m
        BJAOAJB steps whose F_0 holds only the bonded terms, and the same kick
        again; the reciprocal kick again."""
        H_out = 0.5 * m2 * m * self.dt
        H_mid = 0.5 * m * self.dt

        def g_mid():
            self.ensure_rows()
            return self.grad_short_pairs()

        self.kick(self.recip()[1], H_out)
        for _ in range(m2):
            self.kick(g_mid(), H_mid)
            for _ in range(m):
                self.step_bounce(with_recip=False, bonded_only=True)
            self.kick(g_mid(), H_mid)
        self.kick(self.recip()[1], H_out)

    def run(self, n, integrator="bounce", respa_m=2, respa_m2=3):
        if integrator in ("bounce_respa", "bounce_respa_ext"):
            assert n % respa_m == 0
            for _ in range(n // respa_m):
                self.block_bounce_respa(respa_m, extended=integrator == "bounce_respa_ext")
            return
        if integrator == "bounce_respa1":
            assert n % (respa_m * respa_m2) == 0
            for _ in range(n // (respa_m * respa_m2)):
                self.block_bounce_respa1(respa_m, respa_m2)
            return
        for _ in range(n):
            if integrator == "bounce":
                self.step_bounce()
            else:
                self.step_baoab()

    def energies(self):
        self.ensure_rows()
        ii, jj = self.pairs()
        t = self.topo
        ec, el = pair_energies(self.q, t.charge, t.type, ii, jj, self.p)
        eb, ea = bonded_energies(self.q, t.bonds, t.bond_k_r0, t.angles, t.angle_k_t0, self.p.box)
        ek = kinetic_energy(self.v, t.mass)
        er = self.recip()[0]
        return dict(coul=ec, lj=el, bond=eb, angle=ea, recip=er, kin=ek, pot=ec + el + eb + ea + er)
