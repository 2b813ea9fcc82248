"""Seeded synthetic flexible 3-site water systems (inputs only).

This module builds the inputs that both the CUDA library and the FP64 oracle
are run on; it holds none of the integrator's arithmetic.  Random numbers come
from numpy's PCG64 generator seeded by the caller, never from the method's own
Philox streams.

Recipe (the paper's droplet and periodic water workloads, Sec. VI, rebuilt as
synthetic stand-ins since the paper's own boxes are not published):
  * molecules on a simple cubic lattice at 1 g/cm^3 (spacing 3.1037 A);
  * rigid starting geometry O-H 1.0 A, H-O-H 104.5 deg, uniformly random
    orientation per molecule (random unit quaternion);
  * Maxwell-Boltzmann velocities at the requested temperature;
  * charges q_O = -0.834 e, q_H = +0.417 e; Lennard-Jones on O-O only
    (sigma 3.15 A, epsilon 0.152 kcal/mol); harmonic O-H bonds and H-O-H angle.
Units: A, fs, kcal/mol, g/mol, e, K.
"""
from dataclasses import dataclass, field
import math
import numpy as np

KB_KCAL = 0.0019872041          # kcal / (mol K)
ACCEL = 4.184e-4                # (kcal/mol/A) / (g/mol) -> A/fs^2
WATER_MOLAR_MASS = 18.015       # g/mol
AVOGADRO_PER_A3 = 0.6022140857  # N_A * 1e-24 (cm^3 -> A^3)

TYPE_O, TYPE_H = 0, 1


@dataclass
class WaterModel:
    q_O: float = -0.834
    q_H: float = 0.417
    m_O: float = 15.9994
    m_H: float = 1.008
    sigma_OO: float = 3.15
    eps_OO: float = 0.152
    r_OH: float = 1.0
    theta_HOH_deg: float = 104.5
    k_bond: float = 450.0      # E = k (r - r0)^2, kcal/mol/A^2
    k_angle: float = 55.0      # E = k (theta - theta0)^2, kcal/mol/rad^2


@dataclass
class System:
    q: np.ndarray            # (N, 3) positions, A
    v: np.ndarray            # (N, 3) velocities, A/fs
    type: np.ndarray         # (N,) int32 type id (0 = O, 1 = H)
    mass: np.ndarray         # (N,) g/mol
    charge: np.ndarray       # (N,) e
    molecule: np.ndarray     # (N,) int32 molecule id
    bonds: np.ndarray        # (nb, 2) int32 atom pairs
    bond_k_r0: np.ndarray    # (nb, 2) (k, r0)
    angles: np.ndarray       # (na, 3) int32 (end, vertex, end)
    angle_k_t0: np.ndarray   # (na, 2) (k, theta0 in rad)
    lj_sigma: np.ndarray     # (T, T)
    lj_eps: np.ndarray       # (T, T)
    box: np.ndarray = None   # (3,) edge lengths for periodic boxes, None for droplets
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self):
        return int(self.q.shape[0])


def lattice_spacing(density_g_cm3=1.0):
    """Edge of the cube holding one molecule at the given density (A)."""
    n_per_a3 = density_g_cm3 * AVOGADRO_PER_A3 / WATER_MOLAR_MASS
    return n_per_a3 ** (-1.0 / 3.0)


def _random_rotations(rng, n):
    """Uniform random rotation matrices from uniform unit quaternions."""
    u1, u2, u3 = rng.random((3, n))
    a = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2)
    b = np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
    c = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    d = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    # quaternion (d; a, b, c) -> rotation matrix
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (b * b + c * c)
    R[:, 0, 1] = 2 * (a * b - c * d)
    R[:, 0, 2] = 2 * (a * c + b * d)
    R[:, 1, 0] = 2 * (a * b + c * d)
    R[:, 1, 1] = 1 - 2 * (a * a + c * c)
    R[:, 1, 2] = 2 * (b * c - a * d)
    R[:, 2, 0] = 2 * (a * c - b * d)
    R[:, 2, 1] = 2 * (b * c + a * d)
    R[:, 2, 2] = 1 - 2 * (a * a + b * b)
    return R


def _build(centers, rng, model, temperature, box):
    nm = centers.shape[0]
    half = math.radians(model.theta_HOH_deg) / 2
    body = np.array([[0.0, 0.0, 0.0],
                     [model.r_OH * math.sin(half), 0.0, model.r_OH * math.cos(half)],
                     [-model.r_OH * math.sin(half), 0.0, model.r_OH * math.cos(half)]])
    R = _random_rotations(rng, nm)
    q = (centers[:, None, :] + np.einsum('mij,aj->mai', R, body)).reshape(-1, 3)
    n = 3 * nm
    typ = np.tile(np.array([TYPE_O, TYPE_H, TYPE_H], dtype=np.int32), nm)
    mass = np.where(typ == TYPE_O, model.m_O, model.m_H).astype(np.float64)
    charge = np.where(typ == TYPE_O, model.q_O, model.q_H).astype(np.float64)
    mol = np.repeat(np.arange(nm, dtype=np.int32), 3)
    o = 3 * np.arange(nm, dtype=np.int32)
    bonds = np.stack([np.stack([o, o + 1], 1), np.stack([o, o + 2], 1)], 1).reshape(-1, 2)
    bond_k_r0 = np.tile([model.k_bond, model.r_OH], (bonds.shape[0], 1))
    angles = np.stack([o + 1, o, o + 2], 1)
    angle_k_t0 = np.tile([model.k_angle, math.radians(model.theta_HOH_deg)], (nm, 1))
    sig = np.zeros((2, 2))
    eps = np.zeros((2, 2))
    sig[0, 0] = model.sigma_OO
    eps[0, 0] = model.eps_OO
    sd = np.sqrt(KB_KCAL * temperature * ACCEL / mass)
    v = rng.standard_normal((n, 3)) * sd[:, None]
    return System(q=q, v=v, type=typ, mass=mass, charge=charge, molecule=mol, bonds=bonds.astype(np.int32),
                  bond_k_r0=bond_k_r0, angles=angles.astype(np.int32), angle_k_t0=angle_k_t0,
                  lj_sigma=sig, lj_eps=eps, box=None if box is None else np.asarray(box, dtype=np.float64))


def water_droplet(n_side, seed=0, temperature=300.0, model=None, density=1.0):
    """n_side^3 molecules on a cubic lattice, open boundaries (a droplet)."""
    model = model or WaterModel()
    rng = np.random.default_rng(seed)
    a = lattice_spacing(density)
    g = np.arange(n_side, dtype=np.float64) * a
    centers = np.stack(np.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3)
    s = _build(centers, rng, model, temperature, None)
    s.meta.update(kind='droplet', n_side=n_side, seed=seed, spacing=a, temperature=temperature)
    return s


def water_box(n_side, seed=0, temperature=300.0, model=None, density=1.0):
    """n_side^3 molecules filling a periodic cube of edge n_side * spacing."""
    model = model or WaterModel()
    rng = np.random.default_rng(seed)
    a = lattice_spacing(density)
    g = (np.arange(n_side, dtype=np.float64) + 0.5) * a
    centers = np.stack(np.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3)
    L = n_side * a
    s = _build(centers, rng, model, temperature, np.array([L, L, L]))
    s.meta.update(kind='box', n_side=n_side, seed=seed, spacing=a, temperature=temperature)
    return s


def water_droplet_molecules(n_mol, seed=0, temperature=300.0, model=None, density=1.0):
    """A roughly spherical droplet of n_mol molecules: the n_mol lattice sites
    nearest the centre of a cube of ceil(n_mol^(1/3)) + 1 sites per side."""
    model = model or WaterModel()
    rng = np.random.default_rng(seed)
    a = lattice_spacing(density)
    side = int(math.ceil(n_mol ** (1.0 / 3.0))) + 1
    g = np.arange(side, dtype=np.float64) * a
    sites = np.stack(np.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3)
    c = sites.mean(0)
    d2 = ((sites - c) ** 2).sum(1)
    order = np.lexsort((np.arange(len(sites)), d2))
    centers = sites[np.sort(order[:n_mol])]
    s = _build(centers, rng, model, temperature, None)
    s.meta.update(kind='droplet', n_mol=n_mol, seed=seed, spacing=a, temperature=temperature)
    return s


def replica_sizes(n_replicas, lo=64, hi=1024, seed=0):
    """Molecule counts of a batch of independent droplets, uniform on [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=n_replicas)


def concat_systems(systems, spacing=500.0):
    """Back-to-back concatenation of open droplets into one topology (molecule
    ids and bonded indices renumbered, replica r shifted by r * spacing along
    x).  Returns the combined System and the atom offsets [R + 1]."""
    offs = [0]
    parts = {k: [] for k in ("q", "v", "type", "mass", "charge", "molecule", "bonds", "bond_k_r0", "angles",
                             "angle_k_t0")}
    mol0 = 0
    for r, s in enumerate(systems):
        a0 = offs[-1]
        parts["q"].append(s.q + np.array([r * spacing, 0.0, 0.0]))
        parts["v"].append(s.v)
        parts["type"].append(s.type)
        parts["mass"].append(s.mass)
        parts["charge"].append(s.charge)
        parts["molecule"].append(s.molecule + mol0)
        parts["bonds"].append(s.bonds + a0)
        parts["bond_k_r0"].append(s.bond_k_r0)
        parts["angles"].append(s.angles + a0)
        parts["angle_k_t0"].append(s.angle_k_t0)
        mol0 += int(s.molecule.max()) + 1
        offs.append(a0 + s.n_atoms)
    cat = {k: np.concatenate(v) for k, v in parts.items()}
    out = System(q=cat["q"], v=cat["v"], type=cat["type"].astype(np.int32), mass=cat["mass"], charge=cat["charge"],
                 molecule=cat["molecule"].astype(np.int32), bonds=cat["bonds"].astype(np.int32),
                 bond_k_r0=cat["bond_k_r0"], angles=cat["angles"].astype(np.int32), angle_k_t0=cat["angle_k_t0"],
                 lj_sigma=systems[0].lj_sigma, lj_eps=systems[0].lj_eps, box=None)
    out.meta.update(kind="batch", replicas=len(systems))
    return out, np.array(offs, dtype=np.int32)
