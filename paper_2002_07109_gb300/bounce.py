"""Thin ctypes binding of libbounce.so (include/bounce.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module loads the library and raises ImportError if
it has not been built (``python -m paper_2002_07109_gb300.build``); there is
no CPU fallback.

Low-level names mirror the C ABI (``bounce_create``, ``bounce_run``, ...);
``Context`` wraps them for numpy (host) arrays and torch CUDA tensors
(device pointers, passed with ``where=DEVICE``).
"""
import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbounce.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libbounce.so is not built: run `python -m paper_2002_07109_gb300.build` "
                      "(or __graft_entry__.build()) first")
_lib = C.CDLL(LIB_PATH)

OK = 0
ERR = {-1: "INVALID_ARG", -2: "CUDA", -3: "NONFINITE", -4: "LIST_OVERFLOW", -5: "STATE", -6: "UNSUPPORTED"}
HOST, DEVICE = 0, 1
BAOAB, BOUNCE, BOUNCE_RESPA, BOUNCE_RESPA_EXT, BOUNCE_RESPA1 = 0, 1, 2, 3, 4
GRAD_FULL, GRAD_SHORT, GRAD_LONG, GRAD_RECIP = 0, 1, 2, 3
MAX_TYPES = 4


class bounce_config(C.Structure):
    _fields_ = [("dt_fs", C.c_double), ("gamma_per_fs", C.c_double), ("temperature_K", C.c_double),
                ("seed", C.c_uint64), ("r_on", C.c_double), ("r_off", C.c_double), ("r_cut", C.c_double),
                ("skin", C.c_double), ("ewald_beta", C.c_double), ("periodic", C.c_int32),
                ("box", C.c_double * 3), ("max_neighbors", C.c_int32), ("max_short", C.c_int32),
                ("device", C.c_int32), ("pme_grid", C.c_int32 * 3), ("pme_order", C.c_int32),
                ("respa_m", C.c_int32), ("jump_coulomb", C.c_int32),
                ("pair_bounds", C.c_int32), ("respa_m2", C.c_int32), ("pair_skin", C.c_double),
                ("step_kernel", C.c_int32)]


class bounce_tuning(C.Structure):
    _fields_ = [("tile_j", C.c_int32), ("tile_blocks", C.c_int32), ("column_edge", C.c_double),
                ("pair_ms", C.c_double), ("candidates", C.c_int32)]


class bounce_energies(C.Structure):
    _fields_ = [("coulomb", C.c_double), ("lj", C.c_double), ("bond", C.c_double), ("angle", C.c_double),
                ("kinetic", C.c_double), ("potential", C.c_double), ("temperature", C.c_double),
                ("step", C.c_int64), ("proposals", C.c_int64), ("accepts", C.c_int64), ("near_ties", C.c_int64),
                ("rebuilds", C.c_int64), ("short_pairs", C.c_int64), ("full_pairs", C.c_int64),
                ("recip", C.c_double)]


_P = C.c_void_p
_sig = {
    "bounce_config_default": (None, [C.POINTER(bounce_config)]),
    "bounce_create": (C.c_int, [C.POINTER(_P), C.POINTER(bounce_config)]),
    "bounce_set_topology": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, C.c_int32, _P, _P, C.c_int32, _P, _P]),
    "bounce_set_lj": (C.c_int, [_P, C.c_int32, _P, _P]),
    "bounce_set_state": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, _P]),
    "bounce_get_state": (C.c_int, [_P, _P, _P, C.c_int32, _P]),
    "bounce_run": (C.c_int, [_P, C.c_int64, C.c_int32, _P]),
    "bounce_get_energies": (C.c_int, [_P, C.POINTER(bounce_energies), _P]),
    "bounce_reset_counters": (C.c_int, [_P, _P]),
    "bounce_get_bounds": (C.c_int, [_P, _P, _P]),
    "bounce_compute_gradient": (C.c_int, [_P, C.c_int32, _P, C.c_int32, _P]),
    "bounce_jump_half": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, C.c_int32, _P]),
    "bounce_get_rows": (C.c_int, [_P, _P, _P, C.c_int32]),
    "bounce_set_replicas": (C.c_int, [_P, C.c_int32, _P, _P]),
    "bounce_pair_forward": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P, C.POINTER(C.c_double), _P]),
    "bounce_pair_backward": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, C.c_double, _P, _P, _P, _P, _P]),
    "bounce_pair_histogram": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_double, C.c_int32, _P, _P]),
    "bounce_set_msd_reference": (C.c_int, [_P, _P]),
    "bounce_msd": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_double), _P]),
    "bounce_profile_steps": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "bounce_profile_breakdown": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P]),
    "bounce_autotune": (C.c_int, [_P, C.c_int32, _P, C.POINTER(bounce_tuning)]),
    "bounce_run_launch_count": (C.c_int64, [_P, C.c_int64, C.c_int32]),
    "bounce_pair_energy_noalloc": (C.c_int, [C.c_int32, _P, _P, _P, _P, C.c_int32, _P, _P, C.c_double, C.c_double,
                                             _P, _P, _P]),
    "bounce_last_error": (C.c_char_p, [_P]),
    "bounce_destroy": (None, [_P]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return sorted(_sig)


class BounceError(RuntimeError):
    pass


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Context:
    """One system on one GPU."""

    def __init__(self, *, dt=1.0, gamma=0.001, temperature=300.0, seed=0, r_on=4.0, r_off=5.0, r_cut=math.inf,
                 skin=1.0, ewald_beta=0.0, box=None, max_neighbors=2048, max_short=256, device=0, pme_grid=None,
                 pme_order=5, respa_m=2, jump_coulomb=True, pair_bounds=False, respa_m2=3, pair_skin=0.0, step_kernel=0):
        cfg = bounce_config()
        bounce_config_default(C.byref(cfg))
        cfg.dt_fs, cfg.gamma_per_fs, cfg.temperature_K, cfg.seed = dt, gamma, temperature, seed
        cfg.r_on, cfg.r_off, cfg.r_cut, cfg.skin, cfg.ewald_beta = r_on, r_off, r_cut, skin, ewald_beta
        cfg.periodic = 0 if box is None else 1
        if box is not None:
            cfg.box[0], cfg.box[1], cfg.box[2] = [float(x) for x in box]
        cfg.max_neighbors, cfg.max_short, cfg.device = max_neighbors, max_short, device
        if pme_grid is not None:
            cfg.pme_grid[0], cfg.pme_grid[1], cfg.pme_grid[2] = [int(k) for k in pme_grid]
        cfg.pme_order, cfg.respa_m = pme_order, respa_m
        cfg.jump_coulomb = 1 if jump_coulomb else 0
        cfg.pair_bounds = 1 if pair_bounds else 0
        cfg.respa_m2 = respa_m2
        cfg.pair_skin = pair_skin
        cfg.step_kernel = step_kernel
        self.cfg = cfg
        h = C.c_void_p()
        r = bounce_create(C.byref(h), C.byref(cfg))
        if r != OK:
            raise BounceError("bounce_create failed: %s" % ERR.get(r, r))
        self.h = h
        self.n = 0
        self.n_types = 0

    def _check(self, r, what):
        if r != OK:
            msg = bounce_last_error(self.h)
            raise BounceError("%s: %s (%s)" % (what, ERR.get(r, r), msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "h", None):
            bounce_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- set-up
    def set_topology(self, type, mass, charge, molecule, bonds=None, bond_k_r0=None, angles=None, angle_k_t0=None):
        n = len(type)
        t = _host(type, np.int32)
        m = _host(mass, np.float64)
        q = _host(charge, np.float64)
        mol = _host(molecule, np.int32)
        b = _host(bonds if bonds is not None else np.zeros((0, 2)), np.int32).reshape(-1, 2)
        bk = _host(bond_k_r0 if bond_k_r0 is not None else np.zeros((0, 2)), np.float64).reshape(-1, 2)
        a = _host(angles if angles is not None else np.zeros((0, 3)), np.int32).reshape(-1, 3)
        ak = _host(angle_k_t0 if angle_k_t0 is not None else np.zeros((0, 2)), np.float64).reshape(-1, 2)
        self._keep = (t, m, q, mol, b, bk, a, ak)
        self._check(bounce_set_topology(self.h, n, _ptr(t), _ptr(m), _ptr(q), _ptr(mol), len(b), _ptr(b), _ptr(bk),
                                        len(a), _ptr(a), _ptr(ak)), "set_topology")
        self.n = n
        self.n_types = int(t.max()) + 1

    def set_replicas(self, atom_offsets, seeds):
        off = _host(atom_offsets, np.int32)
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        self._keep_rep = (off, sd)
        self._check(bounce_set_replicas(self.h, len(off) - 1, _ptr(off), _ptr(sd)), "set_replicas")

    def set_lj(self, sigma, eps):
        s = _host(sigma, np.float64)
        e = _host(eps, np.float64)
        self._check(bounce_set_lj(self.h, s.shape[0], _ptr(s), _ptr(e)), "set_lj")

    def set_state(self, q, v, step=0, stream=None):
        if hasattr(q, "data_ptr"):
            self._check(bounce_set_state(self.h, _ptr(q), _ptr(v), step, DEVICE, stream), "set_state")
        else:
            qq = _host(q, np.float64)
            vv = _host(v, np.float64)
            self._check(bounce_set_state(self.h, _ptr(qq), _ptr(vv), step, HOST, stream), "set_state")

    # ---- run / read
    def run(self, n_steps, integrator=BOUNCE, stream=None):
        self._check(bounce_run(self.h, int(n_steps), int(integrator), stream), "run")

    def pair_forward(self, q, q_type, sigma, eps, forces, stream=None):
        """Pair forces (into the device tensor `forces`) and pair energy at the
        device positions q (None: the current positions)."""
        qt = _host(q_type, np.float64)
        sg = _host(sigma, np.float64)
        ep = _host(eps, np.float64)
        e = C.c_double()
        self._check(bounce_pair_forward(self.h, None if q is None else _ptr(q), len(qt), _ptr(qt), _ptr(sg), _ptr(ep),
                                        _ptr(forces), C.byref(e), stream), "pair_forward")
        return e.value

    def pair_backward(self, q_type, sigma, eps, grad_forces, grad_energy, grad_pos, stream=None):
        """dL/dq into the device tensor grad_pos; returns host arrays
        (dL/dq_type, dL/dsigma, dL/deps)."""
        qt = _host(q_type, np.float64)
        sg = _host(sigma, np.float64)
        ep = _host(eps, np.float64)
        T = len(qt)
        gq, gs, ge = np.zeros(T), np.zeros(T * T), np.zeros(T * T)
        self._check(bounce_pair_backward(self.h, T, _ptr(qt), _ptr(sg), _ptr(ep), _ptr(grad_forces),
                                         float(grad_energy), _ptr(grad_pos), _ptr(gq), _ptr(gs), _ptr(ge), stream),
                    "pair_backward")
        return gq, gs.reshape(T, T), ge.reshape(T, T)

    def pair_histogram(self, type_a, type_b, r_max, n_bins, stream=None):
        h = np.zeros(int(n_bins), np.int64)
        self._check(bounce_pair_histogram(self.h, int(type_a), int(type_b), float(r_max), int(n_bins), _ptr(h),
                                          stream), "pair_histogram")
        return h

    def set_msd_reference(self, stream=None):
        self._check(bounce_set_msd_reference(self.h, stream), "set_msd_reference")

    def msd(self, type, stream=None):
        out = C.c_double()
        self._check(bounce_msd(self.h, int(type), C.byref(out), stream), "msd")
        return out.value

    def profile_steps(self, n_steps, integrator=BOUNCE, stream=None):
        """(summed step-kernel ms, step-kernel launches) over n_steps."""
        ms = C.c_double()
        nl = C.c_int64()
        self._check(bounce_profile_steps(self.h, int(n_steps), int(integrator), stream, C.byref(ms), C.byref(nl)),
                    "profile_steps")
        return ms.value, nl.value

    def profile_breakdown(self, n_steps, integrator=BOUNCE, stream=None):
        """Summed device ms and timed boundaries of (pairs, step kernel, row
        rebuild, cluster rebuild, SPME) over n_steps run as bounce_run does."""
        ms = np.zeros(5)
        groups = np.zeros(5, np.int64)
        self._check(bounce_profile_breakdown(self.h, int(n_steps), int(integrator), stream, _ptr(ms), _ptr(groups)),
                    "profile_breakdown")
        return dict(zip(("pairs", "step", "rows", "clusters", "pme"), ms)), groups

    def autotune(self, integrator=BOUNCE, stream=None):
        """Time the pair kernel's candidate launch shapes on the current state
        and keep the fastest; returns the choice."""
        t = bounce_tuning()
        self._check(bounce_autotune(self.h, int(integrator), stream, C.byref(t)), "autotune")
        return {k: getattr(t, k) for k, _ in bounce_tuning._fields_}

    def run_launch_count(self, n_steps, integrator=BOUNCE):
        return int(bounce_run_launch_count(self.h, int(n_steps), int(integrator)))

    def get_state(self, q_out=None, v_out=None, stream=None):
        if q_out is not None and hasattr(q_out, "data_ptr"):
            self._check(bounce_get_state(self.h, _ptr(q_out), _ptr(v_out), DEVICE, stream), "get_state")
            return q_out, v_out
        q = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        self._check(bounce_get_state(self.h, _ptr(q), _ptr(v), HOST, stream), "get_state")
        return q, v

    def energies(self, stream=None):
        e = bounce_energies()
        self._check(bounce_get_energies(self.h, C.byref(e), stream), "get_energies")
        return {k: getattr(e, k) for k, _ in bounce_energies._fields_}

    def reset_counters(self, stream=None):
        self._check(bounce_reset_counters(self.h, stream), "reset_counters")

    def bounds(self):
        T = self.n_types
        L = np.zeros(T * T)
        Ls = np.zeros(T)
        self._check(bounce_get_bounds(self.h, _ptr(L), _ptr(Ls)), "get_bounds")
        return L.reshape(T, T), Ls

    def gradient(self, part=GRAD_FULL):
        g = np.empty((self.n, 3))
        self._check(bounce_compute_gradient(self.h, part, _ptr(g), HOST, None), "compute_gradient")
        return g

    def jump_half(self, step, stream_id):
        M = np.zeros(self.n, np.int32)
        A = np.zeros(self.n, np.int32)
        self._check(bounce_jump_half(self.h, int(step), int(stream_id), _ptr(M), _ptr(A), HOST, None), "jump_half")
        return M, A

    def rows(self, capacity=None):
        if capacity is None:
            capacity = self.cfg.max_neighbors if math.isfinite(self.cfg.r_cut) else max(1, self.n - 1)
        cap = int(capacity)
        cnt = np.zeros(self.n, np.int32)
        rows = np.zeros((self.n, cap), np.int32)
        self._check(bounce_get_rows(self.h, _ptr(cnt), _ptr(rows), cap), "get_rows")
        return [rows[i, :min(cnt[i], cap)].astype(np.int64) for i in range(self.n)]


NOALLOC_MAX_ATOMS = 16384


def pair_energy_noalloc(q, charge, type, molecule, sigma, eps, r_cut=math.inf, ewald_beta=0.0, box=None, out=None,
                        stream=None):
    """Coulomb and LJ pair-energy totals of a device-resident state, with no
    device allocation by the library: for callers that may not allocate
    (code inside an allocator that owns the device pool, hosts that forbid
    allocation after start-up).  q (n, 3) float64, charge (n,) float64,
    type and molecule (n,) int32, out (2,) float64: contiguous CUDA tensors
    owned by the caller, all on one device; sigma and eps are square
    (T, T) tables.  Raises ValueError on tensors the C entry point would
    misread; returns the library's status code (0 = ok)."""
    import torch
    ts = {"q": q, "charge": charge, "type": type, "molecule": molecule, "out": out}
    want = {"q": torch.float64, "charge": torch.float64, "type": torch.int32, "molecule": torch.int32,
            "out": torch.float64}
    for name, t in ts.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.dtype != want[name]:
            raise ValueError("%s must be %s, not %s" % (name, want[name], t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.device != q.device:
            raise ValueError("%s is on %s, q on %s" % (name, t.device, q.device))
    n = int(q.shape[0]) if q.dim() == 2 else -1
    if q.dim() != 2 or q.shape[1] != 3:
        raise ValueError("q must have shape (n, 3)")
    for name in ("charge", "type", "molecule"):
        if tuple(ts[name].shape) != (n,):
            raise ValueError("%s must have shape (%d,)" % (name, n))
    if tuple(out.shape) != (2,):
        raise ValueError("out must have shape (2,)")
    s = _host(sigma, np.float64)
    e = _host(eps, np.float64)
    if s.ndim != 2 or s.shape[0] != s.shape[1] or e.shape != s.shape:
        raise ValueError("sigma and eps must be square tables of one size")
    bx = None if box is None else _host(box, np.float64)
    if bx is not None and bx.shape != (3,):
        raise ValueError("box must hold 3 edges")
    with torch.cuda.device(q.device):
        return bounce_pair_energy_noalloc(n, _ptr(q), _ptr(charge), _ptr(type), _ptr(molecule), int(s.shape[0]),
                                          _ptr(s), _ptr(e), float(r_cut), float(ewald_beta),
                                          None if bx is None else _ptr(bx), _ptr(out), stream)


def from_system(sys, **kw):
    """Context for a paper_2002_07109_gb300.water.System."""
    if sys.box is not None:
        kw.setdefault("box", sys.box)
    ctx = Context(**kw)
    ctx.set_topology(sys.type, sys.mass, sys.charge, sys.molecule, sys.bonds, sys.bond_k_r0, sys.angles,
                     sys.angle_k_t0)
    ctx.set_lj(sys.lj_sigma, sys.lj_eps)
    return ctx


def pair_forces_function():
    """A torch.autograd.Function over bounce_pair_forward / bounce_pair_backward:
    apply(q, q_type, sigma, eps, ctx) -> (forces, energy) with q a CUDA
    float64 (n, 3) tensor and the parameters CPU float64 tensors; sigma and
    eps are symmetric tables whose gradients hold, at (a, b) and (b, a), the
    derivative with respect to the shared entry."""
    import torch

    class PairForces(torch.autograd.Function):
        @staticmethod
        def forward(fctx, q, q_type, sigma, eps, ctx):
            q = q.contiguous()
            F = torch.empty_like(q)
            stream = torch.cuda.current_stream(q.device).cuda_stream
            E = ctx.pair_forward(q, q_type.detach().numpy(), sigma.detach().numpy(), eps.detach().numpy(), F,
                                 stream=stream)
            fctx.save_for_backward(q_type, sigma, eps)
            fctx.bctx = ctx
            return F, torch.tensor(E, dtype=torch.float64)

        @staticmethod
        def backward(fctx, gF, gE):
            q_type, sigma, eps = fctx.saved_tensors
            gF = torch.zeros_like(gF) if gF is None else gF.contiguous()
            gpos = torch.empty_like(gF)
            stream = torch.cuda.current_stream(gF.device).cuda_stream
            gq, gs, ge = fctx.bctx.pair_backward(q_type.detach().numpy(), sigma.detach().numpy(),
                                                 eps.detach().numpy(), gF, 0.0 if gE is None else float(gE), gpos,
                                                 stream=stream)
            return (gpos, torch.from_numpy(gq), torch.from_numpy(gs), torch.from_numpy(ge), None)

    return PairForces
