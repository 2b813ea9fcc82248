"""GPU parity of the differentiable pair forces (force matching) against the
FP64 oracle's autograd gradients, through the C ABI and the
torch.autograd.Function binding: a small periodic box, and the full
force-matching workload (4,096 water molecules in a periodic box, Ewald
direct erfc beta 0.35 and LJ within 9 A; target forces from sigma +2 %,
epsilon -5 % and charges x 0.98).

Tolerance: the rule of every FP32 sum in these tests -- the error of each
result against the sum of the magnitudes of the FP32 terms it adds up
(tests/diff_scales.py), 1e-5: forces per atom, and the backward given the
oracle's own upstream gradient dL/dF (dL/dq per atom through the pair
Hessian, and each parameter gradient).  Through the autograd binding the
upstream gradient 2 (F - F_target) is formed from the GPU's FP32 forces,
whose error (within the force tolerance) the small differences F - F_target
amplify; that propagated error is added to the scale of the end-to-end
check.  The full-size case also checks the GPU loss gradient against central
finite differences of the GPU loss itself (h = 1e-4; 1e-2 for epsilon, in
which the loss is quadratic) on sampled coordinates and on every parameter,
within three standard deviations of the rounding noise of the FP32 loss."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

from diff_scales import scales
from oracle.diff import _pairs, force_matching_loss
from paper_2002_07109_gb300.water import water_box

TOL = 1e-5
QT = np.array([-0.834, 0.417])
SIG = np.array([[3.15, 0.0], [0.0, 0.0]])
EPS = np.array([[0.152, 0.0], [0.0, 0.0]])


def _case(n_side, seed, r_cut):
    s = water_box(n_side, seed=seed)
    beta, w_e = 0.35, 0.5
    # target forces from perturbed parameters: sigma +2 %, eps -5 %, charges x 0.98
    _, F_t, *_ = force_matching_loss(s.q, s.type, s.molecule, 0.98 * QT, 1.02 * SIG, 0.95 * EPS,
                                     np.zeros_like(s.q), r_cut, beta, s.box)
    ref = force_matching_loss(s.q, s.type, s.molecule, QT, SIG, EPS, F_t, r_cut, beta, s.box, w_energy=w_e)
    ii, jj = _pairs(s.q, s.molecule, r_cut, s.box)
    u = 2.0 * (ref[1] - F_t)
    sc = scales(s.q, s.type, QT, SIG, EPS, ii, jj, beta, s.box, u, w_e)
    # end to end: u from GPU forces within TOL * (force scale) of the oracle's
    sc_e2e = scales(s.q, s.type, QT, SIG, EPS, ii, jj, beta, s.box, u, w_e, du_in=2.0 * TOL * sc[0])
    ctx = bounce.from_system(s, seed=1, r_on=4.0, r_off=5.0, r_cut=r_cut, ewald_beta=beta, skin=1.0,
                             max_neighbors=1024)
    ctx.set_state(s.q, s.v)
    return s, F_t, ref, sc, sc_e2e, ctx, w_e


def _gpu_loss(ctx, s, q, qt, sig, eps, F_t, w_e):
    dev = torch.device("cuda", 0)
    tq = torch.tensor(q, dtype=torch.float64, device=dev, requires_grad=True)
    tqt = torch.tensor(qt, dtype=torch.float64, requires_grad=True)
    tsig = torch.tensor(sig, dtype=torch.float64, requires_grad=True)
    teps = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    F, E = bounce.pair_forces_function().apply(tq, tqt, tsig, teps, ctx)
    loss = ((F - torch.tensor(F_t, device=dev)) ** 2).sum() + w_e * E.to(dev)
    loss.backward()
    return (float(loss.detach()), F.detach().cpu().numpy(), float(E.detach()), tq.grad.cpu().numpy(), tqt.grad.numpy(),
            tsig.grad.numpy(), teps.grad.numpy())


def _check(got, ref, sc):
    L, F, E, gq, gqt, gs, ge = got
    _, F_ref, E_ref, gq_ref, gqt_ref, gs_ref, ge_ref = ref
    fs, qs, sq, ss, se = sc
    dF = np.linalg.norm(F - F_ref, axis=1) / fs
    assert dF.max() < TOL, ("forces", dF.max())
    dq = np.linalg.norm(gq - gq_ref, axis=1) / qs
    assert dq.max() < TOL, ("dL/dq", dq.max())
    assert np.all(np.abs(gqt - gqt_ref) < TOL * sq), ("dL/dq_type", gqt, gqt_ref, sq)
    assert abs(gs[0, 0] - gs_ref[0, 0]) < TOL * ss[0, 0], ("dL/dsigma", gs[0, 0], gs_ref[0, 0], ss[0, 0])
    assert abs(ge[0, 0] - ge_ref[0, 0]) < TOL * se[0, 0], ("dL/deps", ge[0, 0], ge_ref[0, 0], se[0, 0])
    return dF.max(), dq.max()


def _backward_given_u(ctx, s, ref, F_t, w_e):
    """The GPU backward with the oracle's own upstream gradient dL/dF =
    2 (F_ref - F_t)."""
    dev = torch.device("cuda", 0)
    F = torch.empty((s.n_atoms, 3), dtype=torch.float64, device=dev)
    E = ctx.pair_forward(torch.tensor(s.q, dtype=torch.float64, device=dev), QT, SIG, EPS, F)
    u = torch.tensor(2.0 * (ref[1] - F_t), dtype=torch.float64, device=dev)
    gpos = torch.empty_like(u)
    gq, gs, ge = ctx.pair_backward(QT, SIG, EPS, u, w_e, gpos)
    return (None, F.cpu().numpy(), E, gpos.cpu().numpy(), gq, gs, ge)


def test_force_matching_gradients_match_oracle():
    s, F_t, ref, sc, sc_e2e, ctx, w_e = _case(6, 7, 8.0)
    _check(_backward_given_u(ctx, s, ref, F_t, w_e), ref, sc)
    for _ in range(2):     # twice: the backward reuses the forward's state
        got = _gpu_loss(ctx, s, s.q, QT, SIG, EPS, F_t, w_e)
        _check(got, ref, sc_e2e)
    ctx.close()


def test_force_matching_full_size():
    """4,096 molecules (12,288 atoms), box edge 49.7 A, r_c 9 A: every atom
    and every parameter against the oracle, and the GPU gradient against
    central differences of the GPU loss."""
    s, F_t, ref, sc, sc_e2e, ctx, w_e = _case(16, 7, 9.0)
    _check(_backward_given_u(ctx, s, ref, F_t, w_e), ref, sc)
    got = _gpu_loss(ctx, s, s.q, QT, SIG, EPS, F_t, w_e)
    _check(got, ref, sc_e2e)
    L0, gq, gqt, gs, ge = got[0], got[3], got[4], got[5], got[6]
    h = 1e-4
    rng = np.random.default_rng(3)

    def loss_at(q=s.q, qt=QT, sig=SIG, eps=EPS):
        dev = torch.device("cuda", 0)
        F = torch.empty((s.n_atoms, 3), dtype=torch.float64, device=dev)
        E = ctx.pair_forward(torch.tensor(q, dtype=torch.float64, device=dev), qt, sig, eps, F)
        Fh = F.cpu().numpy()
        return float(((Fh - F_t) ** 2).sum() + w_e * E)

    # the loss from FP32 forces is noisy: a rounding error of ~1e-6 |F| per
    # force component moves it by 2 (F - F_t) dF, adding up like a random
    # walk over the components; the difference quotient divides that by 2h
    # (one standard deviation of it; the bound takes three)
    dF = got[1] - F_t
    noise = 3.0 * 2.0 * math.sqrt((dF ** 2).sum()) * 1e-6 * np.abs(got[1]).max() / (2 * h)
    for a in rng.choice(s.n_atoms, 3, replace=False):
        for c in range(3):
            qp = s.q.copy(); qp[a, c] += h
            qm = s.q.copy(); qm[a, c] -= h
            fd = (loss_at(q=qp) - loss_at(q=qm)) / (2 * h)
            assert abs(fd - gq[a, c]) < 1e-3 * abs(gq[a, c]) + noise, (a, c, fd, gq[a, c], noise)
    for t in range(2):
        p = QT.copy(); p[t] += h
        m = QT.copy(); m[t] -= h
        fd = (loss_at(qt=p) - loss_at(qt=m)) / (2 * h)
        assert abs(fd - gqt[t]) < 1e-3 * abs(gqt[t]) + noise, (t, fd, gqt[t])
    # the forces and the energy are linear in epsilon, so the loss is a
    # quadratic in it and the central difference is exact for any step: a
    # step of 1e-2 divides the rounding noise by 100
    for name, tab, g, hp in (("sigma", SIG, gs, h), ("eps", EPS, ge, 1e-2)):
        p = tab.copy(); p[0, 0] += hp
        m = tab.copy(); m[0, 0] -= hp
        fd = ((loss_at(sig=p) - loss_at(sig=m)) if name == "sigma" else (loss_at(eps=p) - loss_at(eps=m))) / (2 * hp)
        assert abs(fd - g[0, 0]) < 1e-3 * abs(g[0, 0]) + noise * h / hp, (name, fd, g[0, 0])
    ctx.close()
