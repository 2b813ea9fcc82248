"""GPU parity of the differentiable pair forces (force matching, BASELINE
config 5 shape on a smaller periodic box) against the FP64 oracle's autograd
gradients, through the C ABI and the torch.autograd.Function binding.

Tolerances: forces and position gradients against the summed magnitudes of
their FP32 pair terms (1e-5, the reading used for every FP32 sum); parameter
gradients within 1e-4 relative of the gradient vector's norm."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bounce = pytest.importorskip("paper_2002_07109_gb300.bounce")

from oracle.diff import force_matching_loss
from paper_2002_07109_gb300.water import water_box


def test_force_matching_gradients_match_oracle():
    s = water_box(6, seed=7)
    r_cut, beta = 8.0, 0.35
    qt = np.array([-0.834, 0.417])
    sig = np.array([[3.15, 0.0], [0.0, 0.0]])
    eps = np.array([[0.152, 0.0], [0.0, 0.0]])
    # target forces from perturbed parameters: sigma +2 %, eps -5 %, charges x 0.98
    _, F_t, *_ = force_matching_loss(s.q, s.type, s.molecule, 0.98 * qt, 1.02 * sig, 0.95 * eps, np.zeros_like(s.q),
                                     r_cut, beta, s.box)
    L, F_ref, E_ref, gq_ref, gqt_ref, gs_ref, ge_ref = force_matching_loss(
        s.q, s.type, s.molecule, qt, sig, eps, F_t, r_cut, beta, s.box, w_energy=0.5)
    from oracle.forcefield import Params, pair_energy_magnitudes
    from oracle.neighbors import rows, to_pairs
    ii, jj = to_pairs(rows(s.q, s.molecule, r_cut, s.box))
    sc, sl = pair_energy_magnitudes(s.q, s.charge, s.type, ii, jj,
                                    Params(r_cut=r_cut, ewald_beta=beta, box=s.box, lj_sigma=sig, lj_eps=eps))
    ctx = bounce.from_system(s, seed=1, r_on=4.0, r_off=5.0, r_cut=r_cut, ewald_beta=beta, skin=1.0)
    ctx.set_state(s.q, s.v)
    dev = torch.device("cuda", 0)
    q = torch.tensor(s.q, dtype=torch.float64, device=dev, requires_grad=True)
    tqt = torch.tensor(qt, dtype=torch.float64, requires_grad=True)
    tsig = torch.tensor(sig, dtype=torch.float64, requires_grad=True)
    teps = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    Fn = bounce.pair_forces_function()
    for call in range(2):
        F, E = Fn.apply(q, tqt, tsig, teps, ctx)
        loss = ((F - torch.tensor(F_t, device=dev)) ** 2).sum() + 0.5 * E.to(dev)
        for t in (q, tqt, tsig, teps):
            t.grad = None
        loss.backward()
        Fg = F.detach().cpu().numpy()
        # a sum of FP32 pair terms with heavy cancellation: against sum |W|
        assert abs(float(E) - E_ref) < 1e-6 * (sc + sl)
        d = np.linalg.norm(Fg - F_ref, axis=1)
        assert np.median(d / np.linalg.norm(F_ref, axis=1)) < 1e-5
        assert np.max(d) < 1e-4 * np.sqrt((F_ref ** 2).sum(1).mean())
        gq = q.grad.cpu().numpy()
        dq = np.linalg.norm(gq - gq_ref, axis=1)
        assert np.median(dq / np.linalg.norm(gq_ref, axis=1)) < 1e-4, np.median(dq / np.linalg.norm(gq_ref, axis=1))
        assert np.max(dq) < 1e-3 * np.sqrt((gq_ref ** 2).sum(1).mean())
        for got, ref in ((tqt.grad.numpy(), gqt_ref), (tsig.grad.numpy()[0, 0], gs_ref[0, 0]),
                         (teps.grad.numpy()[0, 0], ge_ref[0, 0])):
            assert np.linalg.norm(np.atleast_1d(got - ref)) < 1e-4 * np.linalg.norm(np.atleast_1d(ref)), (got, ref)
    ctx.close()
