"""Gradients through the autograd Function (adjoint kernel) against the
oracle's adjoint and central finite differences of the FP64 forward."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics
from paper_2010_13792_gb300.autograd import gravity

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def loss_and_grad(pos, mass, w, h, precision):
    P = torch.tensor(pos, dtype=torch.float64, device=DEV, requires_grad=True)
    M = torch.tensor(mass, dtype=torch.float64, device=DEV, requires_grad=True)
    W_ = torch.tensor(w, dtype=torch.float64, device=DEV)
    acc, W = gravity(P, M, h=h, precision=precision)
    L = (W_ * (acc * acc).sum(1)).sum() + W
    L.backward()
    return float(L.item()), P.grad.cpu().numpy(), M.grad.cpu().numpy()


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_gradient_vs_oracle(precision):
    n, h = 2048, 0.05
    pos, vel, mass = ics.plummer(n, seed=80)
    w = ics.rng(81).uniform(0, 1, n)
    L, gp, gm = loss_and_grad(pos, mass, w, h, precision)
    o = O.eval_active(pos, vel, mass, h=h)
    pb, mb = O.backward(pos, mass, 2 * w[:, None] * o["acc"], 1.0, o["acc"], o["tidal"], o["pot"], h=h)
    L_o = float((w * (o["acc"] ** 2).sum(1)).sum()) + O.potential_energy(mass, o["pot"])
    tol = 1e-11 if precision == grav.F64 else 1e-4
    assert abs(L - L_o) <= tol * abs(L_o)
    ep = np.linalg.norm(gp - pb, axis=1) / np.linalg.norm(pb, axis=1)
    em = np.abs(gm - mb) / np.abs(mb)
    assert np.median(ep) <= tol and np.max(ep) <= 10 * tol, (np.median(ep), np.max(ep))
    assert np.median(em) <= tol and np.max(em) <= 10 * tol, (np.median(em), np.max(em))


def test_gradient_vs_finite_differences_plummer_2e16():
    """Plummer N = 2^16, L = sum w |a|^2 + W: adjoint gradient (FP64 and mixed)
    against central differences of the FP64 GPU loss (step 1e-6) and against
    the oracle's adjoint on sampled rows."""
    n, h = 1 << 16, 1e-3
    pos, vel, mass = ics.plummer(n, seed=ics.BASE_SEED + 3)
    w = ics.rng(82).uniform(0, 1, n)
    L, gp, gm = loss_and_grad(pos, mass, w, h, grav.F64)
    _, gp32, gm32 = loss_and_grad(pos, mass, w, h, grav.MIXED)
    g = ics.rng(83)
    rows = np.sort(g.choice(n, 24, replace=False)).astype(np.int32)
    o = O.eval_active(pos, vel, mass, h=h)
    pb, mb = O.backward(pos, mass, 2 * w[:, None] * o["acc"], 1.0, o["acc"], o["tidal"], o["pot"],
                        h=h, rows=rows)
    ep = np.linalg.norm(gp[rows] - pb[rows], axis=1) / np.linalg.norm(pb[rows], axis=1)
    assert ep.max() <= 1e-10, ep.max()
    ep32 = np.linalg.norm(gp32[rows] - pb[rows], axis=1) / np.linalg.norm(pb[rows], axis=1)
    assert np.median(ep32) <= 1e-5 and ep32.max() <= 1e-3, (np.median(ep32), ep32.max())
    em = np.abs(gm[rows] - mb[rows]) / np.abs(mb[rows])
    assert em.max() <= 1e-10
    eps = 1e-6
    with torch.no_grad():
        def L_of(p_np, m_np):
            acc, W = gravity(torch.tensor(p_np, device=DEV), torch.tensor(m_np, device=DEV), h=h,
                             precision=grav.F64)
            return float(((torch.tensor(w, device=DEV) * (acc * acc).sum(1)).sum() + W).item())
        for k, c in zip(g.integers(0, n, 4), g.integers(0, 3, 4)):
            pp, pm = pos.copy(), pos.copy()
            pp[k, c] += eps
            pm[k, c] -= eps
            fd = (L_of(pp, mass) - L_of(pm, mass)) / (2 * eps)
            assert abs(fd - gp[k, c]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gp).max()), (fd, gp[k, c])
