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


# Adjoint tolerances (the paper has no adjoint; these restate the forward
# bounds for its gradient).  Per element, the position gradient is compared
# relative to its own norm.  The mass gradient is compared relative to
# |sum of the pair part| + |w_bar Phi|, because its two parts can nearly
# cancel.  Bounds:
#   FP64:  max <= 1e-12, as for the forward;
#   mixed: median <= 1e-5 and max <= 1e-4.
F64_ADJ = 1e-12
MIXED_ADJ_MEDIAN, MIXED_ADJ_MAX = 1e-5, 1e-4


def _adjoint_errors(gp, gm, pb, mb, mb_pairs, pot, rows):
    ep = np.linalg.norm(gp[rows] - pb[rows], axis=1) / np.linalg.norm(pb[rows], axis=1)
    em = np.abs(gm[rows] - mb[rows]) / (np.abs(mb_pairs[rows]) + np.abs(pot[rows]))
    return ep, em


def _assert_adjoint(ep, em, precision):
    if precision == grav.F64:
        assert ep.max() <= F64_ADJ and em.max() <= F64_ADJ, (ep.max(), em.max())
    else:
        for e in (ep, em):
            assert np.median(e) <= MIXED_ADJ_MEDIAN and e.max() <= MIXED_ADJ_MAX, \
                (np.median(e), e.max())


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_gradient_vs_oracle(precision):
    n, h = 2048, 0.05
    pos, vel, mass = ics.plummer(n, seed=80)
    w = ics.rng(81).uniform(0, 1, n)
    L, gp, gm = loss_and_grad(pos, mass, w, h, precision)
    o = O.eval_active(pos, vel, mass, h=h)
    a_bar = 2 * w[:, None] * o["acc"]
    pb, mb = O.backward(pos, mass, a_bar, 1.0, o["acc"], o["tidal"], o["pot"], h=h)
    _, mb_pairs = O.backward(pos, mass, a_bar, 0.0, o["acc"], o["tidal"], o["pot"], h=h)
    L_o = float((w * (o["acc"] ** 2).sum(1)).sum()) + O.potential_energy(mass, o["pot"])
    assert abs(L - L_o) <= (F64_ADJ if precision == grav.F64 else MIXED_ADJ_MAX) * abs(L_o)
    ep, em = _adjoint_errors(gp, gm, pb, mb, mb_pairs, o["pot"], np.arange(n))
    _assert_adjoint(ep, em, precision)


def test_gradient_vs_finite_differences_plummer_2e16():
    """Plummer N = 2^16, L = sum w |a|^2 + W.  The adjoint gradients (FP64
    and mixed) are checked two ways:
    - against the oracle's adjoint on 64 sampled rows, at the bounds above;
    - against central differences of the FP64 GPU loss, step 1e-6, on 64
      random coordinates and on 64 random masses.

    L is quadratic in each mass (a is linear in it, W bilinear), so the
    mass differences are exact up to rounding.  The position differences
    carry O(step^2) truncation.  Each difference carries the loss's
    rounding, about 1e-16 |L| / step in absolute terms.  So both adjoints
    are held to 1e-5 of max(|fd|, 1e-3 max|g|), and the mixed one also to
    the mixed bound against the FP64 one."""
    n, h = 1 << 16, 1e-3
    pos, vel, mass = ics.plummer(n, seed=ics.BASE_SEED + 3)
    w = ics.rng(82).uniform(0, 1, n)
    L, gp, gm = loss_and_grad(pos, mass, w, h, grav.F64)
    _, gp32, gm32 = loss_and_grad(pos, mass, w, h, grav.MIXED)
    g = ics.rng(83)
    rows = np.sort(g.choice(n, 64, replace=False)).astype(np.int32)
    o = O.eval_active(pos, vel, mass, h=h)
    a_bar = 2 * w[:, None] * o["acc"]
    pb, mb = O.backward(pos, mass, a_bar, 1.0, o["acc"], o["tidal"], o["pot"], h=h, rows=rows)
    _, mb_pairs = O.backward(pos, mass, a_bar, 0.0, o["acc"], o["tidal"], o["pot"], h=h, rows=rows)
    for gpx, gmx, prec in ((gp, gm, grav.F64), (gp32, gm32, grav.MIXED)):
        ep, em = _adjoint_errors(gpx, gmx, pb, mb, mb_pairs, o["pot"], rows)
        _assert_adjoint(ep, em, prec)

    eps = 1e-6
    W_ = torch.tensor(w, device=DEV)
    with torch.no_grad():
        def L_of(p_np, m_np):
            acc, W = gravity(torch.tensor(p_np, device=DEV), torch.tensor(m_np, device=DEV), h=h,
                             precision=grav.F64)
            return float(((W_ * (acc * acc).sum(1)).sum() + W).item())
        ks, cs = g.choice(n, 64, replace=False), g.integers(0, 3, 64)
        gscale = np.abs(gp).max()
        for k, c in zip(ks, cs):
            pp, pm = pos.copy(), pos.copy()
            pp[k, c] += eps
            pm[k, c] -= eps
            fd = (L_of(pp, mass) - L_of(pm, mass)) / (2 * eps)
            tol = 1e-5 * max(abs(fd), 1e-3 * gscale)
            assert abs(fd - gp[k, c]) <= tol, ("pos", k, c, fd, gp[k, c])
            assert abs(fd - gp32[k, c]) <= tol + MIXED_ADJ_MAX * abs(gp[k, c]), ("pos", k, c, fd, gp32[k, c])
        mscale = np.abs(gm).max()
        for k in g.choice(n, 64, replace=False):
            mp, mm = mass.copy(), mass.copy()
            mp[k] += eps
            mm[k] -= eps
            fd = (L_of(pos, mp) - L_of(pos, mm)) / (2 * eps)
            tol = 1e-5 * max(abs(fd), 1e-3 * mscale)
            assert abs(fd - gm[k]) <= tol, ("mass", k, fd, gm[k])
            assert abs(fd - gm32[k]) <= tol + MIXED_ADJ_MAX * abs(gm[k]), ("mass", k, fd, gm32[k])
