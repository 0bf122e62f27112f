"""GPU adjoint (grav_eval_backward) against the oracle's adjoint sums and
against central finite differences of the loss L = sum w |a|^2 + W."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics

from gpu_util import DEV, T, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu


def gpu_backward(pos, mass, a_bar, w_bar, acc, tid, pot, h, precision, max_split=0):
    n = mass.size
    pb = torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV)
    mb = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
    p = grav.params(h=h, precision=precision, max_split=max_split)
    grav.eval_backward(p, T(pos), T(mass), None if a_bar is None else T(a_bar), w_bar, T(acc),
                       T(tid), T(pot), pb, mb)
    torch.cuda.synchronize()
    return pb.cpu().numpy(), mb.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 700, 4099])
@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_backward_vs_oracle(n, precision):
    pos, vel, mass = ics.plummer(n, seed=60 + n)
    h = 0.05
    ref = O.eval_active(pos, vel, mass, h=h)
    w = ics.rng(61).uniform(0, 1, n)
    a_bar = 2 * w[:, None] * ref["acc"]
    pb_o, mb_o = O.backward(pos, mass, a_bar, 1.0, ref["acc"], ref["tidal"], ref["pot"], h=h)
    pb, mb = gpu_backward(pos, mass, a_bar, 1.0, ref["acc"], ref["tidal"], ref["pot"], h, precision)
    tol = 1e-11 if precision == grav.F64 else 1e-4
    # error relative to each element's gradient scale; the mass gradient is
    # the sum of two terms, -G sum f (d . a_bar) and w_bar Phi, which can
    # nearly cancel (by 600x for one element here), so its error is taken
    # relative to the sum of their magnitudes
    _, mb_sums = O.backward(pos, mass, a_bar, 0.0, ref["acc"], ref["tidal"], ref["pot"], h=h)
    scale_p = np.linalg.norm(pb_o, axis=1) + 1e-300
    scale_m = np.abs(mb_sums) + np.abs(1.0 * ref["pot"]) + 1e-300
    ep = np.linalg.norm(pb - pb_o, axis=1) / scale_p
    em = np.abs(mb - mb_o) / scale_m
    assert np.max(ep) <= tol, float(np.max(ep))
    assert np.max(em) <= tol, (float(np.median(em)), float(np.max(em)))


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_backward_potential_only(precision):
    n = 500
    pos, vel, mass = ics.uniform_sphere(n, seed=62)
    ref = O.eval_active(pos, vel, mass, h=0.05)
    pb_o, mb_o = O.backward(pos, mass, None, 0.7, ref["acc"], ref["tidal"], ref["pot"], h=0.05)
    pb, mb = gpu_backward(pos, mass, None, 0.7, ref["acc"], ref["tidal"], ref["pot"], 0.05, precision)
    assert np.allclose(pb, pb_o, rtol=1e-14, atol=0)
    assert np.allclose(mb, mb_o, rtol=1e-14, atol=0)


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_backward_split_path(precision):
    n = 3000
    pos, vel, mass = ics.plummer(n, seed=63)
    ref = O.eval_active(pos, vel, mass, h=0.02)
    a_bar = ics.rng(64).normal(size=(n, 3))
    pb_o, mb_o = O.backward(pos, mass, a_bar, 0.0, ref["acc"], ref["tidal"], ref["pot"], h=0.02)
    for ms in (1, 8):
        pb, mb = gpu_backward(pos, mass, a_bar, 0.0, ref["acc"], ref["tidal"], ref["pot"], 0.02,
                              precision, max_split=ms)
        tol = 1e-11 if precision == grav.F64 else 1e-4
        assert np.median(rel_err(pb, pb_o)) <= tol / 10
        assert np.max(rel_err(pb, pb_o)) <= tol * 10
