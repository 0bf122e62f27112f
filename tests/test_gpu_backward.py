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
    tol = 1e-12 if precision == grav.F64 else 1e-4
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
        tol = 1e-12 if precision == grav.F64 else 1e-4
        assert np.median(rel_err(pb, pb_o)) <= tol / 10
        assert np.max(rel_err(pb, pb_o)) <= tol * 10


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_backward_batched_per_system(precision):
    """grav_eval_backward_batched over systems at their own supports: Plummer
    systems at h = 1e-3 and uniform spheres at h = 0.01, one system at the
    call's h (system h = 0).  One system is left out of the table, so its
    elements belong to no system and must stay unwritten.  Each system equals
    grav_eval_backward on it alone (max_split = 1) bit for bit, and the
    oracle's adjoint at the single-system tolerances."""
    pos, vel, mass, offsets, sizes, act = ics.batched_systems(9, 200, 3000, seed=66)
    n = mass.size
    h_sys = np.where(np.arange(9) % 2 == 0, 1e-3, 0.01)
    h_sys[3] = 0.0
    h_call = 0.03
    keep = [s for s in range(9) if s != 6]
    table = grav.systems_table(np.stack([offsets[keep], sizes[keep]], 1), h_sys[keep], device=DEV)
    w = ics.rng(67).uniform(0, 1, n)
    fwd = {k: np.zeros((n,) + sh) for k, sh in (("acc", (3,)), ("tidal", (6,)), ("pot", ()))}
    for s in range(9):
        sl = slice(offsets[s], offsets[s] + sizes[s])
        hs = h_sys[s] if h_sys[s] > 0 else h_call
        r = O.eval_active(pos[sl], vel[sl], mass[sl], h=hs)
        for k in fwd:
            fwd[k][sl] = r[k]
    a_bar = 2 * w[:, None] * fwd["acc"]
    pb = torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV)
    mb = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    p = grav.params(h=h_call, precision=precision)
    grav.eval_backward_batched(p, table, T(pos), T(mass), T(a_bar), 1.0, T(fwd["acc"]),
                               T(fwd["tidal"]), T(fwd["pot"]), pb, mb, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    pb, mb = pb.cpu().numpy(), mb.cpu().numpy()
    tol = 1e-12 if precision == grav.F64 else 1e-4
    for s in range(9):
        sl = slice(offsets[s], offsets[s] + sizes[s])
        if s == 6:
            assert np.all(np.isnan(pb[sl])) and np.all(np.isnan(mb[sl]))
            continue
        hs = h_sys[s] if h_sys[s] > 0 else h_call
        args = (pos[sl], mass[sl], a_bar[sl], 1.0, fwd["acc"][sl], fwd["tidal"][sl], fwd["pot"][sl])
        pb1, mb1 = gpu_backward(*args, hs, precision, max_split=1)
        assert np.array_equal(pb[sl], pb1), s
        assert np.array_equal(mb[sl], mb1), s
        pb_o, mb_o = O.backward(*args, h=hs)
        _, mb_sums = O.backward(pos[sl], mass[sl], a_bar[sl], 0.0, fwd["acc"][sl], fwd["tidal"][sl],
                                fwd["pot"][sl], h=hs)
        ep = np.linalg.norm(pb[sl] - pb_o, axis=1) / (np.linalg.norm(pb_o, axis=1) + 1e-300)
        em = np.abs(mb[sl] - mb_o) / (np.abs(mb_sums) + np.abs(fwd["pot"][sl]) + 1e-300)
        assert np.max(ep) <= tol, (s, float(np.max(ep)))
        assert np.max(em) <= tol, (s, float(np.max(em)))


def test_backward_batched_rejects_bad_system():
    pos, vel, mass, offsets, sizes, act = ics.batched_systems(4, 200, 500, seed=68)
    n = mass.size
    h_sys = np.array([0.0, -1.0, 0.0, 0.0])
    table = grav.systems_table(np.stack([offsets, sizes], 1), h_sys, device=DEV)
    a_bar = ics.rng(69).normal(size=(n, 3))
    z3, z6 = np.zeros((n, 3)), np.zeros((n, 6))
    pb = torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV)
    mb = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    grav.eval_backward_batched(grav.params(h=0.02, precision=grav.F64), table, T(pos), T(mass),
                               T(a_bar), 0.0, T(z3), T(z6), T(np.zeros(n)), pb, mb, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) & grav.FLAG_BADINDEX
    sl = slice(offsets[1], offsets[1] + sizes[1])
    assert np.all(np.isnan(pb.cpu().numpy()[sl]))
    assert np.all(np.isfinite(pb.cpu().numpy()[:offsets[1]]))
