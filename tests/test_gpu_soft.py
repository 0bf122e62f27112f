"""Adaptive softening on the GPU against the oracle: the support solve (h,
Omega, zeta against the oracle's own solve), the force sums with per-element
supports and the correction term (FP64 element by element to 1e-12, mixed to
the mixed tolerances), every tile configuration, target subsets, the
no-convergence flag, and at 2^20 elements the constraint residual of sampled
supports and sampled force rows."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics

from gpu_util import DEV, T, assert_f64, assert_mixed, errors  # noqa: E402

pytestmark = pytest.mark.gpu


def gpu_solve(pos, mass, h0, n_ngb, tol=1e-12, max_iter=100):
    n = mass.size
    h = T(np.broadcast_to(np.asarray(h0, np.float64), (n,)).copy())
    zeta, omega = T(np.full(n, np.nan)), T(np.full(n, np.nan))
    iters = torch.full((n,), -7, dtype=torch.int32, device=DEV)
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    grav.soft_solve(grav.soft_params(n_ngb=n_ngb, tol=tol, max_iter=max_iter), T(pos), T(mass), h,
                    zeta, omega, iters, flags)
    torch.cuda.synchronize()
    return {"h": h.cpu().numpy(), "zeta": zeta.cpu().numpy(), "omega": omega.cpu().numpy(),
            "iters": iters.cpu().numpy(), "flags": int(flags.item())}


def gpu_eval_soft(pos, vel, mass, h, zeta, idx, precision, tile_config=-1):
    n = mass.size
    acc = torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV)
    jerk, tid = acc.clone(), torch.full((n, 6), np.nan, dtype=torch.float64, device=DEV)
    pot = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
    dtg = pot.clone()
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    p = grav.params(h=1.0, precision=precision, want_pot=True, tile_config=tile_config)
    it = None if idx is None else T(idx, torch.int32)
    cnt = None if idx is None else T(np.array([idx.size]), torch.int32)
    grav.eval_soft(p, T(pos), T(vel), T(mass), T(h), None if zeta is None else T(zeta), it, cnt,
                   n if idx is None else idx.size, acc, jerk, tid, pot, dtg, flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    return {"acc": acc.cpu().numpy(), "jerk": jerk.cpu().numpy(), "tidal": tid.cpu().numpy(),
            "pot": pot.cpu().numpy(), "dt_grav": dtg.cpu().numpy()}


@pytest.fixture(scope="module")
def plummer_solved():
    pos, vel, mass = ics.plummer(3001, seed=91)
    ref = O.soft_solve(pos, mass, 0.05, n_ngb=32.0, tol=1e-12, max_iter=100)
    assert ref["converged"]
    return pos, vel, mass, ref


def test_solve_matches_oracle(plummer_solved):
    pos, vel, mass, ref = plummer_solved
    got = gpu_solve(pos, mass, 0.05, 32.0)
    assert got["flags"] == 0
    assert np.all(got["iters"] >= 0)
    np.testing.assert_allclose(got["h"], ref["h"], rtol=1e-10, atol=0)
    np.testing.assert_allclose(got["omega"], ref["omega"], rtol=1e-8, atol=0)
    np.testing.assert_allclose(got["zeta"], ref["zeta"], rtol=1e-8, atol=0)


def test_solve_from_far_guesses_and_unequal_masses():
    """Guesses far too small and far too large, masses spanning a factor 10."""
    pos, vel, mass = ics.uniform_sphere(1500, seed=92)
    mass = mass * ics.rng(93).uniform(0.3, 3.0, mass.size)
    h0 = np.where(np.arange(1500) % 2 == 0, 1e-4, 5.0)
    ref = O.soft_solve(pos, mass, h0, n_ngb=24.0, tol=1e-12, max_iter=200)
    got = gpu_solve(pos, mass, h0, 24.0, max_iter=200)
    assert ref["converged"] and got["flags"] == 0
    np.testing.assert_allclose(got["h"], ref["h"], rtol=1e-10, atol=0)
    np.testing.assert_allclose(got["zeta"], ref["zeta"], rtol=1e-8, atol=0)


def test_solve_flags_no_convergence():
    """A lone element can never gather n_ngb neighbours: its support grows
    until the iteration limit, which is reported, not hung on."""
    pos = np.zeros((1, 3))
    got = gpu_solve(pos, np.ones(1), 0.1, 32.0, max_iter=20)
    assert got["flags"] & grav.FLAG_NOCONVERGE
    assert got["iters"][0] == -1
    assert np.isfinite(got["h"][0]) and got["h"][0] > 0.1


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
@pytest.mark.parametrize("with_zeta", [True, False])
def test_eval_soft_all_targets(plummer_solved, precision, with_zeta):
    pos, vel, mass, ref_s = plummer_solved
    z = ref_s["zeta"] if with_zeta else None
    ref = O.eval_soft(pos, vel, mass, ref_s["h"], z)
    out = gpu_eval_soft(pos, vel, mass, ref_s["h"], z, None, precision)
    (assert_f64 if precision == grav.F64 else assert_mixed)(errors(out, ref, np.arange(mass.size)))


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_eval_soft_target_subset(plummer_solved, precision):
    pos, vel, mass, ref_s = plummer_solved
    idx = ics.active_subset(mass.size, 0.2, 94)
    ref = O.eval_soft(pos, vel, mass, ref_s["h"], ref_s["zeta"], idx)
    out = gpu_eval_soft(pos, vel, mass, ref_s["h"], ref_s["zeta"], idx, precision)
    (assert_f64 if precision == grav.F64 else assert_mixed)(errors(out, ref, idx))
    rest = np.setdiff1d(np.arange(mass.size), idx)
    assert np.all(np.isnan(out["acc"][rest]))


@pytest.mark.parametrize("cfg", range(24))
def test_every_mixed_config_soft(cfg):
    if cfg >= grav.lib().grav_tile_config_count(grav.MIXED):
        pytest.skip("no such tile configuration")
    pos, vel, mass = ics.turbulent_cloud(2500, seed=95, grid=32)
    h, zeta = ics.soft_inputs(pos, 0.08, seed=96)
    idx = ics.active_subset(mass.size, 0.5, 97)
    ref = O.eval_soft(pos, vel, mass, h, zeta, idx)
    out = gpu_eval_soft(pos, vel, mass, h, zeta, idx, grav.MIXED, tile_config=cfg)
    assert_mixed(errors(out, ref, idx))


@pytest.mark.parametrize("cfg", range(3))
def test_every_f64_config_soft(cfg):
    pos, vel, mass = ics.turbulent_cloud(2500, seed=95, grid=32)
    h, zeta = ics.soft_inputs(pos, 0.08, seed=96)
    ref = O.eval_soft(pos, vel, mass, h, zeta)
    out = gpu_eval_soft(pos, vel, mass, h, zeta, None, grav.F64, tile_config=cfg)
    assert_f64(errors(out, ref, np.arange(mass.size)))


def _density_residual(pos, mass, h, n_ngb, rows):
    """(4 pi/3) h^3 sum_j m_j W(r_ij, h) / (n_ngb m_i) - 1 at rows, W from its
    definition (numpy, FP64)."""
    out = []
    for i in rows:
        r = np.linalg.norm(pos - pos[i], axis=1)
        u = r / h[i]
        w = np.where(u < 0.5, 1 - 6 * u**2 + 6 * u**3, np.where(u < 1.0, 2 * (1 - u) ** 3, 0.0))
        rho = float((mass * 8.0 / (np.pi * h[i] ** 3) * w).sum())
        out.append(4.0 * np.pi / 3.0 * h[i] ** 3 * rho / (n_ngb * mass[i]) - 1.0)
    return np.array(out)


def test_solve_2e20_constraint_sampled():
    """2^20 elements of the turbulent cloud: every support converges and
    sampled supports satisfy the constraint (brute-force sums)."""
    pos, vel, mass = ics.turbulent_cloud(1 << 20)
    got = gpu_solve(pos, mass, 2e-2, 32.0)
    assert got["flags"] == 0 and np.all(got["iters"] >= 0)
    rows = ics.rng(98).choice(mass.size, 48, replace=False)
    res = _density_residual(pos, mass, got["h"], 32.0, rows)
    assert np.all(np.abs(res) <= 1e-10), np.abs(res).max()
    assert np.all(np.isfinite(got["zeta"])) and np.all(got["omega"] > 0)


@pytest.mark.parametrize("precision", [grav.MIXED, grav.F64])
def test_eval_soft_2e20_sampled(precision):
    """2^20 elements, seeded supports and coefficients, sampled rows."""
    pos, vel, mass = ics.turbulent_cloud(1 << 20)
    h, zeta = ics.soft_inputs(pos, 4e-3)
    frac = 1.0 if precision == grav.MIXED else 0.01
    idx = ics.active_subset(mass.size, frac, 99)
    out = gpu_eval_soft(pos, vel, mass, h, zeta, idx, precision)
    rows = np.sort(ics.rng(100).choice(idx, 64, replace=False)).astype(np.int32)
    ref = O.eval_soft(pos, vel, mass, h, zeta, rows)
    (assert_f64 if precision == grav.F64 else assert_mixed)(errors(out, ref, rows))
