"""Periodic box (nearest periodic image, the paper's Zeldovich setting) on the
GPU against the oracle, element by element: uniform and pancake-shaped
boxes, a small box in which tiles reach across half the box (per-pair
wrapping loop), lattices with pairs exactly at half a box, every tile
configuration, translation invariance and the batched launch."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics

from gpu_util import (DEV, MIXED_A_MEDIAN, MIXED_MAX, T, assert_f64, assert_mixed,  # noqa: E402
                      errors)

pytestmark = pytest.mark.gpu


def run_periodic(pos, vel, mass, idx, h, L, precision, tile_config=-1):
    n = mass.size
    acc = torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV)
    jerk, tid = acc.clone(), torch.full((n, 6), np.nan, dtype=torch.float64, device=DEV)
    pot = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
    dtg = pot.clone()
    p = grav.params(h=h, precision=precision, want_pot=True, box=L, tile_config=tile_config)
    if idx is None:
        grav.eval_active(p, T(pos), T(vel), T(mass), None, None, n, acc, jerk, tid, pot, dtg)
    else:
        grav.eval_active(p, T(pos), T(vel), T(mass), T(idx, torch.int32),
                         T(np.array([idx.size]), torch.int32), idx.size, acc, jerk, tid, pot, dtg)
    torch.cuda.synchronize()
    return {"acc": acc.cpu().numpy(), "jerk": jerk.cpu().numpy(), "tidal": tid.cpu().numpy(),
            "pot": pot.cpu().numpy(), "dt_grav": dtg.cpu().numpy()}


def _uniform_box(n, L, seed):
    g = ics.rng(seed)
    pos = g.uniform(0.0, L, (n, 3))
    pos = pos[ics.morton_order(pos)]
    return pos, g.normal(0.0, 1.0, (n, 3)), np.full(n, 1.0 / n)


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_uniform_box(precision):
    pos, vel, mass = _uniform_box(6000, 1.0, 81)
    ref = O.eval_active(pos, vel, mass, h=0.01, box=1.0)
    out = run_periodic(pos, vel, mass, None, 0.01, 1.0, precision)
    (assert_f64 if precision == grav.F64 else assert_mixed)(errors(out, ref, np.arange(6000)))


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_small_box_tiles_reach_across(precision):
    """1000 elements: each 256-source tile spans a large part of the box, so
    most tiles take the per-pair wrapping loop."""
    pos, vel, mass = _uniform_box(1000, 0.5, 82)
    idx = ics.active_subset(1000, 0.4, 83)
    ref = O.eval_active(pos, vel, mass, idx, h=0.03, box=0.5)
    out = run_periodic(pos, vel, mass, idx, 0.03, 0.5, precision)
    (assert_f64 if precision == grav.F64 else assert_mixed)(errors(out, ref, idx))


@pytest.mark.parametrize("cfg", range(24))
def test_every_mixed_config_periodic(cfg):
    if cfg >= grav.lib().grav_tile_config_count(grav.MIXED):
        pytest.skip("no such tile configuration")
    pos, vel, mass = ics.zeldovich_box(16, 1.0, amplitude=0.6)
    n = mass.size
    idx = ics.active_subset(n, 0.3, 84)
    ref = O.eval_active(pos, vel, mass, idx, h=0.02, box=1.0)
    out = run_periodic(pos, vel, mass, idx, 0.02, 1.0, grav.MIXED, tile_config=cfg)
    assert_mixed(errors(out, ref, idx))


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_zeldovich_64cubed_sampled(precision):
    """The paper's 64^3 pancake shape (one sinusoidal mode), sampled targets."""
    pos, vel, mass = ics.zeldovich_box(64, 1.0, amplitude=0.8)
    n = mass.size
    idx = ics.active_subset(n, 0.05 if precision == grav.F64 else 1.0, 85)
    out = run_periodic(pos, vel, mass, idx, 2e-3, 1.0, precision)
    rows = np.sort(ics.rng(86).choice(idx, 128, replace=False)).astype(np.int32)
    ref = O.eval_active(pos, vel, mass, rows, h=2e-3, box=1.0)
    (assert_f64 if precision == grav.F64 else assert_mixed)(errors(out, ref, rows))


def test_translation_invariance_on_gpu():
    pos, vel, mass = ics.zeldovich_box(20, 1.0, amplitude=0.5)
    a = run_periodic(pos, vel, mass, None, 0.01, 1.0, grav.MIXED)
    b = run_periodic(np.mod(pos + np.array([0.3, 0.71, -0.2]), 1.0), vel, mass, None, 0.01, 1.0,
                     grav.MIXED)
    e = np.linalg.norm(a["acc"] - b["acc"], axis=1) / np.linalg.norm(a["acc"], axis=1)
    assert np.median(e) < 1e-5 and e.max() < 1e-4


def test_batched_periodic_and_open_limit():
    pos, vel, mass = _uniform_box(3000, 1.0, 87)
    systems = np.array([[0, 1000], [1000, 2000]], np.int64)
    idx = np.arange(3000, dtype=np.int32)
    n = 3000
    acc = torch.zeros(n, 3, dtype=torch.float64, device=DEV)
    jerk, tid = torch.zeros_like(acc), torch.zeros(n, 6, dtype=torch.float64, device=DEV)
    p = grav.params(h=0.02, precision=grav.F64, box=1.0)
    grav.eval_batched(p, grav.systems_table(systems, device=DEV), T(pos), T(vel), T(mass), T(idx, torch.int32), None,
                      n, acc, jerk, tid)
    torch.cuda.synchronize()
    for off, ns in systems:
        sl = slice(off, off + ns)
        ref = O.eval_active(pos[sl], vel[sl], mass[sl], h=0.02, box=1.0)
        assert_f64(errors({"acc": acc.cpu().numpy()[sl], "jerk": jerk.cpu().numpy()[sl],
                           "tidal": tid.cpu().numpy()[sl]}, ref, np.arange(ns)))
    # a box far larger than the system equals open boundaries
    sp, sv, sm = ics.uniform_sphere(1500, seed=88)
    # (the oracle sees the same shifted, rounded coordinates)
    big = run_periodic(sp + 50.0, sv, sm, None, 0.02, 100.0, grav.F64)
    ref = O.eval_active(sp + 50.0, sv, sm, h=0.02)
    assert_f64(errors(big, ref, np.arange(1500)))


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
@pytest.mark.parametrize("n_side,L", [(8, 1.0), (6, 0.3)])
def test_exact_half_box_ties(n_side, L, precision):
    """A lattice without jitter: a large share of the pairs lie at (or within
    a rounding of) half a box along some axis, where the two images are
    equally near and rint's ties-to-even decides.  Both sides must pick the
    same image for every such pair: the force would otherwise differ by the
    difference of the two images' contributions.  The lattice's cubic
    symmetry cancels most of each tidal sum (sum_j ||T_ij|| / ||T_i|| is about
    500 on the 8^3 lattice), and the stated bounds hold all the same."""
    pos, vel, mass = ics.zeldovich_box(n_side, L, amplitude=0.0, jitter=0.0)
    ref = O.eval_active(pos, vel, mass, h=0.02, box=L)
    out = run_periodic(pos, vel, mass, None, 0.02, L, precision)
    e = errors(out, ref, np.arange(mass.size))
    if precision == grav.F64:
        assert_f64(e)
        return
    assert_mixed(e)
    # diagnostic: the error against the sum's own scale, sum_j ||T_ij||_F =
    # sum_j sqrt(6) m_j / r_ij^3 (no pair is softened here); a pair taken to
    # the other image would flip the sign of some off-diagonal terms, about
    # 1e-3 of that scale
    d = pos[None, :, :] - pos[:, None, :]
    d -= L * np.rint(d / L)
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    assert r.min() > 0.02
    scale = (np.sqrt(6.0) * mass[None, :] / r**3).sum(axis=1)
    dt = out["tidal"] - ref["tidal"]
    frob = np.sqrt((dt[:, :3] ** 2).sum(1) + 2.0 * (dt[:, 3:] ** 2).sum(1))
    assert (frob / scale).max() <= 1e-7, (frob / scale).max()


@pytest.fixture(scope="module")
def pancake48():
    """The pancake-shaped 48^3 lattice (one sinusoidal mode of amplitude 0.8,
    jitter 1% of the spacing) and the oracle at every element."""
    pos, vel, mass = ics.zeldovich_box(48, 1.0, amplitude=0.8)
    return pos, vel, mass, O.eval_active(pos, vel, mass, h=2e-3, box=1.0)


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_pancake_lattice_48cubed_every_target(pancake48, precision):
    """Every one of the 110592 targets of the 48^3 pancake lattice.  Where the
    lattice is locally undistorted its tidal tensor and jerk nearly cancel:
    sum_j ||T_ij|| / ||T_i|| reaches about 8000 here, and the mixed kernels'
    close field (FP64 nearest pairs, FP32 sums in short runs near the
    target) keeps T, j and a inside the stated bounds at those targets too."""
    pos, vel, mass, ref = pancake48
    out = run_periodic(pos, vel, mass, None, 2e-3, 1.0, precision)
    e = errors(out, ref, np.arange(mass.size))
    (assert_f64 if precision == grav.F64 else assert_mixed)(e)


def test_box_narrower_than_two_softenings_is_rejected():
    p = grav.params(h=0.3, box=0.5)
    assert grav.lib().grav_eval_workspace_bytes(p, 10, 10) == grav.GRAV_EINVAL
