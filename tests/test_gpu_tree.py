"""Oct-tree solver on the GPU against the oracle's tree: the same tree order
(bit for bit), the same number of nodes and interactions (every opening
decision taken the same way), a, j, T, Phi and dt_grav element by element
to the FP64 tolerance (and, for the mixed walk, to the mixed tolerances);
Theta = 0 against the direct sum; the relative criterion; degenerate
inputs; at 2^20 elements sampled rows and the accuracy against the direct
sum."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics

from gpu_util import DEV, T, assert_f64, assert_mixed, errors  # noqa: E402

pytestmark = pytest.mark.gpu


def gpu_tree(pos, vel, mass, idx=None, *, h, theta=0.5, leaf=8, alpha=0.0, a_old=None, G=1.0,
             precision=grav.F64):
    n = mass.size
    acc = torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV)
    jerk, tid = acc.clone(), torch.full((n, 6), np.nan, dtype=torch.float64, device=DEV)
    pot = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
    dtg = pot.clone()
    order = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    stats = torch.full((2,), -1, dtype=torch.int64, device=DEV)
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    p = grav.params(G=G, h=h, precision=precision, want_pot=True)
    tp = grav.tree_params(theta=theta, alpha=alpha, leaf_size=leaf)
    it = None if idx is None else T(idx, torch.int32)
    cnt = None if idx is None else T(np.array([idx.size]), torch.int32)
    grav.eval_tree(p, tp, T(pos), T(vel), T(mass), it, cnt, n if idx is None else idx.size, acc,
                   jerk, tid, pot, dtg, a_old=None if a_old is None else T(a_old), order=order,
                   stats=stats, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    return {"acc": acc.cpu().numpy(), "jerk": jerk.cpu().numpy(), "tidal": tid.cpu().numpy(),
            "pot": pot.cpu().numpy(), "dt_grav": dtg.cpu().numpy(), "order": order.cpu().numpy(),
            "n_nodes": int(stats[0].item()), "interactions": int(stats[1].item())}


@pytest.mark.parametrize("leaf", [1, 8, 32])
@pytest.mark.parametrize("theta", [0.3, 0.5, 0.8])
def test_tree_matches_oracle_tree(theta, leaf):
    pos, vel, mass = ics.plummer(5000, seed=111, sort=False)
    ref = O.tree_eval(pos, vel, mass, h=0.01, theta=theta, leaf_size=leaf)
    out = gpu_tree(pos, vel, mass, h=0.01, theta=theta, leaf=leaf)
    assert np.array_equal(out["order"], ref["order"])
    assert out["n_nodes"] == ref["n_nodes"]
    assert out["interactions"] == ref["interactions"]
    assert_f64(errors(out, ref, np.arange(5000)), keys=("acc", "jerk", "tidal", "pot", "dt_grav"))


def test_tree_target_subset_and_relative_criterion():
    pos, vel, mass = ics.turbulent_cloud(6000, seed=112, grid=32, sort=False)
    idx = ics.active_subset(6000, 0.3, 113)
    direct = O.eval_active(pos, vel, mass, h=0.005)
    a_old = direct["acc"]
    ref = O.tree_eval(pos, vel, mass, idx, h=0.005, theta=0.5, alpha=0.0025, a_old=a_old)
    out = gpu_tree(pos, vel, mass, idx, h=0.005, theta=0.5, alpha=0.0025, a_old=a_old)
    assert out["interactions"] == ref["interactions"]
    assert_f64(errors(out, ref, idx))
    rest = np.setdiff1d(np.arange(6000), idx)
    assert np.all(np.isnan(out["acc"][rest]))


def test_theta_zero_is_the_direct_sum():
    pos, vel, mass = ics.uniform_sphere(3000, seed=114)
    ref = O.eval_active(pos, vel, mass, h=0.02)
    out = gpu_tree(pos, vel, mass, h=0.02, theta=0.0)
    assert out["interactions"] == 3000 * 2999
    assert_f64(errors(out, ref, np.arange(3000)))


@pytest.mark.parametrize("case", ["single", "coincident", "two", "line"])
def test_degenerate_inputs(case):
    g = ics.rng(115)
    if case == "single":
        pos = np.zeros((1, 3))
    elif case == "coincident":              # zero extent: every key equal, one deep leaf
        pos = np.tile(np.array([[0.3, -0.2, 0.1]]), (50, 1))
    elif case == "two":
        pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, -0.25]])
    else:                                   # all on a line: flat in two axes
        pos = np.zeros((300, 3))
        pos[:, 0] = g.uniform(-1, 1, 300)
    n = pos.shape[0]
    vel = g.normal(size=(n, 3))
    mass = g.uniform(0.5, 1.5, n)
    ref = O.tree_eval(pos, vel, mass, h=0.05, theta=0.5, leaf_size=4)
    out = gpu_tree(pos, vel, mass, h=0.05, theta=0.5, leaf=4)
    assert np.array_equal(out["order"], ref["order"])
    assert out["interactions"] == ref["interactions"]
    for k in ("acc", "jerk", "tidal", "pot"):
        assert np.allclose(out[k], ref[k], rtol=1e-12, atol=1e-12 * max(1.0, np.abs(ref[k]).max())), k


def test_tree_2e20_sampled_and_accuracy():
    """2^20 elements of the turbulent cloud, every element a target: sampled
    rows against the oracle's tree (same decisions) and against the direct
    sum (monopole accuracy at Theta = 0.5)."""
    pos, vel, mass = ics.turbulent_cloud(1 << 20)
    out = gpu_tree(pos, vel, mass, h=2e-3, theta=0.5, leaf=8)
    rows = np.sort(ics.rng(116).choice(1 << 20, 64, replace=False)).astype(np.int32)
    ref = O.tree_eval(pos, vel, mass, rows, h=2e-3, theta=0.5, leaf_size=8)
    assert out["n_nodes"] == ref["n_nodes"]
    assert np.array_equal(out["order"], ref["order"])
    assert_f64(errors(out, ref, rows))
    direct = O.eval_active(pos, vel, mass, rows, h=2e-3)
    e = np.linalg.norm(out["acc"][rows] - direct["acc"], axis=1) / np.linalg.norm(direct["acc"], axis=1)
    assert np.median(e) < 5e-3 and e.max() < 5e-2, (np.median(e), e.max())
    assert out["interactions"] < 0.01 * (1 << 20) * (1 << 20)


@pytest.mark.parametrize("leaf", [8, 32])
def test_mixed_walk_matches_oracle_tree(leaf):
    pos, vel, mass = ics.plummer(5000, seed=117, sort=False)
    ref = O.tree_eval(pos, vel, mass, h=0.01, theta=0.5, leaf_size=leaf)
    out = gpu_tree(pos, vel, mass, h=0.01, theta=0.5, leaf=leaf, precision=grav.MIXED)
    assert out["interactions"] == ref["interactions"]
    assert_mixed(errors(out, ref, np.arange(5000)))


def test_mixed_walk_2e20_sampled():
    pos, vel, mass = ics.turbulent_cloud(1 << 20)
    idx = ics.active_subset(1 << 20, 0.5, 118)
    out = gpu_tree(pos, vel, mass, idx, h=2e-3, theta=0.5, leaf=8, precision=grav.MIXED)
    rows = np.sort(ics.rng(119).choice(idx, 64, replace=False)).astype(np.int32)
    ref = O.tree_eval(pos, vel, mass, rows, h=2e-3, theta=0.5, leaf_size=8)
    assert_mixed(errors(out, ref, rows))
