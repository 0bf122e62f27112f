"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
measure its error against the oracle per target (|da|/|a|, |dj|/|j|,
||dT||_F/||T||_F)."""
from __future__ import annotations

import numpy as np
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def T(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def run_eval(pos, vel, mass, idx=None, *, h, precision, G=1.0, eta=0.01, want_pot=True,
             tile_config=-1, max_split=0, device_count=True, fill=np.nan, flags=None,
             tensors=None):
    """Force evaluation at idx (None: all) on the GPU; returns numpy arrays
    indexed by element (rows of non-targets keep `fill`)."""
    n = mass.shape[0]
    P, V, M = (tensors if tensors is not None else (T(pos), T(vel), T(mass)))
    acc = torch.full((n, 3), fill, dtype=torch.float64, device=DEV)
    jerk = torch.full((n, 3), fill, dtype=torch.float64, device=DEV)
    tid = torch.full((n, 6), fill, dtype=torch.float64, device=DEV)
    pot = torch.full((n,), fill, dtype=torch.float64, device=DEV) if want_pot else None
    dtg = torch.full((n,), fill, dtype=torch.float64, device=DEV)
    p = grav.params(G=G, h=h, eta=eta, precision=precision, want_pot=want_pot,
                    tile_config=tile_config, max_split=max_split)
    if idx is None:
        grav.eval_active(p, P, V, M, None, None, n, acc, jerk, tid, pot, dtg, flags=flags)
    else:
        it = T(idx, torch.int32)
        cnt = T(np.array([idx.size]), torch.int32) if device_count else None
        grav.eval_active(p, P, V, M, it, cnt, idx.size, acc, jerk, tid, pot, dtg, flags=flags)
    torch.cuda.synchronize()
    out = {"acc": acc.cpu().numpy(), "jerk": jerk.cpu().numpy(), "tidal": tid.cpu().numpy(),
           "dt_grav": dtg.cpu().numpy()}
    if want_pot:
        out["pot"] = pot.cpu().numpy()
    return out


def rel_err(gpu, ref):
    """Per-row relative error |d|/|ref| (vectors) or |d|/|ref| (scalars)."""
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    if ref.ndim == 1:
        return np.abs(gpu - ref) / np.abs(ref)
    return np.linalg.norm(gpu - ref, axis=1) / np.linalg.norm(ref, axis=1)


def errors(out, ref, rows):
    """Error statistics of GPU rows `rows` against oracle slots 0..len(rows):
    (median, max) of |d|/|ref| per target (||dT||_F / ||T||_F for T)."""
    e = {}
    for k in ("acc", "jerk", "tidal", "pot", "dt_grav"):
        if k in out and k in ref and ref[k] is not None:
            if k == "tidal":
                r = tidal_norm(out[k][rows] - ref[k]) / tidal_norm(ref[k])
            else:
                r = rel_err(out[k][rows], ref[k])
            e[k] = (float(np.median(r)), float(np.max(r)))
    return e


# BASELINE tolerances: FP64 path <= 1e-12 relative; mixed path median <= 1e-5
# and max <= 1e-4 on |a|, max <= 1e-4 on j and T.
F64_TOL = 1e-12
MIXED_A_MEDIAN = 1e-5
MIXED_MAX = 1e-4


def assert_f64(e, keys=("acc", "jerk", "tidal", "pot")):
    for k in keys:
        if k in e:
            assert e[k][1] <= F64_TOL, (k, e[k])


def assert_mixed(e):
    assert e["acc"][0] <= MIXED_A_MEDIAN, ("acc median", e["acc"])
    assert e["acc"][1] <= MIXED_MAX, ("acc max", e["acc"])
    assert e["jerk"][1] <= MIXED_MAX, ("jerk max", e["jerk"])
    assert e["tidal"][1] <= MIXED_MAX, ("tidal max", e["tidal"])
    if "pot" in e:
        assert e["pot"][1] <= MIXED_MAX, ("pot max", e["pot"])


def tidal_norm(t6):
    """||T||_F of [n, 6] tidal tensors (off-diagonal components twice)."""
    t6 = np.asarray(t6)
    return np.sqrt((t6[:, :3] ** 2).sum(1) + 2.0 * (t6[:, 3:] ** 2).sum(1))


def tree_accel_norm(pos, vel, mass, h):
    """|a_i| of every element from the oracle's oct-tree (Theta = 0.5), a
    cheap estimate used only to rank candidates for the worst-conditioned
    targets (the conditioning's |a_i| is small where |a_i| is)."""
    return np.linalg.norm(O.tree_eval(pos, vel, mass, None, h=h, theta=0.5, leaf_size=8,
                                      want_pot=False)["acc"], axis=1)


def stratified_rows(pos, vel, mass, idx, h, a_est, *, seed, worst=512, total=4096, pool=2048,
                    box=0.0):
    """Rows of a full-size parity check, stratified on the conditioning
    kappa_i = sum_j |a_ij| / |a_i| (the error metric's conditioning): the
    `worst` targets of idx with the largest kappa among the `pool` targets of
    idx with the smallest estimated |a_i| (a_est, by element), plus targets
    drawn at random from the rest of idx up to `total`.  Returns (rows,
    ref, kappa): sorted element indices, the oracle at those rows and, per
    row, kappa of a, j and T (sums of pair magnitudes over |a|, |j|, ||T||)."""
    idx = np.asarray(idx, np.int64)
    if idx.size <= total:
        rows = idx.astype(np.int32)
    else:
        cand = np.sort(idx[np.argsort(a_est[idx], kind="stable")[:pool]]).astype(np.int32)
        ref_c = O.eval_active(pos, vel, mass, cand, h=h, box=box)
        kap_c = O.conditioning(pos, vel, mass, cand, h=h, box=box)[:, 0] / \
            np.linalg.norm(ref_c["acc"], axis=1)
        hard = cand[np.argsort(kap_c, kind="stable")[-worst:]]
        rest = np.setdiff1d(idx, hard)
        rnd = ics.rng(seed).choice(rest, size=total - hard.size, replace=False)
        rows = np.sort(np.concatenate([hard, rnd])).astype(np.int32)
    ref = O.eval_active(pos, vel, mass, rows, h=h, box=box)
    cond = O.conditioning(pos, vel, mass, rows, h=h, box=box)
    kappa = np.stack([cond[:, 0] / np.linalg.norm(ref["acc"], axis=1),
                      cond[:, 1] / np.linalg.norm(ref["jerk"], axis=1),
                      cond[:, 2] / tidal_norm(ref["tidal"])], axis=1)
    return rows, ref, kappa


def error_table(out, ref, rows, kappa):
    """Per quantity: median and max relative error over the rows, with the
    conditioning kappa of the row of the max and the largest kappa."""
    tab = {}
    for k, col in (("acc", 0), ("jerk", 1), ("tidal", 2)):
        if k == "tidal":
            r = tidal_norm(out[k][rows] - ref[k]) / tidal_norm(ref[k])
        else:
            r = rel_err(out[k][rows], ref[k])
        w = int(np.argmax(r))
        tab[k] = {"median": float(np.median(r)), "max": float(r.max()),
                  "kappa_at_max": float(kappa[w, col]), "kappa_max": float(kappa[:, col].max())}
    return tab


def assert_table(tab, precision):
    """The stated bounds on an error_table."""
    if precision == grav.F64:
        for k, v in tab.items():
            assert v["max"] <= F64_TOL, (k, v)
        return
    assert tab["acc"]["median"] <= MIXED_A_MEDIAN, ("acc median", tab["acc"])
    for k, v in tab.items():
        assert v["max"] <= MIXED_MAX, (k, v)
