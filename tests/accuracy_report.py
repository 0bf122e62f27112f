"""Accuracy report of the CUDA path against the FP64 oracle (run on a GPU).

Prints one JSON object with, per workload and precision, the median and
maximum relative error per target of a, j and T (|d|/|ref|,
||dT||_F/||T||_F), the conditioning kappa (sum of the pair magnitudes over
the magnitude of the sum) at the target of the maximum and the largest kappa
among the targets compared, and the adjoint gradients' errors; then checks
every row against the stated bounds (FP64 <= 1e-12; mixed median <= 1e-5
and max <= 1e-4 on |a|, max <= 1e-4 on j and T) and exits non-zero if one
is missed.  Workloads, each with the library's default tile configuration:
  - uniform sphere, N = 4096, every target;
  - Plummer sphere, N = 2^17, every element active, and the turbulent cloud,
    N = 2^20, 1%, 10% and 100% active: 4096 targets each, the 512 worst
    conditioned (largest kappa of a among the 2048 with the smallest
    oracle-tree |a|) plus 3584 at random;
  - the oct-tree on the cloud against the oracle's tree walk (sampled);
  - periodic boxes: the exact 8^3 and 6^3 lattices and the 48^3 pancake
    lattice, every target;
  - the adjoint on the Plummer sphere N = 2^16 (sampled rows).

    python tests/accuracy_report.py > accuracy.json
"""
import json
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from oracle import oracle as O  # noqa: E402
from paper_2010_13792_gb300 import grav, ics  # noqa: E402
from gpu_util import (F64_TOL, MIXED_A_MEDIAN, MIXED_MAX, T, error_table, run_eval,  # noqa: E402
                      stratified_rows, tree_accel_norm)


def sample(idx, k, seed):
    return np.sort(ics.rng(seed).choice(idx, size=min(k, idx.size), replace=False)).astype(np.int32)


def all_rows(pos, vel, mass, h, box=0.0):
    n = mass.size
    rows = np.arange(n, dtype=np.int32)
    ref = O.eval_active(pos, vel, mass, h=h, box=box)
    cond = O.conditioning(pos, vel, mass, h=h, box=box)
    tn = np.sqrt((ref["tidal"][:, :3] ** 2).sum(1) + 2 * (ref["tidal"][:, 3:] ** 2).sum(1))
    kappa = np.stack([cond[:, 0] / np.linalg.norm(ref["acc"], axis=1),
                      cond[:, 1] / np.linalg.norm(ref["jerk"], axis=1), cond[:, 2] / tn], axis=1)
    return rows, ref, kappa


def check(rep):
    bad = []
    for name, tab in rep.items():
        if not isinstance(tab, dict) or "acc" not in tab:
            continue
        tol = F64_TOL if "_f64" in name else MIXED_MAX
        for k in ("acc", "jerk", "tidal"):
            if tab[k]["max"] > tol:
                bad.append((name, k, tab[k]["max"]))
        if "_mixed" in name and tab["acc"]["median"] > MIXED_A_MEDIAN:
            bad.append((name, "acc median", tab["acc"]["median"]))
    return bad


def main():
    from test_gpu_periodic import run_periodic
    from test_gpu_tree import gpu_tree
    rep = {"device": torch.cuda.get_device_name(0), "oracle_threads": O.max_threads()}
    pos, vel, mass = ics.uniform_sphere(4096, seed=ics.BASE_SEED + 0)
    rows, ref, kappa = all_rows(pos, vel, mass, 0.01)
    for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
        out = run_eval(pos, vel, mass, None, h=0.01, precision=prec)
        rep[f"uniform_sphere_N4096_{name}_all"] = error_table(out, ref, rows, kappa)

    pos, vel, mass = ics.plummer(1 << 17, seed=ics.BASE_SEED + 1)
    a_est = tree_accel_norm(pos, vel, mass, 1e-3)
    rows, ref, kappa = stratified_rows(pos, vel, mass, np.arange(mass.size), 1e-3, a_est, seed=31)
    for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
        out = run_eval(pos, vel, mass, None, h=1e-3, precision=prec)
        rep[f"plummer_N131072_{name}_4096_stratified"] = error_table(out, ref, rows, kappa)

    pos, vel, mass = ics.turbulent_cloud(1 << 20, seed=ics.BASE_SEED + 2)
    n = mass.size
    a_est = tree_accel_norm(pos, vel, mass, 2e-3)
    for frac in (0.01, 0.1, 1.0):
        idx = ics.active_subset(n, frac, 40 + int(frac * 100))
        rows, ref, kappa = stratified_rows(pos, vel, mass, idx, 2e-3, a_est, seed=41)
        out = run_eval(pos, vel, mass, idx, h=2e-3, precision=grav.MIXED)
        rep[f"cloud_N1048576_active{frac}_mixed_4096_stratified"] = error_table(out, ref, rows, kappa)
        if frac == 0.01:
            out = run_eval(pos, vel, mass, idx, h=2e-3, precision=grav.F64)
            rep[f"cloud_N1048576_active{frac}_f64_4096_stratified"] = \
                error_table(out, ref, rows, kappa)

    # oct-tree (Theta = 0.5, leaves of 8) against the oracle's tree walk
    rows = sample(np.arange(n), 128, 4)
    ref = O.tree_eval(pos, vel, mass, rows, h=2e-3, theta=0.5, leaf_size=8)
    ones = np.ones((rows.size, 3))
    for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
        out = gpu_tree(pos, vel, mass, h=2e-3, theta=0.5, leaf=8, precision=prec)
        rep[f"tree_cloud_N1048576_{name}_128_sampled"] = error_table(out, ref, rows, ones)

    # periodic boxes (nearest image), every target
    for tag, (p_, v_, m_), L, h in (
            ("lattice_8cubed", ics.zeldovich_box(8, 1.0, amplitude=0.0, jitter=0.0), 1.0, 0.02),
            ("lattice_6cubed", ics.zeldovich_box(6, 0.3, amplitude=0.0, jitter=0.0), 0.3, 0.02),
            ("pancake_48cubed", ics.zeldovich_box(48, 1.0, amplitude=0.8), 1.0, 2e-3)):
        rows, ref, kappa = all_rows(p_, v_, m_, h, box=L)
        for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
            out = run_periodic(p_, v_, m_, None, h, L, prec)
            rep[f"periodic_{tag}_{name}_all"] = error_table(out, ref, rows, kappa)

    from paper_2010_13792_gb300.autograd import gravity
    pos, vel, mass = ics.plummer(1 << 16, seed=ics.BASE_SEED + 3)
    w = ics.rng(82).uniform(0, 1, mass.size)
    rows = sample(np.arange(mass.size), 96, 3)
    o = O.eval_active(pos, vel, mass, h=1e-3)
    pb, mb = O.backward(pos, mass, 2 * w[:, None] * o["acc"], 1.0, o["acc"], o["tidal"], o["pot"],
                        h=1e-3, rows=rows)
    for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
        P = T(pos).requires_grad_(True)
        M = T(mass).requires_grad_(True)
        acc, W = gravity(P, M, h=1e-3, precision=prec)
        L = (T(w) * (acc * acc).sum(1)).sum() + W
        L.backward()
        gp, gm = P.grad.cpu().numpy()[rows], M.grad.cpu().numpy()[rows]
        ep = np.linalg.norm(gp - pb[rows], axis=1) / np.linalg.norm(pb[rows], axis=1)
        em = np.abs(gm - mb[rows]) / np.abs(mb[rows])
        rep[f"plummer_N65536_adjoint_{name}_96_sampled"] = {
            "pos_grad": {"median": float(np.median(ep)), "max": float(ep.max())},
            "mass_grad": {"median": float(np.median(em)), "max": float(em.max())}}
    bad = check(rep)
    rep["bounds_missed"] = bad
    print(json.dumps(rep, indent=1))
    if bad:
        sys.exit(1)


if __name__ == "__main__":
    main()
