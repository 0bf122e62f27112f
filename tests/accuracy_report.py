"""Accuracy report of the CUDA path against the FP64 oracle (run on a GPU).

Prints one JSON object with, per workload and precision, the median and
maximum relative error per target of a, j, T and Phi (|d|/|ref|,
||dT||_F/||T||_F) and of the adjoint gradients.  Workloads: the uniform
sphere N = 4096 (all targets), the Plummer sphere N = 2^17 (all active,
sampled targets), the turbulent cloud N = 2^20 at 1%, 10% and 100% active
(sampled targets), the oct-tree on the cloud against the oracle's tree
(sampled targets), the periodic box on a 48^3 lattice (sampled targets) and
the Plummer N = 2^16 adjoint (sampled rows).

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
from gpu_util import DEV, T, errors, run_eval  # noqa: E402


def stats(e):
    return {k: {"median": v[0], "max": v[1]} for k, v in e.items()}


def sample(idx, k, seed):
    return np.sort(ics.rng(seed).choice(idx, size=min(k, idx.size), replace=False)).astype(np.int32)


def main():
    rep = {"device": torch.cuda.get_device_name(0), "oracle_threads": O.max_threads()}
    pos, vel, mass = ics.uniform_sphere(4096, seed=ics.BASE_SEED + 0)
    ref = O.eval_active(pos, vel, mass, h=0.01)
    rows = np.arange(4096)
    for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
        out = run_eval(pos, vel, mass, None, h=0.01, precision=prec)
        rep[f"uniform_sphere_N4096_{name}"] = stats(errors(out, ref, rows))

    pos, vel, mass = ics.plummer(1 << 17, seed=ics.BASE_SEED + 1)
    rows = sample(np.arange(mass.size), 512, 1)
    ref = O.eval_active(pos, vel, mass, rows, h=1e-3)
    for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
        out = run_eval(pos, vel, mass, None, h=1e-3, precision=prec)
        rep[f"plummer_N131072_{name}_512_sampled"] = stats(errors(out, ref, rows))

    pos, vel, mass = ics.turbulent_cloud(1 << 20, seed=ics.BASE_SEED + 2)
    n = mass.size
    for frac in (0.01, 0.1, 1.0):
        idx = ics.active_subset(n, frac, ics.BASE_SEED + 5)
        rows = sample(idx, 384, 2)
        ref = O.eval_active(pos, vel, mass, rows, h=2e-3)
        out = run_eval(pos, vel, mass, idx, h=2e-3, precision=grav.MIXED)
        rep[f"cloud_N1048576_active{frac}_mixed_384_sampled"] = stats(errors(out, ref, rows))
        if frac == 0.01:
            out = run_eval(pos, vel, mass, idx, h=2e-3, precision=grav.F64)
            rep[f"cloud_N1048576_active{frac}_f64_384_sampled"] = stats(errors(out, ref, rows))

    # oct-tree (Theta = 0.5, leaves of 8) against the oracle's tree walk
    from test_gpu_periodic import run_periodic
    from test_gpu_tree import gpu_tree
    pos, vel, mass = ics.turbulent_cloud(1 << 20, seed=ics.BASE_SEED + 2)
    rows = sample(np.arange(mass.size), 128, 4)
    ref = O.tree_eval(pos, vel, mass, rows, h=2e-3, theta=0.5, leaf_size=8)
    for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
        out = gpu_tree(pos, vel, mass, h=2e-3, theta=0.5, leaf=8, precision=prec)
        rep[f"tree_cloud_N1048576_{name}_128_sampled"] = stats(errors(out, ref, rows))

    # periodic box (nearest image), 48^3 Zeldovich-shaped lattice, all targets
    pos, vel, mass = ics.zeldovich_box(48, 1.0, amplitude=0.8)
    rows = sample(np.arange(mass.size), 256, 5)
    ref = O.eval_active(pos, vel, mass, rows, h=2e-3, box=1.0)
    for name, prec in (("f64", grav.F64), ("mixed", grav.MIXED)):
        out = run_periodic(pos, vel, mass, None, 2e-3, 1.0, prec)
        rep[f"periodic_lattice_48cubed_{name}_256_sampled"] = stats(errors(out, ref, rows))

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
    print(json.dumps(rep, indent=1))


if __name__ == "__main__":
    main()
