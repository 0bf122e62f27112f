"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
measure its error against the oracle per target (|da|/|a|, |dj|/|j|,
||dT||_F/||T||_F)."""
from __future__ import annotations

import numpy as np
import torch

from paper_2010_13792_gb300 import grav

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
    """Error statistics of GPU rows `rows` against oracle slots 0..len(rows)."""
    e = {}
    for k in ("acc", "jerk", "tidal", "pot", "dt_grav"):
        if k in out and k in ref and ref[k] is not None:
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
