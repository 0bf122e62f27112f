"""Tile-shape autotuner for the force kernels.

Times every tile configuration libgrav offers (threads per CTA, targets per
thread, sources per tile, accumulator placement, unroll depth) on the
caller's own inputs with CUDA events, and remembers the fastest per device,
precision, boundary mode (open or periodic box), potential on or off, launch
kind (single system or batched) and size class in a JSON cache next to the
built library.  Only timing happens here; every
configuration computes the same sums.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import grav
from .build import BUILD

CACHE = os.path.join(BUILD, "autotune.json")
_lock = threading.Lock()


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def shape_key(precision: int, kind: str, n_src: int, n_targets: int, device=None, *,
              periodic: bool = False, pot: bool = False) -> str:
    """Device, precision, boundary mode, potential, launch kind and log2 size
    classes of sources and targets (the periodic and potential kernels are
    separate instantiations with their own timings)."""
    name = torch.cuda.get_device_name(device)
    ls = int(math.log2(max(n_src, 1)))
    lt = int(math.log2(max(n_targets, 1)))
    mode = "periodic" if periodic else "open"
    return (f"{name}|{'mixed' if precision == grav.MIXED else 'f64'}|{mode}|"
            f"{'pot' if pot else 'nopot'}|{kind}|src2^{ls}|tgt2^{lt}")


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_eval(params: grav.Params, pos, vel, mass, idx, n_idx: int, *, systems=None, reps: int = 3,
              use_cache: bool = True):
    """Fastest tile configuration for this workload; returns (index, {index: ms})."""
    precision = params.precision
    kind = "batched" if systems is not None else "single"
    key = shape_key(precision, kind, mass.numel(), n_idx, pos.device, periodic=params.box > 0.0,
                    pot=bool(params.want_pot))
    if use_cache:
        with _lock:
            hit = _load().get(key)
        if hit is not None:
            return int(hit["best"]), {int(k): v for k, v in hit["ms"].items()}
    n = mass.numel()
    acc = torch.empty(n, 3, dtype=torch.float64, device=pos.device)
    jerk = torch.empty_like(acc)
    tid = torch.empty(n, 6, dtype=torch.float64, device=pos.device)
    pot = torch.empty(n, dtype=torch.float64, device=pos.device) if params.want_pot else None
    ms = {}
    for cfg in range(grav.lib().grav_tile_config_count(precision)):
        p = grav.Params(params.G, params.h, params.eta, precision, params.want_pot, cfg,
                        params.max_split, params.box)
        ws = grav.Workspace()
        if systems is not None:
            fn = lambda: grav.eval_batched(p, systems, pos, vel, mass, idx, None, n_idx, acc, jerk,
                                           tid, pot, None, workspace=ws)
        else:
            fn = lambda: grav.eval_active(p, pos, vel, mass, idx, None, n_idx, acc, jerk, tid, pot,
                                          None, workspace=ws)
        ms[cfg] = _time(fn, reps)
    best = min(ms, key=ms.get)
    with _lock:
        cache = _load()
        cache[key] = {"best": best, "ms": {str(k): v for k, v in ms.items()}}
        _store(cache)
    return best, ms
