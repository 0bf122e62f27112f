"""The tile-shape autotuner (autotune.tune_eval), single-system and batched.

The test checks three things:
- the configuration it returns is a valid index for the precision;
- its JSON cache round-trips, so the second call is a hit that times
  nothing;
- a launch with the tuned configuration matches a default launch.  The match
  is bit for bit when both use the same configuration, and within the mixed
  bounds otherwise.

The cache goes to a temporary file, never the library's own.
"""
import numpy as np
import pytest
import torch

from paper_2010_13792_gb300 import autotune, grav, ics

from gpu_util import DEV, MIXED_MAX, T, errors

pytestmark = pytest.mark.gpu


def _single_inputs():
    pos, vel, mass = ics.uniform_sphere(6000, seed=ics.BASE_SEED + 0)
    idx = np.sort(ics.rng(71).choice(mass.size, 3000, replace=False)).astype(np.int32)
    return pos, vel, mass, idx


def _batched_inputs():
    pos, vel, mass, offsets, sizes, act = ics.batched_systems(6, 500, 4000, seed=72, frac_lo=0.1,
                                                              frac_hi=0.6)
    idx = np.concatenate([a + o for a, o in zip(act, offsets)]).astype(np.int32)
    systems = np.stack([offsets, sizes], axis=1).astype(np.int64)
    return pos, vel, mass, idx, systems


def _run(p, P, V, M, idx, systems=None):
    n = M.numel()
    outs = [torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV),
            torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV),
            torch.full((n, 6), np.nan, dtype=torch.float64, device=DEV)]
    I = T(idx, torch.int32)
    if systems is None:
        grav.eval_active(p, P, V, M, I, None, idx.size, *outs)
    else:
        grav.eval_batched(p, grav.systems_table(systems, device=DEV), P, V, M, I, None, idx.size,
                          *outs)
    torch.cuda.synchronize()
    return {k: t.cpu().numpy() for k, t in zip(("acc", "jerk", "tidal"), outs)}


@pytest.mark.parametrize("kind", ["single", "batched"])
@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_tune_eval_valid_cached_and_consistent(kind, precision, tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    if kind == "single":
        pos, vel, mass, idx = _single_inputs()
        systems = None
        h = 0.01
    else:
        pos, vel, mass, idx, systems = _batched_inputs()
        h = 1e-3
    P, V, M = T(pos), T(vel), T(mass)
    p = grav.params(h=h, precision=precision)
    sys_t = grav.systems_table(systems, device=DEV) if systems is not None else None
    best, ms = autotune.tune_eval(p, P, V, M, T(idx, torch.int32), idx.size, systems=sys_t, reps=2)
    count = grav.lib().grav_tile_config_count(precision)
    assert 0 <= best < count
    assert sorted(ms) == list(range(count))
    assert all(np.isfinite(v) and v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())

    # the second call is a cache hit: it must time nothing
    def no_timing(*a, **k):
        raise AssertionError("cache miss: tune_eval timed again")
    monkeypatch.setattr(autotune, "_time", no_timing)
    best2, ms2 = autotune.tune_eval(p, P, V, M, T(idx, torch.int32), idx.size, systems=sys_t)
    assert best2 == best and ms2 == ms

    # a different boundary mode or potential setting is a different entry
    key = autotune.shape_key(precision, kind, mass.size, idx.size, DEV)
    assert key != autotune.shape_key(precision, kind, mass.size, idx.size, DEV, periodic=True)
    assert key != autotune.shape_key(precision, kind, mass.size, idx.size, DEV, pot=True)

    tuned = _run(grav.params(h=h, precision=precision, tile_config=best, max_split=1), P, V, M, idx,
                 systems)
    default_cfg = grav.default_tile_config(precision, idx.size)
    same = _run(grav.params(h=h, precision=precision, tile_config=best, max_split=1), P, V, M, idx,
                systems)
    dflt = _run(grav.params(h=h, precision=precision, tile_config=-1, max_split=1), P, V, M, idx,
                systems)
    for k in tuned:
        assert np.array_equal(tuned[k][idx], same[k][idx]), k
    ref = {k: v[idx] for k, v in dflt.items()}
    if best == default_cfg and systems is None:
        for k in tuned:
            assert np.array_equal(tuned[k][idx], dflt[k][idx]), k
    e = errors(tuned, ref, idx)
    tol = 1e-12 if precision == grav.F64 else MIXED_MAX
    for k in ("acc", "jerk", "tidal"):
        assert e[k][1] <= tol, (k, e[k])
