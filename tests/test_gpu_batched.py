"""Batched force evaluation (many independent systems, one persistent launch)
against per-system grav_eval_active (bit-identical with max_split = 1) and
against the oracle, including the batch of 256 systems of BASELINE's
batching workload (sizes log-uniform in [512, 65536], 1-50% active)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics

from gpu_util import DEV, T, assert_f64, assert_mixed, errors  # noqa: E402

pytestmark = pytest.mark.gpu


def _packed(n_sys, n_min, n_max, seed, frac_lo=0.01, frac_hi=0.5):
    pos, vel, mass, offsets, sizes, act = ics.batched_systems(n_sys, n_min, n_max, seed=seed,
                                                              frac_lo=frac_lo, frac_hi=frac_hi)
    idx = np.concatenate([a + o for a, o in zip(act, offsets)]).astype(np.int32)
    systems = np.stack([offsets, sizes], axis=1).astype(np.int64)
    return pos, vel, mass, systems, idx, act


def _outputs(n):
    return (torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV),
            torch.full((n, 3), np.nan, dtype=torch.float64, device=DEV),
            torch.full((n, 6), np.nan, dtype=torch.float64, device=DEV),
            torch.full((n,), np.nan, dtype=torch.float64, device=DEV),
            torch.full((n,), np.nan, dtype=torch.float64, device=DEV))


def run_batched(pos, vel, mass, systems, idx, h, precision, device_count=True, tile_config=-1,
                flags=None, h_sys=None):
    n = mass.size
    acc, jerk, tid, pot, dtg = _outputs(n)
    p = grav.params(h=h, precision=precision, want_pot=True, tile_config=tile_config)
    cnt = T(np.array([idx.size]), torch.int32) if device_count else None
    grav.eval_batched(p, grav.systems_table(systems, h_sys, device=DEV), T(pos), T(vel), T(mass),
                      T(idx, torch.int32), cnt,
                      idx.size, acc, jerk, tid, pot, dtg, flags=flags)
    torch.cuda.synchronize()
    return {"acc": acc.cpu().numpy(), "jerk": jerk.cpu().numpy(), "tidal": tid.cpu().numpy(),
            "pot": pot.cpu().numpy(), "dt_grav": dtg.cpu().numpy()}


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_batched_equals_single_system_launches(precision):
    pos, vel, mass, systems, idx, act = _packed(24, 100, 5000, seed=91)
    h = 0.01
    out = run_batched(pos, vel, mass, systems, idx, h, precision)
    n = mass.size
    P, V, M = T(pos), T(vel), T(mass)
    for s, (off, ns) in enumerate(systems):
        sl = slice(off, off + ns)
        acc, jerk, tid, pot, dtg = _outputs(int(ns))
        p = grav.params(h=h, precision=precision, want_pot=True, max_split=1)
        li = T(act[s], torch.int32)
        grav.eval_active(p, P[sl].contiguous(), V[sl].contiguous(), M[sl].contiguous(), li, None,
                         act[s].size, acc, jerk, tid, pot, dtg)
        torch.cuda.synchronize()
        rows = act[s] + off
        for k, t in (("acc", acc), ("jerk", jerk), ("tidal", tid), ("pot", pot), ("dt_grav", dtg)):
            assert np.array_equal(out[k][rows], t.cpu().numpy()[act[s]]), (s, k)
    others = np.setdiff1d(np.arange(n), idx)
    assert np.all(np.isnan(out["acc"][others]))


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_batched_256_systems_vs_oracle(precision):
    """The batching workload: 256 systems, half Plummer half uniform, sizes
    log-uniform in [512, 65536], 1-50% of each active.  Every system, 16 of
    its targets: the 4 active targets nearest its centre of mass (where |a|
    is smallest and the sums cancel most) and 12 drawn at random."""
    pos, vel, mass, systems, idx, act = _packed(256, 512, 65536, seed=ics.BASE_SEED + 4)
    h = 1e-3
    out = run_batched(pos, vel, mass, systems, idx, h, precision)
    g = ics.rng(92)
    errs = {k: [] for k in ("acc", "jerk", "tidal", "pot")}
    for s in range(256):
        off, ns = systems[s]
        sl = slice(off, off + ns)
        a = act[s]
        com = (mass[sl, None] * pos[sl]).sum(0) / mass[sl].sum()
        central = a[np.argsort(np.linalg.norm(pos[sl][a] - com, axis=1), kind="stable")[:4]]
        rest = np.setdiff1d(a, central)
        rnd = g.choice(rest, min(12, rest.size), replace=False)
        rows = np.sort(np.concatenate([central, rnd])).astype(np.int32)
        ref = O.eval_active(pos[sl], vel[sl], mass[sl], rows, h=h)
        e = errors(out, ref, rows + off)
        for k in errs:
            errs[k].append(e[k])
    agg = {k: (float(np.median([x[0] for x in v])), float(np.max([x[1] for x in v])))
           for k, v in errs.items()}
    (assert_f64 if precision == grav.F64 else assert_mixed)(agg)


def test_batched_device_count_from_compaction_and_configs():
    pos, vel, mass, systems, idx, act = _packed(40, 64, 3000, seed=93)
    n = mass.size
    flags = np.zeros(n, np.uint8)
    flags[idx] = 1
    it = torch.zeros(n, dtype=torch.int32, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
    grav.compact_active(T(flags, torch.uint8), it, cnt)
    ref = run_batched(pos, vel, mass, systems, idx, 0.02, grav.MIXED, device_count=False)
    for cfg in range(grav.lib().grav_tile_config_count(grav.MIXED)):
        acc, jerk, tid, pot, dtg = _outputs(n)
        p = grav.params(h=0.02, precision=grav.MIXED, want_pot=True, tile_config=cfg)
        grav.eval_batched(p, grav.systems_table(systems, device=DEV), T(pos), T(vel), T(mass), it,
                          cnt, n, acc, jerk, tid, pot, dtg)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        assert np.all(np.isfinite(a[idx]))
        e = np.linalg.norm(a[idx] - ref["acc"][idx], axis=1) / np.linalg.norm(ref["acc"][idx], axis=1)
        assert e.max() < 1e-5, (cfg, e.max())


def test_batched_rejects_overlapping_system():
    pos, vel, mass, systems, idx, act = _packed(6, 200, 400, seed=94)
    bad = systems.copy()
    bad[3, 0] = bad[2, 0] + 10          # overlaps system 2
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    out = run_batched(pos, vel, mass, bad, idx, 0.02, grav.F64, flags=flags)
    assert int(flags.item()) & grav.FLAG_BADINDEX
    good = run_batched(pos, vel, mass, systems, idx, 0.02, grav.F64)
    rows = act[0] + systems[0, 0]
    assert np.array_equal(out["acc"][rows], good["acc"][rows])


@pytest.mark.parametrize("precision", [grav.F64, grav.MIXED])
def test_batched_per_system_softening(precision):
    """Plummer systems at h = 1e-3 next to uniform spheres at h = 0.01 in one
    launch (each system's own h from grav_system.h, the call's h = 0.05
    unused but by the systems that give h = 0): bit for bit the per-system
    grav_eval_active with that h, and the oracle on every system's targets."""
    pos, vel, mass, systems, idx, act = _packed(20, 300, 6000, seed=95)
    h_sys = np.where(np.arange(20) % 2 == 0, 1e-3, 0.01)
    h_sys[5] = 0.0                       # this one takes the call's h
    h_call = 0.05
    out = run_batched(pos, vel, mass, systems, idx, h_call, precision, h_sys=h_sys)
    P, V, M = T(pos), T(vel), T(mass)
    errs = {k: [] for k in ("acc", "jerk", "tidal", "pot")}
    for s, (off, ns) in enumerate(systems):
        hs = h_sys[s] if h_sys[s] > 0 else h_call
        sl = slice(off, off + ns)
        acc, jerk, tid, pot, dtg = _outputs(int(ns))
        p = grav.params(h=hs, precision=precision, want_pot=True, max_split=1)
        grav.eval_active(p, P[sl].contiguous(), V[sl].contiguous(), M[sl].contiguous(),
                         T(act[s], torch.int32), None, act[s].size, acc, jerk, tid, pot, dtg)
        torch.cuda.synchronize()
        rows = act[s] + off
        for k, t in (("acc", acc), ("jerk", jerk), ("tidal", tid), ("pot", pot), ("dt_grav", dtg)):
            assert np.array_equal(out[k][rows], t.cpu().numpy()[act[s]]), (s, k)
        ref = O.eval_active(pos[sl], vel[sl], mass[sl], act[s].astype(np.int32), h=hs)
        e = errors(out, ref, rows)
        for k in errs:
            errs[k].append(e[k])
    agg = {k: (float(np.median([m for m, _ in v])), max(x for _, x in v)) for k, v in errs.items()}
    (assert_f64 if precision == grav.F64 else assert_mixed)(agg)


@pytest.mark.parametrize("bad_h", [-1e-3, float("nan"), float("inf")])
def test_batched_rejects_bad_system_softening(bad_h):
    pos, vel, mass, systems, idx, act = _packed(6, 200, 400, seed=96)
    h_sys = np.zeros(6)
    h_sys[2] = bad_h
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    out = run_batched(pos, vel, mass, systems, idx, 0.02, grav.F64, flags=flags, h_sys=h_sys)
    assert int(flags.item()) & grav.FLAG_BADINDEX
    assert np.all(np.isnan(out["acc"][act[2] + systems[2, 0]]))
    good = run_batched(pos, vel, mass, systems, idx, 0.02, grav.F64)
    for s in (0, 1, 3, 4, 5):
        rows = act[s] + systems[s, 0]
        assert np.array_equal(out["acc"][rows], good["acc"][rows])
