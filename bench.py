"""Benchmark of the adaptive-force-update hot path on one GB300.

Workload: turbulent cloud, N = 2^20 equal-mass elements in a uniform sphere
(R = 1, G = M = 1), k^-4 Gaussian random velocities at virial parameter 2,
cubic-spline softening h = 2e-3 (synthetic stand-in for the paper's
STARFORGE cloud, whose initial conditions are not public).

One step = one pass of the whole path at tick t:
  grav_select_due -> grav_compact_active -> grav_eval_active (mixed
  precision, FP32 pair arithmetic) -> grav_predict -> grav_assign_bins.
A fraction f of the elements sits in the finest time bin (active every tick,
hydro-limited: dt_hydro = dt_min) and the rest in the coarsest bin (inactive
at the ticks timed); q_f = 0, so every active element is due.  The headline
uses f = 1 (all 2^20 elements evaluated against all 2^20 sources per step).

Metric: acceleration + jerk + tidal-tensor interactions per second, counted
as n_due * N per evaluation.  Printed as ONE JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_DEFAULT = 1 << 20
H = 2e-3
K_MAX = 6
DT_MAX = 2.0**-4
FLOPS_PER_INTERACTION = 56      # FP32 flops of the Newtonian pair body (FFMA = 2), MUFU not counted
BWD_FLOPS_PER_INTERACTION = 31  # the adjoint's Newtonian pair body, counted the same way
WORKLOAD = "turbulent_cloud_N1048576_h2e-3"
METRIC = "acc+jerk+tidal interactions/s at N=2^20 (mixed precision)"
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write, dram__bytes_read.sum + dram__bytes_write.sum) of
# one force-kernel launch, from an ncu capture of the tile configuration the
# library picks for this workload (17) on the turbulent cloud with N = 2^18,
# all active.  The traffic is the sources and targets streamed once, so it
# scales with N.
TRAFFIC_CAPTURE = {"tile_config": 17, "n": 262144, "bytes": 26887424 + 50837504}
# DRAM bytes (read + write) of one predictor launch on 2^24 elements, all
# active, none due, from an ncu capture of the same launch (82 B per element
# algorithmic; some of the writes were still in L2 when the launch ended).
PREDICT_TRAFFIC_CAPTURE = {"n": 16777216, "bytes": 973454080 + 381213696}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--fraction", type=float, default=1.0)
    ap.add_argument("--tile-config", type=int, default=-1)
    ap.add_argument("--no-extras", action="store_true",
                    help="headline steps only (no sweeps, FP64 path, e2e, CPU baseline)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--clocks-csv", default=None,
                    help="also copy the nvidia-smi clock samples of the timed region here")
    ap.add_argument("--predict-only", action="store_true",
                    help="time only the predictor (grav_predict) on --n elements, all active, "
                         "none due, and print its bandwidth")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (N > 1: independent replicas, one per GPU)
# ---------------------------------------------------------------------------

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda() else "gloo"
        dist.init_process_group(backend)
    return rank, local, ws


def _cuda():
    import torch
    return torch.cuda.is_available()


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int, device=None) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, ws: int, device=None) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, keep: str | None = None):
        self.gpu = gpu_index
        self.keep = keep    # where to copy the samples' CSV afterwards (None: nowhere)
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            self.dir = tempfile.mkdtemp(prefix="grav_clocks_")
            self.path = os.path.join(self.dir, f"clocks_gpu{self.gpu}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()
            if self.keep:
                import shutil
                os.makedirs(os.path.dirname(os.path.abspath(self.keep)), exist_ok=True)
                shutil.copyfile(self.path, self.keep)

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# the path
# ---------------------------------------------------------------------------

class Path:
    """Device state of one replica and one pass of the hot path."""

    def __init__(self, n, fraction, device, tile_config=-1):
        import torch

        from paper_2010_13792_gb300 import grav, ics
        self.torch, self.grav = torch, grav
        self.n, self.dev = n, device
        pos, vel, mass = ics.turbulent_cloud(n, seed=ics.BASE_SEED + 2)
        self.host = {"pos": pos, "vel": vel, "mass": mass}
        fine = ics.active_subset(n, fraction, ics.BASE_SEED + 3)
        bins = np.zeros(n, np.int8)
        bins[fine] = K_MAX
        self.n_due_expected = fine.size
        self.dt_min = DT_MAX * 2.0**-K_MAX
        dt_hydro = np.full(n, self.dt_min)
        f64 = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device)
        self.pos, self.vel, self.mass = f64(pos), f64(vel), f64(mass)
        self.bins = torch.as_tensor(bins, device=device)
        self.dt_hydro = f64(dt_hydro)
        self.tf = torch.zeros(n, dtype=torch.int64, device=device)
        self.dt_grav = torch.zeros(n, dtype=torch.float64, device=device)
        self.active = torch.zeros(n, dtype=torch.uint8, device=device)
        self.due = torch.zeros(n, dtype=torch.uint8, device=device)
        self.idx = torch.zeros(n, dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        self.acc = torch.zeros(n, 3, dtype=torch.float64, device=device)
        self.jerk = torch.zeros(n, 3, dtype=torch.float64, device=device)
        self.tidal = torch.zeros(n, 6, dtype=torch.float64, device=device)
        self.a_out = torch.zeros(n, 3, dtype=torch.float64, device=device)
        self.params = grav.params(h=H, precision=grav.MIXED, tile_config=tile_config)
        self.ws_compact = grav.Workspace()
        self.ws_eval = grav.Workspace()
        self.launches_per_step = 9   # select 1, compact 3, pack 1, eval 1, reduce 1, predict 1, bins 1

    def step(self, tick, ev=None):
        """One pass of the path at `tick` (odd ticks: only the fine bin is active)."""
        g = self.grav
        g.select_due(tick, K_MAX, self.bins, self.tf, self.dt_grav, 0.0, self.dt_min, self.active,
                     self.due)
        g.compact_active(self.due, self.idx, self.count, workspace=self.ws_compact)
        if ev is not None:
            ev[0].record()
        g.eval_active(self.params, self.pos, self.vel, self.mass, self.idx, self.count, self.n,
                      self.acc, self.jerk, self.tidal, None, self.dt_grav,
                      workspace=self.ws_eval)
        if ev is not None:
            ev[1].record()
        g.predict(self.active, self.due, self.acc, self.jerk, self.tf, self.dt_min, self.a_out)
        g.assign_bins(tick, K_MAX, DT_MAX, self.active, self.dt_grav, self.dt_hydro, self.bins)


def l2_flush(buf):
    buf.zero_()


def run_ours(args, rank, local, ws):
    import torch

    from paper_2010_13792_gb300 import grav
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    path = Path(args.n, args.fraction, dev, args.tile_config)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    n_due = path.n_due_expected
    tick = 1
    for _ in range(max(args.warmup, 0)):
        path.step(tick)
        tick += 2
    torch.cuda.synchronize()
    got = int(path.count.item())
    if got != n_due:
        raise RuntimeError(f"due count {got} != expected {n_due}")

    # ---- timed region: K steps, L2 flushed between steps ----
    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    ev_eval = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local, args.clocks_csv if rank == 0 else None) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            l2_flush(flush)
            ev_step[k][0].record()
            path.step(tick, ev_eval[k])
            ev_step[k][1].record()
            tick += 2
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    eval_ms = [a.elapsed_time(b) for a, b in ev_eval]
    t_total = max_over_ranks(sum(step_ms) * 1e-3, ws, dev)
    interactions = float(n_due) * args.n
    total_units = sum_over_ranks(interactions * args.steps, ws, dev)
    value = total_units / t_total
    clocks = clk.summary()

    # the step passes n_idx_max = N (the due count stays on the device)
    used_cfg = args.tile_config if args.tile_config >= 0 else grav.default_tile_config(grav.MIXED, args.n)
    result = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32-mixed",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": args.n, "active_fraction": args.fraction,
                   "n_due_per_step": n_due, "h": H, "sources": args.n,
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "tile_config": grav.tile_configs(grav.MIXED)[used_cfg]},
        "gpu_launches": path.launches_per_step * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }

    traffic = None
    if used_cfg == TRAFFIC_CAPTURE["tile_config"] and args.fraction == 1.0:
        traffic = TRAFFIC_CAPTURE["bytes"] * args.n / TRAFFIC_CAPTURE["n"]
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak32 = sms * 128 * 2 * 2070e6 / 1e12       # FP32 lanes x FMA x max SM clock
    eval_s = statistics.mean(eval_ms) * 1e-3
    achieved = FLOPS_PER_INTERACTION * interactions / eval_s / 1e12
    result["roofline"] = {
        "bound": "alu", "kernel": "eval_mixed_kernel (grav_eval_active: pack + direct sum)",
        "achieved": achieved, "peak": peak32, "unit": "TFLOP/s", "frac": achieved / peak32,
        "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x 2070 MHz (derived)",
        "flops_per_interaction": FLOPS_PER_INTERACTION, "traffic": traffic,
        "traffic_basis": "ncu dram bytes of the same kernel at N=2^18, scaled by N",
        "eval_ms_mean": 1e3 * eval_s,
    }

    if not args.no_extras:
        # end to end on every rank (units of all ranks over the slowest rank)
        result["e2e"] = e2e(args, path, dev, flush, ws)
    if rank == 0 and ws == 1 and not args.no_extras:
        # the other workloads and the oracle baseline at one GPU only (with
        # more ranks they would hold every GPU for minutes)
        result["extras"] = extras(args, path, dev, sms, peak32, flush)
        # the predictor (HBM-bound) against the measured copy bandwidth
        pb = result["extras"]["predict_N16777216"]
        hbm = measured_hbm_peak()
        if hbm:
            result["predictor_roofline"] = {
                "bound": "hbm", "kernel": "predict_pair_kernel (grav_predict), 2^24 elements",
                "achieved": pb["GB_per_s"], "peak": hbm, "unit": "GB/s", "frac": pb["GB_per_s"] / hbm,
                "peak_basis": "measured copy bandwidth (burst)", "bytes_per_element": 82,
                "traffic": PREDICT_TRAFFIC_CAPTURE["bytes"] * pb["n"] / PREDICT_TRAFFIC_CAPTURE["n"]}
        tree = result["extras"]["tree_N1048576"]
        if args.n == tree["n"] and args.fraction == 1.0:
            tree["speedup_over_mixed_direct"] = 1e3 * eval_s / tree["mixed"]["ms"]
        result["cpu_baseline"] = cpu_baseline(path, args.cpu_seconds)
    return result


def _time_eval(path, params, idx, cnt, n_idx, reps, flush):
    import torch
    from paper_2010_13792_gb300 import grav
    ws = grav.Workspace()
    grav.eval_active(params, path.pos, path.vel, path.mass, idx, cnt, n_idx, path.acc, path.jerk,
                     path.tidal, None, path.dt_grav, workspace=ws)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        grav.eval_active(params, path.pos, path.vel, path.mass, idx, cnt, n_idx, path.acc,
                         path.jerk, path.tidal, None, path.dt_grav, workspace=ws)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    return statistics.median(ts)


def extras(args, path, dev, sms, peak32, flush):
    """Active-fraction sweep (mixed), the FP64 GPU path, the predictor's
    bandwidth and the measured FMA peaks."""
    import torch

    from paper_2010_13792_gb300 import grav, ics
    out = {}
    n = args.n
    sweep = {}
    for frac in (0.01, 0.1):
        idx_np = ics.active_subset(n, frac, ics.BASE_SEED + 5)
        idx = torch.as_tensor(idx_np, device=dev)
        cnt = torch.tensor([idx_np.size], dtype=torch.int32, device=dev)
        t = _time_eval(path, path.params, idx, cnt, idx_np.size, 3, flush)
        sweep[str(frac)] = {"interactions_per_s": idx_np.size * n / t, "eval_ms": 1e3 * t}
    out["mixed_fraction_sweep"] = sweep
    # FP64 path on the 1% and 10% active sets (all N sources), and the mixed
    # path's throughput over it at the same fraction
    p64 = grav.params(h=H, precision=grav.F64)
    f64 = {}
    for frac in (0.01, 0.1):
        idx_np = ics.active_subset(n, frac, ics.BASE_SEED + 5)
        idx = torch.as_tensor(idx_np, device=dev)
        cnt = torch.tensor([idx_np.size], dtype=torch.int32, device=dev)
        t64 = _time_eval(path, p64, idx, cnt, idx_np.size, 2, flush)
        ips = idx_np.size * n / t64
        f64[str(frac)] = {"interactions_per_s": ips, "eval_ms": 1e3 * t64,
                          "mixed_over_fp64": sweep[str(frac)]["interactions_per_s"] / ips}
    ips64 = f64["0.1"]["interactions_per_s"]
    out["fp64_path"] = f64
    # predictor (HBM-bound): all elements active, none due
    ones = torch.ones(n, dtype=torch.uint8, device=dev)
    zeros = torch.zeros(n, dtype=torch.uint8, device=dev)
    ts = []
    for _ in range(5):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        grav.predict(ones, zeros, path.acc, path.jerk, path.tf, path.dt_min, path.a_out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    tp = statistics.median(ts)
    bytes_pred = n * (1 + 1 + 8 + 24 + 24 + 24)
    out["predict"] = {"bytes_per_element": 82, "GB_per_s": bytes_pred / tp / 1e9, "us": tp * 1e6}
    out["predict_N16777216"] = predict_bandwidth(dev, 1 << 24)
    out["periodic_zeldovich_64cubed"] = periodic_extra(dev, flush)
    out["adaptive_softening_N1048576"] = soft_extra(path, dev, flush)
    out["tree_N1048576"] = tree_extra(path, dev, flush)
    out["adjoint"] = backward_extra(path, dev, flush)
    out["other_workloads_mixed_all_active"] = workloads_extra(dev, flush, peak32)
    out["batched_256_systems"] = batched_extra(dev, flush)
    out["adaptive_plummer_131072"] = adaptive_extra(dev)
    try:
        f32 = grav.measure_fma_peak(grav.MIXED, 0.5)
        f64p = grav.measure_fma_peak(grav.F64, 0.5)
        f32x2 = grav.measure_fma_peak(grav.PEAK_F32X2, 0.5)
        out["measured_fma_peak_tflops"] = {"fp32": f32 / 1e12, "fp32x2": f32x2 / 1e12,
                                           "fp64": f64p / 1e12}
        # the FP64 path (10% active) against the measured FP64 FMA peak, same
        # 56-flop tally
        out["fp64_path"]["frac_of_measured_fp64_peak_at_0.1"] = FLOPS_PER_INTERACTION * ips64 / f64p
    except grav.GravError as e:
        out["measured_fma_peak_tflops"] = {"error": str(e)}
    return out


def predict_bandwidth(dev, n, reps=5, warmup=1):
    """The predictor (HBM-bound) on n elements, all active, none due:
    82 B per element (flags 2, T_f 8, a_last 24, j_last 24 read; a_out 24
    written); inputs larger than L2, median of `reps` event-timed launches."""
    import torch

    from paper_2010_13792_gb300 import grav
    g = torch.Generator(device=dev).manual_seed(5)
    ones = torch.ones(n, dtype=torch.uint8, device=dev)
    zeros = torch.zeros(n, dtype=torch.uint8, device=dev)
    a_last = torch.randn(n, 3, dtype=torch.float64, device=dev, generator=g)
    j_last = torch.randn(n, 3, dtype=torch.float64, device=dev, generator=g)
    tf = torch.randint(0, 64, (n,), dtype=torch.int64, device=dev, generator=g)
    a_out = torch.empty_like(a_last)
    for _ in range(max(warmup, 1)):
        grav.predict(ones, zeros, a_last, j_last, tf, 2.0**-10, a_out)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        grav.predict(ones, zeros, a_last, j_last, tf, 2.0**-10, a_out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    t = statistics.median(ts)
    return {"n": n, "bytes": 82 * n, "us": 1e6 * t, "GB_per_s": 82 * n / t / 1e9}


def measured_hbm_peak():
    """The machine's measured copy bandwidth (GB/s), if the machine provides it."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def periodic_extra(dev, flush):
    """Periodic box (nearest image), 64^3 elements in the pancake shape of the
    paper's Zeldovich test (one sinusoidal mode), h = 2e-3: mixed with all
    elements active, FP64 with 5% active, against all sources."""
    import torch

    from paper_2010_13792_gb300 import grav, ics
    pos, vel, mass = ics.zeldovich_box(64, 1.0, amplitude=0.8)
    n = mass.size
    f64 = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    P, V, M = f64(pos), f64(vel), f64(mass)
    acc = torch.empty(n, 3, dtype=torch.float64, device=dev)
    jerk, tid = torch.empty_like(acc), torch.empty(n, 6, dtype=torch.float64, device=dev)
    res = {"n": n, "box": 1.0, "h": 2e-3}
    for name, prec, frac in (("mixed", grav.MIXED, 1.0), ("f64", grav.F64, 0.05)):
        idx_np = ics.active_subset(n, frac, ics.BASE_SEED + 7)
        idx = torch.as_tensor(idx_np, device=dev)
        p = grav.params(h=2e-3, precision=prec, box=1.0)
        ws = grav.Workspace()
        grav.eval_active(p, P, V, M, idx, None, idx_np.size, acc, jerk, tid, workspace=ws)
        ts = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            grav.eval_active(p, P, V, M, idx, None, idx_np.size, acc, jerk, tid, workspace=ws)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        t = statistics.median(ts)
        res[name] = {"active_fraction": frac, "interactions_per_s": idx_np.size * n / t,
                     "ms": 1e3 * t}
    return res


def soft_extra(path, dev, flush):
    """Adaptive softening on the headline cloud (2^20 elements): the support
    solve for 32 neighbours from a uniform guess, then the mixed force sums of
    every element with per-element supports and the correction term."""
    import torch

    from paper_2010_13792_gb300 import grav
    n = path.n
    f64 = lambda: torch.empty(n, dtype=torch.float64, device=dev)
    h, zeta, omega = f64(), f64(), f64()
    iters = torch.empty(n, dtype=torch.int32, device=dev)
    flags = torch.zeros(1, dtype=torch.int32, device=dev)
    sp = grav.soft_params(n_ngb=32.0, tol=1e-12, max_iter=100)
    ws_s = grav.Workspace()
    ts = []
    for _ in range(3):
        h.fill_(2e-2)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        grav.soft_solve(sp, path.pos, path.mass, h, zeta, omega, iters, flags, workspace=ws_s)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    it = iters.to(torch.float64)
    res = {"n": n, "n_ngb": 32.0, "solve_ms": 1e3 * statistics.median(ts),
           "iterations_median": float(it.median()), "iterations_max": int(iters.max()),
           "flags": int(flags.item()), "h_median": float(h.median()),
           "h_range": [float(h.min()), float(h.max())]}
    acc = torch.empty(n, 3, dtype=torch.float64, device=dev)
    jerk, tid = torch.empty_like(acc), torch.empty(n, 6, dtype=torch.float64, device=dev)
    p = grav.params(h=1.0, precision=grav.MIXED)
    ws_e = grav.Workspace()
    grav.eval_soft(p, path.pos, path.vel, path.mass, h, zeta, None, None, n, acc, jerk, tid,
                   workspace=ws_e)
    ts = []
    for _ in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        grav.eval_soft(p, path.pos, path.vel, path.mass, h, zeta, None, None, n, acc, jerk, tid,
                       workspace=ws_e)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    t = statistics.median(ts)
    res["eval_mixed"] = {"interactions_per_s": n * n / t, "ms": 1e3 * t}
    return res


def tree_extra(path, dev, flush):
    """The oct-tree solver (Theta = 0.5, leaves of 8) on the headline cloud
    with every element a target, mixed walk and FP64 walk: build plus walk,
    nodes and interactions, and the accuracy of a against the mixed direct
    sum of the timed steps (the same positions)."""
    import torch

    from paper_2010_13792_gb300 import grav
    n = path.n
    acc = torch.empty(n, 3, dtype=torch.float64, device=dev)
    jerk, tid = torch.empty_like(acc), torch.empty(n, 6, dtype=torch.float64, device=dev)
    stats = torch.zeros(2, dtype=torch.int64, device=dev)
    tp = grav.tree_params(theta=0.5, leaf_size=8)
    ws = grav.Workspace()
    res = {"n": n, "theta": 0.5, "leaf_size": 8, "speedup_over_mixed_direct": None}
    for name, prec in (("mixed", grav.MIXED), ("f64", grav.F64)):
        p = grav.params(h=H, precision=prec)
        grav.eval_tree(p, tp, path.pos, path.vel, path.mass, None, None, n, acc, jerk, tid,
                       stats=stats, workspace=ws)
        ts = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            grav.eval_tree(p, tp, path.pos, path.vel, path.mass, None, None, n, acc, jerk, tid,
                           stats=stats, workspace=ws)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        t = statistics.median(ts)
        e = ((acc - path.acc).norm(dim=1) / path.acc.norm(dim=1)).cpu()
        q = torch.quantile(e[::16], torch.tensor([0.5, 0.99], dtype=e.dtype))
        inter = int(stats[1].item())
        res["nodes"] = int(stats[0].item())
        res["interactions_per_target"] = inter / n
        res[name] = {"ms": 1e3 * t, "interactions_per_s": inter / t,
                     "acc_rel_error_vs_direct": {"median": float(q[0]), "p99": float(q[1]),
                                                 "max": float(e.max())}}
    return res


def workloads_extra(dev, flush, peak32):
    """The mixed force evaluation, every element a target, on the other
    synthetic inputs shaped like the paper's tests: the Plummer sphere of
    2^17 (h = 1e-3, centrally concentrated: many softened tiles near the
    centre) and a uniform sphere of 2^20 (h = 0.01)."""
    import torch

    from paper_2010_13792_gb300 import grav, ics
    res = {}
    for name, (pos, vel, mass), h in (
            ("plummer_N131072_h1e-3", ics.plummer(1 << 17, seed=ics.BASE_SEED + 1), 1e-3),
            ("uniform_sphere_N1048576_h1e-2", ics.uniform_sphere(1 << 20, seed=ics.BASE_SEED), 1e-2)):
        n = mass.size
        f64 = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
        P, V, M = f64(pos), f64(vel), f64(mass)
        acc = torch.empty(n, 3, dtype=torch.float64, device=dev)
        jerk, tid = torch.empty_like(acc), torch.empty(n, 6, dtype=torch.float64, device=dev)
        p = grav.params(h=h, precision=grav.MIXED)
        ws = grav.Workspace()
        grav.eval_active(p, P, V, M, None, None, n, acc, jerk, tid, workspace=ws)
        ts = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            grav.eval_active(p, P, V, M, None, None, n, acc, jerk, tid, workspace=ws)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        t = statistics.median(ts)
        ips = n * n / t
        res[name] = {"ms": 1e3 * t, "interactions_per_s": ips,
                     "frac_of_fp32_peak": FLOPS_PER_INTERACTION * ips / 1e12 / peak32}
    return res


def backward_extra(path, dev, flush):
    """The adjoint (grav_eval_backward): gradients of L = sum w |a|^2 with
    respect to positions and masses, every element a target and a source.
    On the headline cloud (mixed; a_bar = 2 w a from the timed steps) and on
    the differentiation workload, a Plummer sphere of 2^16 (mixed and FP64,
    with the potential-energy term).  Flops per pair from the kernel's
    Newtonian pair body: 20 FP32 instructions, 11 of them FMAs = 31 flops."""
    import torch

    from paper_2010_13792_gb300 import grav, ics
    res = {"flops_per_interaction": BWD_FLOPS_PER_INTERACTION}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        return statistics.median(ts)

    g = torch.Generator(device=dev).manual_seed(11)
    n = path.n
    w = torch.rand(n, 1, dtype=torch.float64, device=dev, generator=g)
    a_bar = 2.0 * w * path.acc
    pos_bar = torch.empty(n, 3, dtype=torch.float64, device=dev)
    mass_bar = torch.empty(n, dtype=torch.float64, device=dev)
    ws = grav.Workspace()
    pm = grav.params(h=H, precision=grav.MIXED)
    t = timed(lambda: grav.eval_backward(pm, path.pos, path.mass, a_bar, 0.0, None, path.tidal,
                                         None, pos_bar, mass_bar, workspace=ws), 2)
    res[f"cloud_N{n}_mixed"] = {"ms": 1e3 * t, "interactions_per_s": n * n / t,
                                "tflops": BWD_FLOPS_PER_INTERACTION * n * n / t / 1e12}

    m = 1 << 16
    pos, vel, mass = ics.plummer(m)
    f64 = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
    P, V, M = f64(pos), f64(vel), f64(mass)
    wp = f64(ics.rng(ics.BASE_SEED + 4).uniform(size=(m, 1)))
    for name, prec in (("mixed", grav.MIXED), ("f64", grav.F64)):
        p = grav.params(h=1e-3, precision=prec, want_pot=True)
        acc = torch.empty(m, 3, dtype=torch.float64, device=dev)
        jerk, tid = torch.empty_like(acc), torch.empty(m, 6, dtype=torch.float64, device=dev)
        pot = torch.empty(m, dtype=torch.float64, device=dev)
        grav.eval_active(p, P, V, M, None, None, m, acc, jerk, tid, pot, workspace=ws)
        ab = 2.0 * wp * acc
        pb = torch.empty(m, 3, dtype=torch.float64, device=dev)
        mb = torch.empty(m, dtype=torch.float64, device=dev)
        t = timed(lambda: grav.eval_backward(p, P, M, ab, 1.0, acc, tid, pot, pb, mb,
                                             workspace=ws), 3)
        res[f"plummer_N{m}_{name}"] = {"ms": 1e3 * t, "interactions_per_s": m * m / t,
                                       "tflops": BWD_FLOPS_PER_INTERACTION * m * m / t / 1e12}
    return res


def batched_extra(dev, flush):
    """256 independent systems (half Plummer, half uniform; sizes log-uniform
    in [512, 65536]; 1-50% of each active) in one persistent launch with
    autotuned tiles, mixed and FP64; and 100 substeps of the batched adaptive
    loop captured as one CUDA graph."""
    import torch

    from paper_2010_13792_gb300 import autotune, grav, ics
    from paper_2010_13792_gb300.adaptive import AdaptiveIntegrator
    pos, vel, mass, offsets, sizes, act = ics.batched_systems(256, 512, 65536,
                                                              seed=ics.BASE_SEED + 4)
    n = mass.size
    idx_np = np.concatenate([a + o for a, o in zip(act, offsets)]).astype(np.int32)
    inter = float(sum(a.size * int(s) for a, s in zip(act, sizes)))
    f64 = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    P, V, M = f64(pos), f64(vel), f64(mass)
    systems = grav.systems_table(np.stack([offsets, sizes], 1), device=dev)
    idx = torch.as_tensor(idx_np, device=dev)
    acc = torch.empty(n, 3, dtype=torch.float64, device=dev)
    jerk, tid = torch.empty_like(acc), torch.empty(n, 6, dtype=torch.float64, device=dev)
    res = {"n_total": int(n), "n_targets": int(idx_np.size), "interactions": inter}
    for name, prec in (("mixed", grav.MIXED), ("f64", grav.F64)):
        p = grav.params(h=1e-3, precision=prec)
        best, ms = autotune.tune_eval(p, P, V, M, idx, idx_np.size, systems=systems, reps=2,
                                      use_cache=False)
        p = grav.params(h=1e-3, precision=prec, tile_config=best)
        ws = grav.Workspace()
        ts = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            grav.eval_batched(p, systems, P, V, M, idx, None, idx_np.size, acc, jerk, tid,
                              workspace=ws)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        t = statistics.median(ts)
        res[name] = {"interactions_per_s": inter / t, "ms": 1e3 * t, "tile_config": best,
                     "autotune_ms": {str(k): round(v, 3) for k, v in ms.items()}}
    it = AdaptiveIntegrator(pos, vel, mass, h=1e-3, q_f=0.5, k_max=6, dt_max=2.0**-4,
                            precision=grav.MIXED, systems=np.stack([offsets, sizes], 1),
                            tile_config=res["mixed"]["tile_config"])
    it.start()
    it.capture(99)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    it.replay(1)
    b.record()
    torch.cuda.synchronize()
    res["graph_100_substeps"] = {"ms": a.elapsed_time(b), "work_ratio": it.work_ratio(),
                                 "substeps": 100}
    return res


def adaptive_extra(dev):
    """The adaptive update loop on a Plummer sphere of 2^17 (h = 1e-3,
    k_max = 6, dt_max = 2^-4): one cycle of 64 substeps captured as a CUDA
    graph.  q_f runs over {1/8, 1/4, 1/2, 1}, the paper's range, against
    updating every active element at every substep (q_f = 0).  Both precisions
    are run.  Per run: the cycle time, the work ratio (force evaluations over
    those of q_f = 0), the relative energy change over the cycle and the
    speedup over q_f = 0 of the same precision.  For q_f > 0 also: the jerk
    predictor's error quantiles at the cycle's end, and the median distance
    from the q_f = 0 positions."""
    import torch

    from paper_2010_13792_gb300 import grav, ics
    from paper_2010_13792_gb300.adaptive import AdaptiveIntegrator
    pos, vel, mass = ics.plummer(1 << 17, seed=ics.BASE_SEED + 1)
    res = {"n": 1 << 17, "h": 1e-3, "k_max": 6, "dt_max": 2.0**-4, "substeps": 64}
    for pname, prec in (("mixed", grav.MIXED), ("f64", grav.F64)):
        runs, out = {}, {}
        for q_f in (0.0, 0.125, 0.25, 0.5, 1.0):
            it = AdaptiveIntegrator(pos, vel, mass, h=1e-3, q_f=q_f, k_max=6, dt_max=2.0**-4,
                                    precision=prec)
            e0 = sum(it.energy())
            it.start()
            it.capture_cycle()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            it.replay(1)
            b.record()
            torch.cuda.synchronize()
            e1 = sum(it.energy())
            rec = {"ms_per_64_substeps": a.elapsed_time(b), "work_ratio": it.work_ratio(),
                   "rel_energy_change": abs(e1 - e0) / abs(e0)}
            if q_f > 0:
                rec["predicted_a_rel_error"] = it.predictor_error()["jerk"]
            runs[q_f] = it
            out[f"qf{q_f:g}"] = rec
        std = out["qf0"]
        for q_f, it in runs.items():
            if q_f > 0:
                r = out[f"qf{q_f:g}"]
                r["speedup_over_qf0"] = std["ms_per_64_substeps"] / r["ms_per_64_substeps"]
                r["median_position_difference"] = float((it.pos - runs[0.0].pos).norm(dim=1).median().item())
        res[pname] = out
    res["mixed_over_f64_qf0.5"] = (res["f64"]["qf0.5"]["ms_per_64_substeps"] /
                                   res["mixed"]["qf0.5"]["ms_per_64_substeps"])
    # the paper's predictor ablation (q_f = 1/2): none, linear polynomial, jerk
    abl = {}
    for mode in ("none", "poly", "jerk"):
        it = AdaptiveIntegrator(pos, vel, mass, h=1e-3, q_f=0.5, k_max=6, dt_max=2.0**-4,
                                precision=grav.MIXED, predictor=mode)
        e0 = sum(it.energy())
        it.run(64)
        err = it.predictor_error()
        abl[mode] = {"predicted_a_rel_error": err[mode],
                     "rel_energy_change": abs(sum(it.energy()) - e0) / abs(e0),
                     "work_ratio": it.work_ratio()}
    res["predictor_ablation"] = abl
    return res


def e2e(args, path, dev, flush, ws=1):
    """The same step through the C ABI with inputs in pinned HOST memory:
    host->device copies of the step's inputs and device->host copies of its
    results are inside the timed region."""
    import torch
    host_in = {
        "pos": torch.as_tensor(path.host["pos"]).pin_memory(),
        "vel": torch.as_tensor(path.host["vel"]).pin_memory(),
        "mass": torch.as_tensor(path.host["mass"]).pin_memory(),
        "tf": path.tf.cpu().pin_memory(),
        "dt_grav": path.dt_grav.cpu().pin_memory(),
        "bins": path.bins.cpu().pin_memory(),
        "dt_hydro": path.dt_hydro.cpu().pin_memory(),
    }
    dev_in = {"pos": path.pos, "vel": path.vel, "mass": path.mass, "tf": path.tf,
              "dt_grav": path.dt_grav, "bins": path.bins, "dt_hydro": path.dt_hydro}
    host_out = {"acc": torch.empty_like(path.acc, device="cpu").pin_memory(),
                "jerk": torch.empty_like(path.jerk, device="cpu").pin_memory(),
                "tidal": torch.empty_like(path.tidal, device="cpu").pin_memory(),
                "dt_grav": torch.empty_like(path.dt_grav, device="cpu").pin_memory(),
                "a_out": torch.empty_like(path.a_out, device="cpu").pin_memory()}
    dev_out = {"acc": path.acc, "jerk": path.jerk, "tidal": path.tidal, "dt_grav": path.dt_grav,
               "a_out": path.a_out}
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())
    steps = max(1, min(args.steps, 3))
    tick = 10001
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for k, t in host_in.items():
            dev_in[k].copy_(t, non_blocking=True)
        path.step(tick)
        for k, t in host_out.items():
            t.copy_(dev_out[k], non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
        tick += 2
    t = max_over_ranks(statistics.mean(ts), ws, dev)
    units = sum_over_ranks(float(path.n_due_expected) * path.n, ws, dev)
    return {"value": units / t, "unit": "interactions/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps}


def cpu_baseline(path, seconds):
    """The FP64 oracle as it stands, on this host's cores, on a strided target
    sample of the same workload against all N sources."""
    from oracle import oracle as O
    n = path.n
    pos, vel, mass = path.host["pos"], path.host["vel"], path.host["mass"]
    threads = O.max_threads()
    k = 64
    t = 0.0
    while True:
        idx = np.arange(0, n, max(1, n // k), dtype=np.int32)[:k]
        t0 = time.perf_counter()
        O.eval_active(pos, vel, mass, idx, h=H, want_pot=False)
        t = time.perf_counter() - t0
        if t >= 0.3 * seconds or k >= n:
            break
        k = int(min(n, k * max(2.0, min(16.0, 0.5 * seconds / max(t, 1e-3)))))
    res = {"value": idx.size * n / t, "unit": "interactions/s", "cores": threads,
           "kind": "oracle", "sample": f"{idx.size} strided targets x {n} sources, FP64, "
           f"{t:.1f} s", "seconds": t}
    # one core, a smaller strided sample
    k1 = max(8, int(idx.size / max(threads, 1) / 2))
    idx1 = np.arange(0, n, max(1, n // k1), dtype=np.int32)[:k1]
    t0 = time.perf_counter()
    O.eval_active(pos, vel, mass, idx1, h=H, want_pot=False, nthreads=1)
    t1 = time.perf_counter() - t0
    res["one_core"] = {"value": idx1.size * n / t1, "sample": f"{idx1.size} strided targets x {n}",
                       "seconds": t1}
    return res


def run_reference(args, rank, ws):
    """Reference arm: the FP64 oracle on the host cores, same workload and
    metric; each step a bounded strided target sample against all N sources."""
    if rank != 0:
        return None
    from oracle import oracle as O
    from paper_2010_13792_gb300 import ics
    n = args.n
    pos, vel, mass = ics.turbulent_cloud(n, seed=ics.BASE_SEED + 2)
    threads = O.max_threads()
    k = max(threads * 4, 32)
    idx = np.arange(0, n, max(1, n // k), dtype=np.int32)[:k]
    for _ in range(max(args.warmup, 0)):
        O.eval_active(pos, vel, mass, idx[: max(threads, 1)], h=H, want_pot=False)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.eval_active(pos, vel, mass, idx, h=H, want_pot=False)
        ts.append(time.perf_counter() - t0)
    t = sum(ts)
    value = idx.size * n * args.steps / t
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "sample_targets_per_step": int(idx.size)},
        "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": threads,
                         "kind": "oracle", "sample": f"{idx.size} strided targets x {n} sources per step"},
        "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank, local, ws = dist_setup()
    if args.predict_only:
        import torch
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        res = predict_bandwidth(dev, args.n, reps=max(args.steps, 1), warmup=max(args.warmup, 0))
        res["peak_GB_per_s"] = measured_hbm_peak()
        if rank == 0:
            print(json.dumps({"predict": res}), flush=True)
        return
    if args.impl == "reference":
        res = run_reference(args, rank, ws)
    else:
        res = run_ours(args, rank, local, ws)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
