"""Adaptive force updates inside a block-timestep KDK integrator.

This is the loop the paper's method lives in (Section 2; Section 3's
hierarchical power-of-two block timesteps), driven through libgrav's C ABI:
every tick (one dt_min) the whole system drifts, the elements at the end of
their step are selected (Eq. 3 counter, Eq. updatecondition), the due ones
are compacted and re-evaluated, the rest get the jerk predictor
(Eq. jerkupdate), the active elements are kicked, re-binned from
dt_i = min(dt_grav, dt_hydro) and kicked again.  Drift and kick are plain
tensor updates of the harness; every step of the gravity path runs in
libgrav's kernels.

``q_f = 0`` re-evaluates every active element each step (the standard
scheme the paper compares against).  A whole cycle of 2^k_max ticks can be
captured once as a CUDA graph and replayed: every kernel argument that
depends on the tick depends only on tick mod 2^k_max, and all counts stay on
the device.
"""
from __future__ import annotations

import torch

from . import grav


class AdaptiveIntegrator:
    def __init__(self, pos, vel, mass, *, h: float, q_f: float, k_max: int = 6,
                 dt_max: float = 2.0**-4, eta: float = 0.01, G: float = 1.0,
                 precision: int = grav.MIXED, dt_hydro=None, predictor="jerk",
                 systems=None, tile_config: int = -1, device=None):
        """predictor: "jerk" (Eq. jerkupdate), "poly" (first-order polynomial
        through the last two logged evaluations, Section 2.2) or "none" (keep the
        last evaluated acceleration).  systems: optional [n_sys, 2] (offset, n)
        or a grav.systems_table (offset, n, h)
        of independent systems packed back to back; their forces come from one
        batched launch per tick."""
        device = device or torch.device("cuda", torch.cuda.current_device())
        f64 = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
        self.dev = device
        self.pos, self.vel, self.mass = f64(pos).clone(), f64(vel).clone(), f64(mass).clone()
        n = self.n = self.mass.numel()
        self.h, self.q_f, self.k_max, self.dt_max, self.G = h, q_f, k_max, dt_max, G
        self.dt_min = dt_max * 2.0**-k_max
        if predictor is True:
            predictor = "jerk"
        elif predictor is False or predictor is None:
            predictor = "none"
        if predictor not in ("jerk", "poly", "none"):
            raise ValueError(f"unknown predictor {predictor!r}")
        self.predictor = predictor
        self.params = grav.params(G=G, h=h, eta=eta, precision=precision, tile_config=tile_config)
        self.systems = None if systems is None else grav.systems_table(systems, device=device)
        self.acc = torch.zeros(n, 3, dtype=torch.float64, device=device)
        self.jerk = torch.zeros_like(self.acc)
        self.tidal = torch.zeros(n, 6, dtype=torch.float64, device=device)
        self.dt_grav = torch.zeros(n, dtype=torch.float64, device=device)   # 0: never evaluated
        self.dt_hydro = (torch.full((n,), self.dt_min, dtype=torch.float64, device=device)
                         if dt_hydro is None else f64(dt_hydro))
        self.tf = torch.zeros(n, dtype=torch.int64, device=device)
        self.bins = torch.full((n,), k_max, dtype=torch.int8, device=device)
        self.active = torch.zeros(n, dtype=torch.uint8, device=device)
        self.due = torch.zeros(n, dtype=torch.uint8, device=device)
        self.idx = torch.zeros(n, dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        self.a_kick = torch.zeros(n, 3, dtype=torch.float64, device=device)
        # half of the step of each bin (exact powers of two), for the kicks
        self.half_step = torch.tensor([0.5 * self.dt_min * 2.0 ** (k_max - k) for k in range(k_max + 1)],
                                      dtype=torch.float64, device=device)
        self.zero_j = torch.zeros_like(self.acc)
        # history of the polynomial predictor
        self.elapsed = torch.zeros(n, dtype=torch.int64, device=device)
        self.a_prev = torch.zeros(n, 3, dtype=torch.float64, device=device)
        self.dt_prev = torch.zeros(n, dtype=torch.float64, device=device)
        # device-side work counters: sum of n_due and of n_active over ticks
        self.n_due_total = torch.zeros(1, dtype=torch.int64, device=device)
        self.n_active_total = torch.zeros(1, dtype=torch.int64, device=device)
        self.ws_compact = grav.Workspace()
        self.ws_eval = grav.Workspace()
        self.ws_compact.get(grav.compact_workspace_bytes(n), device)
        if self.systems is None:
            self.ws_eval.get(grav.eval_workspace_bytes(self.params, n, n), device)
        else:
            self.ws_eval.get(grav.batched_workspace_bytes(self.params, self.systems.shape[0], n),
                             device)
        self.tick = 0
        self.graph = None
        self.graph_ticks = 0

    # -- pieces ---------------------------------------------------------------
    def _gravity(self, tick: int):
        g = grav
        poly = self.predictor == "poly"
        g.select_due(tick, self.k_max, self.bins, self.tf, self.dt_grav, self.q_f, self.dt_min,
                     self.active, self.due, elapsed_out=self.elapsed if poly else None)
        if poly:
            g.push_history(self.due, self.elapsed, self.dt_grav, self.acc, self.a_prev, self.dt_prev,
                           self.dt_min)
        g.compact_active(self.due, self.idx, self.count, workspace=self.ws_compact)
        if self.systems is None:
            g.eval_active(self.params, self.pos, self.vel, self.mass, self.idx, self.count, self.n,
                          self.acc, self.jerk, self.tidal, None, self.dt_grav, workspace=self.ws_eval)
        else:
            g.eval_batched(self.params, self.systems, self.pos, self.vel, self.mass, self.idx,
                           self.count, self.n, self.acc, self.jerk, self.tidal, None, self.dt_grav,
                           workspace=self.ws_eval)
        if self.predictor == "poly":
            g.predict_poly(self.active, self.due, self.acc, self.a_prev, self.dt_prev, self.tf,
                           self.dt_min, self.a_kick)
        else:
            g.predict(self.active, self.due, self.acc,
                      self.jerk if self.predictor == "jerk" else self.zero_j, self.tf, self.dt_min,
                      self.a_kick)
        self.n_due_total += self.count.to(torch.int64)
        self.n_active_total += self.active.sum(dtype=torch.int64)

    def _kick(self):
        # half a step of the element's bin for active elements, 0 for the rest
        # (one gather and one product: these launches run every tick)
        w = self.half_step[self.bins.long()] * self.active
        self.vel.addcmul_(self.a_kick, w.unsqueeze(1))

    def substep(self, tick: int):
        """One tick: drift, gravity for the elements at a step boundary, kicks."""
        if tick > 0:
            self.pos.add_(self.vel, alpha=self.dt_min)
        self._gravity(tick)
        if tick > 0:
            self._kick()                           # closes the step that ends now
        grav.assign_bins(tick, self.k_max, self.dt_max, self.active, self.dt_grav, self.dt_hydro,
                         self.bins)
        self._kick()                               # opens the next step

    # -- driving --------------------------------------------------------------
    def start(self):
        """Tick 0: every element is evaluated and binned."""
        if self.tick != 0:
            raise RuntimeError("start() must come first")
        self.substep(0)
        self.tick = 1

    def run(self, n_ticks: int):
        """Eager: n_ticks further ticks."""
        if self.tick == 0:
            self.start()
        for _ in range(n_ticks):
            self.substep(self.tick)
            self.tick += 1

    def capture_cycle(self):
        """Capture one cycle of 2^k_max ticks as a CUDA graph (after start())."""
        if self.tick == 0:
            self.start()
        torch.cuda.synchronize()
        period = 1 << self.k_max
        g = torch.cuda.CUDAGraph()
        base = self.tick
        with torch.cuda.graph(g):
            for r in range(period):
                self.substep(base + r)
        # capture records the work without running it
        self.graph = g
        self.graph_ticks = period
        return g

    def capture(self, n_ticks: int):
        """Capture the next n_ticks ticks as one CUDA graph (after start()).  It
        may be replayed repeatedly only when n_ticks is a multiple of 2^k_max."""
        if self.tick == 0:
            self.start()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        base = self.tick
        with torch.cuda.graph(g):
            for r in range(n_ticks):
                self.substep(base + r)
        self.graph = g
        self.graph_ticks = n_ticks
        return g

    def replay(self, cycles: int = 1):
        if self.graph is None:
            raise RuntimeError("capture_cycle() first")
        period = 1 << self.k_max
        if cycles > 1 and self.graph_ticks % period:
            raise RuntimeError("a graph of a partial cycle can be replayed once only")
        for _ in range(cycles):
            self.graph.replay()
            self.tick += self.graph_ticks

    # -- diagnostics ----------------------------------------------------------
    def energy(self):
        """Kinetic + potential energy from a fresh all-element evaluation (one
        system; for packed systems the sum over systems is not a physical
        energy)."""
        n = self.n
        p = grav.params(G=self.G, h=self.h, precision=grav.F64, want_pot=True)
        acc = torch.empty(n, 3, dtype=torch.float64, device=self.dev)
        jerk = torch.empty_like(acc)
        tid = torch.empty(n, 6, dtype=torch.float64, device=self.dev)
        pot = torch.empty(n, dtype=torch.float64, device=self.dev)
        grav.eval_active(p, self.pos, self.vel, self.mass, None, None, n, acc, jerk, tid, pot)
        kin = 0.5 * (self.mass * (self.vel * self.vel).sum(1)).sum()
        w = 0.5 * (self.mass * pot).sum()
        return float(kin.item()), float(w.item())

    def predictor_error(self):
        """Relative error |a_pred - a|/|a| of the predicted acceleration of every
        element not re-evaluated at the current tick, against a fresh FP64
        evaluation at the current positions; call it right after a tick that
        is a multiple of 2^k_max has run (every element is then at a step
        boundary, so T_f is its exact time since the last evaluation).  Returns quantiles for
        this integrator's predictor and, on the same state, for the other
        predictors whose inputs it keeps."""
        if self.tick == 0 or (self.tick - 1) % (1 << self.k_max) != 0:
            raise RuntimeError("call right after a tick that is a multiple of 2^k_max")
        n = self.n
        p = grav.params(G=self.G, h=self.h, precision=grav.F64)
        acc = torch.empty(n, 3, dtype=torch.float64, device=self.dev)
        jerk = torch.empty_like(acc)
        tid = torch.empty(n, 6, dtype=torch.float64, device=self.dev)
        if self.systems is None:
            grav.eval_active(p, self.pos, self.vel, self.mass, None, None, n, acc, jerk, tid)
        else:
            idx = torch.arange(n, dtype=torch.int32, device=self.dev)
            grav.eval_batched(p, self.systems, self.pos, self.vel, self.mass, idx, None, n, acc,
                              jerk, tid)
        ones = torch.ones(n, dtype=torch.uint8, device=self.dev)
        zeros = torch.zeros(n, dtype=torch.uint8, device=self.dev)
        stale = self.due == 0
        preds = {"none": self.acc.clone()}
        out = torch.empty_like(acc)
        grav.predict(ones, zeros, self.acc, self.jerk, self.tf, self.dt_min, out)
        preds["jerk"] = out.clone()
        if self.predictor == "poly":
            grav.predict_poly(ones, zeros, self.acc, self.a_prev, self.dt_prev, self.tf, self.dt_min,
                              out)
            preds["poly"] = out.clone()
        res = {}
        ref = acc[stale]
        nrm = ref.norm(dim=1)
        for k, a in preds.items():
            e = ((a[stale] - ref).norm(dim=1) / nrm).cpu()
            if e.numel() == 0:
                res[k] = None
                continue
            q = torch.quantile(e, torch.tensor([0.5, 0.9, 0.99], dtype=e.dtype))
            res[k] = {"median": float(q[0]), "p90": float(q[1]), "p99": float(q[2]),
                      "max": float(e.max()), "elements": int(e.numel())}
        res["mode"] = self.predictor
        return res

    def work_ratio(self) -> float:
        """sum(n_due) / sum(n_active): fraction of the standard scheme's force work."""
        a = float(self.n_active_total.item())
        return float(self.n_due_total.item()) / a if a else 0.0
