"""Predictor ablation (run on a GPU): no predictor, the first-order
polynomial through the last two evaluations (Section 2.2) and the jerk
predictor (Eq. jerkupdate), on Plummer spheres, for softenings below and
above the interparticle spacing and for long and short update gaps (q_f).
Prints, per case, the median and 90th-percentile relative error of the
predicted acceleration against a fresh FP64 evaluation after three cycles of
32 ticks, and the fraction of force evaluations done.

    python tests/predictor_ablation.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2010_13792_gb300 import grav, ics  # noqa: E402
from paper_2010_13792_gb300.adaptive import AdaptiveIntegrator  # noqa: E402


def main():
    print("n h q_f | mode median p90 ... | work ratio")
    for n in (1 << 12, 1 << 15):
        pos, vel, mass = ics.plummer(n, seed=ics.BASE_SEED + 1)
        for h in (1e-3, 0.05, 0.2, 0.5):
            for qf in (1.0, 0.25):
                row = []
                for mode in ("none", "poly", "jerk"):
                    it = AdaptiveIntegrator(pos, vel, mass, h=h, q_f=qf, k_max=5, dt_max=2.0**-4,
                                            precision=grav.F64, predictor=mode)
                    it.run(96)
                    r = it.predictor_error()[mode]
                    row.append(f"{mode} {r['median']:.4f} {r['p90']:.4f}")
                print(n, h, qf, "|", " | ".join(row), f"| work {it.work_ratio():.3f}", flush=True)


if __name__ == "__main__":
    main()
