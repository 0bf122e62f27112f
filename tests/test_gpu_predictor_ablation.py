"""Predictor ablation on the GPU (Section 2.2 and Eq. jerkupdate).

Three predictors are compared on Plummer spheres:
- no predictor: the last evaluated acceleration is kept;
- the first-order polynomial through the last two evaluations;
- the jerk predictor.

Softenings lie below and above the interparticle spacing, and the update
gaps are long (q_f = 1) and short (q_f = 1/4).  After three cycles of 32
ticks (k_max = 5, dt_max = 2^-4, FP64 path), each predictor's acceleration
for the elements not re-evaluated at that tick is compared with a fresh FP64
evaluation.  The test asserts that the jerk predictor's median relative error
is below both others' in every case.  That ordering is why the paper uses it.
Run with -s to print the table:

    python -m pytest tests/test_gpu_predictor_ablation.py -m gpu -q -s
"""
import pytest

from paper_2010_13792_gb300 import grav, ics
from paper_2010_13792_gb300.adaptive import AdaptiveIntegrator

CASES = [(n, h, qf) for n in (1 << 12, 1 << 15) for h in (1e-3, 0.05, 0.2, 0.5) for qf in (1.0, 0.25)]
_IC = {}


def _plummer(n):
    if n not in _IC:
        _IC[n] = ics.plummer(n, seed=ics.BASE_SEED + 1)
    return _IC[n]


@pytest.mark.gpu
@pytest.mark.parametrize("n,h,qf", CASES)
def test_jerk_predictor_beats_none_and_polynomial(n, h, qf):
    pos, vel, mass = _plummer(n)
    res, work = {}, None
    for mode in ("none", "poly", "jerk"):
        it = AdaptiveIntegrator(pos, vel, mass, h=h, q_f=qf, k_max=5, dt_max=2.0**-4,
                                precision=grav.F64, predictor=mode)
        it.run(96)
        res[mode] = it.predictor_error()[mode]
        work = it.work_ratio()
    print(f"| {n} | {h:g} | {qf:g} | "
          + " | ".join(f"{res[m]['median']:.4f} / {res[m]['p90']:.3f}" for m in ("none", "poly", "jerk"))
          + f" | {work:.3f} |")
    assert res["jerk"]["median"] < res["none"]["median"]
    assert res["jerk"]["median"] < res["poly"]["median"]
    assert 0.0 < work < 1.0
