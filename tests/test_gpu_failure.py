"""Failure detection on the GPU without a fault: a bounded wait is made to run
out (a transfer that is never issued), the kernel reports GRAV_FLAG_TIMEOUT,
the host reads GRAV_ETIMEOUT, and the context keeps working afterwards.
Also: the predictor's unaligned fallback and host-side rejections."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics

from gpu_util import DEV, T  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    rc = grav.selftest_wait_timeout(2000, flags)
    assert rc == grav.GRAV_ETIMEOUT
    assert int(flags.item()) & grav.FLAG_TIMEOUT
    assert b"expired" in grav.lib().grav_last_error_string()
    # the context is intact: a normal evaluation still runs and is right
    pos, vel, mass = ics.uniform_sphere(700, seed=97)
    ref = O.eval_active(pos, vel, mass, h=0.05)
    n = 700
    acc = torch.zeros(n, 3, dtype=torch.float64, device=DEV)
    jerk, tid = torch.zeros_like(acc), torch.zeros(n, 6, dtype=torch.float64, device=DEV)
    flags.zero_()
    grav.eval_active(grav.params(h=0.05, precision=grav.F64), T(pos), T(vel), T(mass), None, None, n,
                     acc, jerk, tid, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    e = np.linalg.norm(acc.cpu().numpy() - ref["acc"], axis=1) / np.linalg.norm(ref["acc"], axis=1)
    assert e.max() <= 1e-12


def test_selftest_rejects_bad_limits():
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert grav.selftest_wait_timeout(0, flags) == grav.GRAV_EINVAL
    assert grav.selftest_wait_timeout(1 << 21, flags) == grav.GRAV_EINVAL


def test_predict_unaligned_views_bitexact():
    """Row views starting one element in (24-byte offset) take the scalar kernel."""
    n = 4001
    g = ics.rng(98)
    active = (g.uniform(size=n + 1) < 0.8).astype(np.uint8)
    due = ((g.uniform(size=n + 1) < 0.3) & (active == 1)).astype(np.uint8)
    a_last, j_last = g.normal(size=(n + 1, 3)), g.normal(size=(n + 1, 3))
    tf = g.integers(0, 1000, n + 1).astype(np.int64)
    init = g.normal(size=(n + 1, 3))
    want = O.predict(active[1:], due[1:], a_last[1:], j_last[1:], tf[1:], 2.0**-9, init[1:])
    out = T(init)
    grav.predict(T(active, torch.uint8)[1:], T(due, torch.uint8)[1:], T(a_last)[1:], T(j_last)[1:],
                 T(tf, torch.int64)[1:], 2.0**-9, out[1:])
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy()[1:].view(np.uint64), want.view(np.uint64))
