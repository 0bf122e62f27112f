"""GPU selection, compaction, predictor and bins against the oracle: bit-exact
(integer and flag outputs are compared exactly, the predictor's FP64 output
byte for byte, since both sides make the same correctly rounded operations)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2010_13792_gb300 import grav, ics

pytestmark = pytest.mark.gpu

from gpu_util import DEV, T  # noqa: E402


def _state(n, k_max, seed, dt_min):
    g = ics.rng(seed)
    bins = g.integers(0, k_max + 1, n).astype(np.int8)
    tf = g.integers(0, 3 * 2**k_max, n).astype(np.int64)
    dtg = g.uniform(0.0, 4.0 * 2**k_max, n) * dt_min
    if n:
        dtg[g.uniform(size=n) < 0.1] = 0.0
        dtg[g.uniform(size=n) < 0.05] = np.inf
        k = g.integers(1, 200, n)
        eq = g.uniform(size=n) < 0.2
        dtg[eq] = (k[eq] * dt_min) * 2.0                # equality cases at q_f = 1/2
    return bins, tf, dtg


@pytest.mark.parametrize("n", [0, 1, 17, 4097, (1 << 20) + 3])
@pytest.mark.parametrize("q_f", [0.0, 0.5, 1.0])
def test_select_due_bitexact(n, q_f):
    k_max, dt_min = 6, 2.0**-10
    bins, tf, dtg = _state(n, k_max, 100 + n, dt_min)
    el0 = np.full(n, -5, np.int64)
    for tick in (0, 1, 2, 8, 64, 37, 96):
        a_o, d_o, tf_o, el_o = O.select_due(tick, k_max, bins, tf, dtg, q_f, dt_min, elapsed=el0)
        tf_t = T(tf, torch.int64)
        a_t = torch.full((n,), 7, dtype=torch.uint8, device=DEV)
        d_t = torch.full((n,), 7, dtype=torch.uint8, device=DEV)
        el_t = T(el0, torch.int64)
        grav.select_due(tick, k_max, T(bins, torch.int8), tf_t, T(dtg), q_f, dt_min, a_t, d_t,
                        elapsed_out=el_t)
        torch.cuda.synchronize()
        assert np.array_equal(a_t.cpu().numpy(), a_o)
        assert np.array_equal(d_t.cpu().numpy(), d_o)
        assert np.array_equal(tf_t.cpu().numpy(), tf_o)
        assert np.array_equal(el_t.cpu().numpy(), el_o)
        tf = tf_o


def test_select_bad_bin_sets_flag():
    n, k_max = 64, 4
    bins = np.full(n, 2, np.int8)
    bins[5] = 9
    bins[6] = -1
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    a_t = torch.zeros(n, dtype=torch.uint8, device=DEV)
    d_t = torch.zeros(n, dtype=torch.uint8, device=DEV)
    grav.select_due(0, k_max, T(bins, torch.int8), T(np.zeros(n, np.int64), torch.int64),
                    T(np.zeros(n)), 0.5, 1.0, a_t, d_t, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) & grav.FLAG_BADINDEX
    a = a_t.cpu().numpy()
    assert a[5] == 0 and a[6] == 0 and a[0] == 1


@pytest.mark.parametrize("n", [1, 15, 16, 4095, 4096, 4097, 65536 + 7, (1 << 20) + 5])
@pytest.mark.parametrize("p", [0.0, 0.01, 0.5, 1.0])
def test_compact_bitexact(n, p):
    g = ics.rng(200 + n)
    flags = (g.uniform(size=n) < p).astype(np.uint8)
    flags[flags == 1] = g.integers(1, 256, int(flags.sum()))
    idx_t = torch.full((n,), -7, dtype=torch.int32, device=DEV)
    cnt_t = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    grav.compact_active(T(flags, torch.uint8), idx_t, cnt_t)
    torch.cuda.synchronize()
    want = O.compact(flags)
    c = int(cnt_t.item())
    assert c == want.size
    got = idx_t.cpu().numpy()
    assert np.array_equal(got[:c], want)
    assert np.all(got[c:] == -7)


def test_compact_unaligned_and_empty():
    n = 10001
    g = ics.rng(301)
    big = (g.uniform(size=n + 3) < 0.3).astype(np.uint8)
    bt = T(big, torch.uint8)
    view = bt[3:]                       # 3-byte offset: not 16-byte aligned
    idx_t = torch.zeros(n, dtype=torch.int32, device=DEV)
    cnt_t = torch.zeros(1, dtype=torch.int32, device=DEV)
    grav.compact_active(view, idx_t, cnt_t)
    torch.cuda.synchronize()
    want = O.compact(big[3:])
    assert int(cnt_t.item()) == want.size
    assert np.array_equal(idx_t[: want.size].cpu().numpy(), want)
    e = torch.zeros(0, dtype=torch.uint8, device=DEV)
    cnt_t.fill_(5)
    grav.compact_active(e, torch.zeros(0, dtype=torch.int32, device=DEV), cnt_t)
    torch.cuda.synchronize()
    assert int(cnt_t.item()) == 0


@pytest.mark.parametrize("row_offset", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 1000, (1 << 20) + 1])
def test_predict_bitexact(n, row_offset):
    """Both kernels: 16-byte-aligned [n][3] arrays (pairs of doubles per
    thread, odd and even 3n) and views starting one row (24 bytes) into a
    buffer (one double per thread)."""
    g = ics.rng(400 + n)
    active = (g.uniform(size=n) < 0.7).astype(np.uint8)
    due = ((g.uniform(size=n) < 0.3) & (active == 1)).astype(np.uint8)
    a_last = g.normal(size=(n, 3))
    j_last = g.normal(size=(n, 3)) * 10.0
    tf = g.integers(0, 1 << 12, n).astype(np.int64)
    dt_min = 2.0**-13 * 3.0
    init = g.normal(size=(n, 3))
    want = O.predict(active, due, a_last, j_last, tf, dt_min, init)

    def rows(x):      # a contiguous view row_offset rows into a larger buffer
        buf = T(np.concatenate([np.zeros((row_offset, 3)), x]))
        return buf[row_offset:]
    out = rows(init)
    grav.predict(T(active, torch.uint8), T(due, torch.uint8), rows(a_last), rows(j_last),
                 T(tf, torch.int64), dt_min, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("n", [1, 3000, (1 << 20) + 9])
def test_assign_bins_bitexact(n):
    k_max, dt_max = 10, 0.37
    g = ics.rng(500 + n)
    dtg = dt_max * 2.0 ** g.uniform(-12, 2, n)
    m = min(n, 12)
    dtg[:m] = (dt_max * 2.0 ** -np.arange(12))[:m]
    if n > 24:
        dtg[12:24] = np.nextafter(dtg[:12], 0)
        dtg[24 % n] = np.inf
        dtg[25 % n] = 0.0
        dtg[26 % n] = np.nan
        dtg[27 % n] = -1.0
    dth = np.where(g.uniform(size=n) < 0.3, dt_max * 2.0 ** g.uniform(-12, 1, n), np.inf)
    if n > 30:
        dth[30] = np.nan
    for tick in (0, 1, 6, 512, 1024, 768, 999):
        active = (g.uniform(size=n) < 0.8).astype(np.uint8)
        old = g.integers(0, k_max + 1, n).astype(np.int8)
        for hyd in (dth, None):
            want = O.assign_bins(tick, k_max, dt_max, active, dtg, hyd, old)
            bt = T(old, torch.int8)
            grav.assign_bins(tick, k_max, dt_max, T(active, torch.uint8), T(dtg),
                             None if hyd is None else T(hyd), bt)
            torch.cuda.synchronize()
            assert np.array_equal(bt.cpu().numpy(), want), tick


@pytest.mark.parametrize("n", [1, 999, (1 << 20) + 3])
def test_polynomial_predictor_bitexact(n):
    """Logged history and the first-order polynomial predictor against the
    oracle over a sequence of selections with mixed bins (byte for byte)."""
    g = ics.rng(600 + n)
    dt_min, k_max = 2.0**-11, 3
    bins = g.integers(0, k_max + 1, n).astype(np.int8)
    dtg = np.zeros(n)
    tf = np.zeros(n, np.int64)
    el = np.zeros(n, np.int64)
    a_prev = np.zeros((n, 3))
    dt_prev = np.zeros(n)
    a_last = g.normal(size=(n, 3))
    tf_t, el_t, ap_t, dp_t = T(tf, torch.int64), T(el, torch.int64), T(a_prev), T(dt_prev)
    act_t = torch.zeros(n, dtype=torch.uint8, device=DEV)
    due_t = torch.zeros(n, dtype=torch.uint8, device=DEV)
    for tick in range(0, 20):
        q_f = 0.0 if tick == 0 else 1.0
        active, due, tf, el = O.select_due(tick, k_max, bins, tf, dtg, q_f, dt_min, elapsed=el)
        a_prev, dt_prev = O.push_history(due, el, dtg, a_last, a_prev, dt_prev, dt_min)
        dtg_t = T(dtg)
        grav.select_due(tick, k_max, T(bins, torch.int8), tf_t, dtg_t, q_f, dt_min, act_t, due_t,
                        elapsed_out=el_t)
        grav.push_history(due_t, el_t, dtg_t, T(a_last), ap_t, dp_t, dt_min)
        torch.cuda.synchronize()
        assert np.array_equal(ap_t.cpu().numpy(), a_prev)
        assert np.array_equal(dp_t.cpu().numpy().view(np.uint64), dt_prev.view(np.uint64))
        a_last = np.where(due[:, None] == 1, g.normal(size=(n, 3)), a_last)
        dtg = np.where(due == 1, g.uniform(0.5, 10.0, n) * dt_min, dtg)
        due2 = ((g.uniform(size=n) < 0.2) & (active == 1)).astype(np.uint8)
        init = g.normal(size=(n, 3))
        want = O.predict_poly(active, due2, a_last, a_prev, dt_prev, tf, dt_min, init)
        out = T(init)
        grav.predict_poly(T(active, torch.uint8), T(due2, torch.uint8), T(a_last), ap_t, dp_t,
                          tf_t, dt_min, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), want.view(np.uint64))
