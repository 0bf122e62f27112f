"""grav_compact_active_noalloc: the compaction entry point that allocates
nothing, for callers that cannot allocate device memory (its scratch is a
fixed array inside the library).  Called through the C ABI and compared with
grav_compact_active on two calls in a row; kept in a file of its own that
runs last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2010_13792_gb300 import grav, ics

pytestmark = pytest.mark.gpu


def _compact_both(flags_np, dev):
    n = flags_np.size
    L = grav.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    f = torch.as_tensor(flags_np, device=dev)
    idx_a = torch.full((n,), -1, dtype=torch.int32, device=dev)
    cnt_a = torch.full((1,), -1, dtype=torch.int32, device=dev)
    ws_bytes = L.grav_compact_workspace_bytes(n)
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    off = (-ws.data_ptr()) % 256
    rc = L.grav_compact_active(n, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(idx_a.data_ptr()),
                               ctypes.c_void_p(cnt_a.data_ptr()),
                               ctypes.c_void_p(ws.data_ptr() + off), ws_bytes, stream)
    assert rc == grav.GRAV_OK
    idx_b = torch.full((n,), -1, dtype=torch.int32, device=dev)
    cnt_b = torch.full((1,), -1, dtype=torch.int32, device=dev)
    rc = L.grav_compact_active_noalloc(n, ctypes.c_void_p(f.data_ptr()),
                                       ctypes.c_void_p(idx_b.data_ptr()),
                                       ctypes.c_void_p(cnt_b.data_ptr()), stream)
    assert rc == grav.GRAV_OK, L.grav_last_error_string()
    torch.cuda.synchronize()
    return idx_a.cpu().numpy(), int(cnt_a.item()), idx_b.cpu().numpy(), int(cnt_b.item())


def test_noalloc_matches_workspace_compaction_twice():
    dev = torch.device("cuda:0")
    g = ics.rng(900)
    # two calls in a row with different sizes and densities: the second must
    # not see anything the first left in the shared scratch
    for n, p in (((1 << 20) + 77, 0.3), (50001, 0.9)):
        flags = (g.uniform(size=n) < p).astype(np.uint8)
        ia, ca, ib, cb = _compact_both(flags, dev)
        assert ca == cb == int(flags.astype(bool).sum())
        assert np.array_equal(ia, ib)
        assert np.array_equal(ib[:cb], np.flatnonzero(flags))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = grav.lib()
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    rc = L.grav_compact_active_noalloc(grav.COMPACT_NOALLOC_MAX_N + 1, ctypes.c_void_p(8),
                                       ctypes.c_void_p(8), ctypes.c_void_p(cnt.data_ptr()), None)
    assert rc == grav.GRAV_EINVAL
    assert b"outside" in L.grav_last_error_string()


@pytest.mark.parametrize("n", [grav.COMPACT_NOALLOC_MAX_N - 1, grav.COMPACT_NOALLOC_MAX_N])
def test_noalloc_at_its_size_limit(n):
    """n = 2^26 (16384 blocks of 4096 flags: every scratch element, one
    single-CTA scan over all of them) and one flag below it (a ragged last
    block)."""
    dev = torch.device("cuda:0")
    flags = (ics.rng(901 + n % 7).uniform(size=n) < 0.25).astype(np.uint8)
    flags[-1] = 1
    ia, ca, ib, cb = _compact_both(flags, dev)
    assert ca == cb == int(flags.astype(bool).sum())
    assert np.array_equal(ia, ib)
    assert ib[cb - 1] == n - 1
