"""The C-ABI library loads and exports every symbol include/grav.h declares;
host-side argument checks reject bad calls before launching anything (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgrav():
    from paper_2010_13792_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"GRAV_API\s+[\w\s\*]+?\b(grav_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_path():
    names = declared_symbols()
    for want in ("grav_select_due", "grav_compact_active", "grav_eval_active", "grav_predict",
                 "grav_eval_backward", "grav_assign_bins"):
        assert want in names


def test_every_declared_symbol_is_exported(libgrav):
    missing = [n for n in declared_symbols() if not hasattr(libgrav, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2010_13792_gb300 import grav
    assert sorted(grav.EXPORTED) == declared_symbols()


def test_internal_symbols_hidden(libgrav):
    assert not hasattr(libgrav, "_ZN4grav9set_errorEPKcz")


def test_host_side_argument_checks(libgrav):
    from paper_2010_13792_gb300 import grav
    L = grav.lib()
    assert L.grav_select_due(-1, 0, 3, None, None, None, 0.5, 1.0, None, None, None, None, None) == grav.GRAV_EINVAL
    assert L.grav_select_due(4, 0, 63, None, None, None, 0.5, 1.0, None, None, None, None, None) == grav.GRAV_EINVAL
    assert L.grav_select_due(4, 0, 3, None, None, None, -0.5, 1.0, None, None, None, None, None) == grav.GRAV_EINVAL
    assert L.grav_select_due(4, 0, 3, None, None, None, 0.5, 1.0, None, None, None, None, None) == grav.GRAV_EINVAL
    assert b"null" in L.grav_last_error_string()
    assert L.grav_select_due(0, 0, 3, None, None, None, 0.5, 1.0, None, None, None, None, None) == grav.GRAV_OK
    assert L.grav_predict(-2, None, None, None, None, None, 1.0, None, None) == grav.GRAV_EINVAL
    assert L.grav_predict(5, None, None, None, None, None, 0.0, None, None) == grav.GRAV_EINVAL
    assert L.grav_assign_bins(5, -1, 3, 1.0, None, None, None, None, None) == grav.GRAV_EINVAL
    assert L.grav_assign_bins(5, 0, 3, float("inf"), None, None, None, None, None) == grav.GRAV_EINVAL
    assert L.grav_compact_active(-1, None, None, None, None, 0, None) == grav.GRAV_EINVAL
    assert L.grav_compact_workspace_bytes(-5) == grav.GRAV_EINVAL
    assert L.grav_compact_workspace_bytes(10**6) >= 4 * (10**6 // 4096)
    bad = [grav.params(h=0.0), grav.params(h=1.0, eta=0.0), grav.params(h=1.0, G=-1.0),
           grav.params(h=1.0, precision=7), grav.params(h=1.0, tile_config=99),
           grav.params(h=float("nan"))]
    for p in bad:
        assert L.grav_eval_workspace_bytes(ctypes.byref(p), 10, 10) == grav.GRAV_EINVAL
        assert L.grav_eval_active(ctypes.byref(p), 10, None, None, None, None, None, 10, None,
                                  None, None, None, None, None, None, 0, None) == grav.GRAV_EINVAL
    p = grav.params(h=0.1)
    assert L.grav_eval_active(ctypes.byref(p), -1, None, None, None, None, None, 0, None, None,
                              None, None, None, None, None, 0, None) == grav.GRAV_EINVAL
    # idx NULL requires n_idx_max == n_src
    assert L.grav_eval_active(ctypes.byref(p), 10, None, None, None, None, None, 5, None, None,
                              None, None, None, None, None, 0, None) == grav.GRAV_EINVAL
    # empty problems are a no-op
    assert L.grav_eval_active(ctypes.byref(p), 0, None, None, None, None, None, 0, None, None,
                              None, None, None, None, None, 0, None) == grav.GRAV_OK
    assert L.grav_eval_backward(ctypes.byref(p), 0, None, None, None, 0.0, None, None, None,
                                None, None, None, None, 0, None) == grav.GRAV_OK
    assert L.grav_eval_backward(ctypes.byref(p), 4, None, None, None, float("nan"), None, None,
                                None, None, None, None, None, 0, None) == grav.GRAV_EINVAL
    assert L.grav_measure_fma_peak(5, 1.0, None, None) == grav.GRAV_EINVAL


def test_tree_argument_checks(libgrav):
    from paper_2010_13792_gb300 import grav
    L = grav.lib()
    p = grav.params(h=0.01)
    args = lambda n, nmax: (n, None, None, None, None, None, None, nmax, None, None, None, None,
                            None, None, None, None, None, 0, None)
    for tp in (grav.tree_params(theta=-0.1), grav.tree_params(theta=float("nan")),
               grav.tree_params(alpha=-1.0), grav.tree_params(leaf_size=0),
               grav.tree_params(leaf_size=65)):
        assert L.grav_eval_tree(ctypes.byref(p), ctypes.byref(tp), *args(10, 10)) == grav.GRAV_EINVAL
    tp = grav.tree_params()
    assert L.grav_eval_tree(ctypes.byref(p), ctypes.byref(tp), *args(0, 0)) == grav.GRAV_OK
    assert L.grav_eval_tree(ctypes.byref(p), ctypes.byref(tp), *args(10, 11)) == grav.GRAV_EINVAL
    assert L.grav_eval_tree(ctypes.byref(p), ctypes.byref(tp), *args(10, 10)) == grav.GRAV_EINVAL
    pb = grav.params(h=0.01, box=1.0)
    assert L.grav_eval_tree(ctypes.byref(pb), ctypes.byref(tp), *args(10, 10)) == grav.GRAV_EINVAL
    assert L.grav_tree_workspace_bytes(-1, 8) == grav.GRAV_EINVAL
    assert L.grav_tree_workspace_bytes(100, 0) == grav.GRAV_EINVAL
    assert L.grav_tree_workspace_bytes(1 << 20, 8) > (1 << 20) * 24
    assert L.grav_tree_workspace_bytes(1 << 28, 1) == grav.GRAV_EINVAL   # node bound >= 2^31


def test_adaptive_softening_argument_checks(libgrav):
    from paper_2010_13792_gb300 import grav
    L = grav.lib()
    for sp in (grav.soft_params(n_ngb=10.0), grav.soft_params(n_ngb=float("inf")),
               grav.soft_params(tol=0.0), grav.soft_params(tol=1e-17), grav.soft_params(max_iter=0),
               grav.soft_params(max_iter=10001)):
        assert L.grav_soft_solve(ctypes.byref(sp), 10, None, None, None, None, None, None, None,
                                 None, 0, None) == grav.GRAV_EINVAL
    sp = grav.soft_params()
    assert L.grav_soft_solve(ctypes.byref(sp), -1, None, None, None, None, None, None, None, None,
                             0, None) == grav.GRAV_EINVAL
    assert L.grav_soft_solve(ctypes.byref(sp), 0, None, None, None, None, None, None, None, None,
                             0, None) == grav.GRAV_OK
    assert L.grav_soft_solve(ctypes.byref(sp), 10, None, None, None, None, None, None, None, None,
                             0, None) == grav.GRAV_EINVAL
    assert L.grav_soft_workspace_bytes(-1) == grav.GRAV_EINVAL
    assert L.grav_soft_workspace_bytes(1000) >= 1000 * 32
    # adaptive softening is for open boundaries only
    p = grav.params(h=0.1, box=1.0)
    assert L.grav_eval_soft_workspace_bytes(ctypes.byref(p), 10, 10) == grav.GRAV_EINVAL
    assert L.grav_eval_soft(ctypes.byref(p), 10, None, None, None, None, None, None, None, 10, None,
                            None, None, None, None, None, None, 0, None) == grav.GRAV_EINVAL
    p = grav.params(h=0.1)
    assert L.grav_eval_soft(ctypes.byref(p), 0, None, None, None, None, None, None, None, 0, None,
                            None, None, None, None, None, None, 0, None) == grav.GRAV_OK
    # per-element supports are required
    assert L.grav_eval_soft(ctypes.byref(p), 10, None, None, None, None, None, None, None, 10, None,
                            None, None, None, None, None, None, 0, None) == grav.GRAV_EINVAL


def test_python_binding_rejects_cpu_tensors():
    import torch
    from paper_2010_13792_gb300 import grav
    x = torch.zeros(4, dtype=torch.int8)
    with pytest.raises(grav.GravError):
        grav.select_due(0, 2, x, torch.zeros(4, dtype=torch.int64), torch.zeros(4, dtype=torch.float64),
                        0.5, 1.0, torch.zeros(4, dtype=torch.uint8), torch.zeros(4, dtype=torch.uint8))


def test_default_tile_config_choice(libgrav):
    """The configuration tile_config = -1 selects: 768-thread CTAs from 8192
    targets in every mode, 256-thread CTAs below; one FP64 default; bad
    arguments rejected.  Host logic only."""
    from paper_2010_13792_gb300 import grav
    L = grav.lib()
    big = grav.tile_configs(grav.MIXED)[grav.default_tile_config(grav.MIXED, 1 << 20)]
    small = grav.tile_configs(grav.MIXED)[grav.default_tile_config(grav.MIXED, 100)]
    assert big["threads"] == 768 and small["threads"] == 256
    assert grav.default_tile_config(grav.MIXED, 8192) == grav.default_tile_config(grav.MIXED, 1 << 20)
    assert grav.default_tile_config(grav.MIXED, 8191) == grav.default_tile_config(grav.MIXED, 100)
    assert grav.default_tile_config(grav.MIXED, 8191, periodic=True) == \
        grav.default_tile_config(grav.MIXED, 100)
    assert grav.default_tile_config(grav.MIXED, 1 << 18, periodic=True) == \
        grav.default_tile_config(grav.MIXED, 1 << 20)
    assert grav.default_tile_config(grav.MIXED, 1 << 20, soft=True) == \
        grav.default_tile_config(grav.MIXED, 1 << 20)
    assert grav.default_tile_config(grav.F64, 1 << 20) == grav.default_tile_config(grav.F64, 1)
    assert L.grav_default_tile_config(7, 0, 0, 10) == grav.GRAV_EINVAL
    assert L.grav_default_tile_config(grav.MIXED, 0, 0, -1) == grav.GRAV_EINVAL
    # index -1 of grav_tile_config describes the small-set default
    ti = grav.TileInfo()
    assert L.grav_tile_config(grav.MIXED, -1, ctypes.byref(ti)) == grav.GRAV_OK
    assert ti.threads == small["threads"]


def test_batched_argument_checks(libgrav):
    """Host-side checks of the batched force evaluation and the batched
    adjoint (no launch happens for any of these)."""
    from paper_2010_13792_gb300 import grav
    L = grav.lib()
    p = grav.params(h=0.01)
    fwd = lambda n_sys, n_total, nmax: L.grav_eval_batched(
        ctypes.byref(p), n_sys, None, n_total, None, None, None, None, None, nmax, None, None,
        None, None, None, None, None, 0, None)
    assert fwd(-1, 10, 10) == grav.GRAV_EINVAL
    assert fwd(16385, 10, 10) == grav.GRAV_EINVAL          # past GRAV_BATCH_MAX_SYSTEMS
    assert fwd(2, 10, 11) == grav.GRAV_EINVAL              # n_idx_max > n_total
    assert fwd(0, 10, 10) == grav.GRAV_OK                  # no systems: nothing to do
    assert fwd(2, 10, 10) == grav.GRAV_EINVAL              # null arrays
    bwd = lambda pp, n_sys, n_total, w: L.grav_eval_backward_batched(
        ctypes.byref(pp), n_sys, None, n_total, None, None, None, w, None, None, None, None, None,
        None, None, 0, None)
    assert bwd(p, -1, 10, 0.0) == grav.GRAV_EINVAL
    assert bwd(p, 16385, 10, 0.0) == grav.GRAV_EINVAL
    assert bwd(p, 2, -1, 0.0) == grav.GRAV_EINVAL
    assert bwd(p, 2, 10, float("nan")) == grav.GRAV_EINVAL
    assert bwd(p, 0, 10, 0.0) == grav.GRAV_OK
    assert bwd(p, 2, 10, 0.0) == grav.GRAV_EINVAL          # null arrays
    assert bwd(grav.params(h=0.01, box=1.0), 2, 10, 0.0) == grav.GRAV_EINVAL   # open boundaries only
    assert L.grav_backward_batched_workspace_bytes(ctypes.byref(p), -1, 10) == grav.GRAV_EINVAL
    assert L.grav_backward_batched_workspace_bytes(ctypes.byref(p), 4, 1 << 20) > (1 << 20) * 16


def test_systems_table_layout():
    """grav.systems_table: int64 [n_sys, 3] of (offset, n, bits of h), the
    layout of grav_system {int64 offset; int64 n; double h;}."""
    import numpy as np
    import torch

    from paper_2010_13792_gb300 import grav

    class GravSystem(ctypes.Structure):
        _fields_ = [("offset", ctypes.c_int64), ("n", ctypes.c_int64), ("h", ctypes.c_double)]

    assert ctypes.sizeof(GravSystem) == 24
    t = grav.systems_table([[0, 10], [10, 5], [15, 7]], h=[1e-3, 0.0, 0.25], device="cpu")
    assert t.dtype == torch.int64 and tuple(t.shape) == (3, 3)
    raw = bytes(t.contiguous().numpy().tobytes())
    recs = (GravSystem * 3).from_buffer_copy(raw)
    assert [(r.offset, r.n, r.h) for r in recs] == [(0, 10, 1e-3), (10, 5, 0.0), (15, 7, 0.25)]
    # no h: every system takes the call's h (0); one h: broadcast
    assert torch.equal(grav.systems_table(np.array([[0, 4]]), device="cpu")[:, 2], torch.zeros(1, dtype=torch.int64))
    t2 = grav.systems_table(torch.tensor([[0, 4], [4, 4]]), h=0.5, device="cpu")
    assert t2[:, 2].clone().view(torch.float64).tolist() == [0.5, 0.5]
    # a table already in this form passes through unchanged
    assert grav.systems_table(t) is t
