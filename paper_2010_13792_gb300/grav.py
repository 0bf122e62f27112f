"""Python binding of libgrav's C ABI (``include/grav.h``).

Argument marshalling only: every function checks dtypes, devices, shapes and
contiguity of PyTorch CUDA tensors, passes their device pointers and the
current CUDA stream to the library, and raises :class:`GravError` with the
library's error text on a non-zero status.  All arithmetic of the path runs
in libgrav's kernels.  There is no fallback: if the library is missing or was
not built, :func:`lib` raises.

Names follow the C ABI: ``select_due``, ``compact_active``, ``eval_active``,
``predict``, ``assign_bins``, ``eval_backward``, ``measure_fma_peak``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

GRAV_OK = 0
GRAV_EINVAL = -1
GRAV_ECUDA = -2
GRAV_ENONFINITE = -3
GRAV_ETIMEOUT = -4
GRAV_ENOMEM = -5

FLAG_NONFINITE = 1
FLAG_TIMEOUT = 2
FLAG_BADINDEX = 4
FLAG_NOCONVERGE = 8
FLAG_OVERFLOW = 16

F64 = 0
MIXED = 1
PEAK_F32X2 = 2      # grav_measure_fma_peak only: packed FP32x2 FMA

_c_i64 = ctypes.c_int64
_c_i32 = ctypes.c_int32
_c_dbl = ctypes.c_double
_c_ptr = ctypes.c_void_p


class GravError(RuntimeError):
    """A libgrav call returned a non-zero status."""

    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: status {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("G", _c_dbl), ("h", _c_dbl), ("eta", _c_dbl), ("precision", _c_i32),
                ("want_pot", _c_i32), ("tile_config", _c_i32), ("max_split", _c_i32),
                ("box", _c_dbl)]


class TileInfo(ctypes.Structure):
    _fields_ = [("threads", _c_i32), ("targets_per_thread", _c_i32), ("sources_per_tile", _c_i32),
                ("targets_per_block", _c_i32), ("unroll", _c_i32), ("shared_accumulators", _c_i32)]


def params(*, G: float = 1.0, h: float, eta: float = 0.01, precision: int = MIXED,
           want_pot: bool = False, tile_config: int = -1, max_split: int = 0,
           box: float = 0.0) -> Params:
    """box > 0: periodic cube of that side, nearest periodic image."""
    return Params(float(G), float(h), float(eta), int(precision), int(bool(want_pot)),
                  int(tile_config), int(max_split), float(box))


class SoftParams(ctypes.Structure):
    _fields_ = [("n_ngb", _c_dbl), ("tol", _c_dbl), ("max_iter", _c_i32), ("pad", _c_i32)]


def soft_params(*, n_ngb: float = 32.0, tol: float = 1e-12, max_iter: int = 100) -> SoftParams:
    """Support constraint (4 pi/3) h^3 rho = n_ngb m and its iteration limits."""
    return SoftParams(float(n_ngb), float(tol), int(max_iter), 0)


class TreeParams(ctypes.Structure):
    _fields_ = [("theta", _c_dbl), ("alpha", _c_dbl), ("leaf_size", _c_i32), ("pad", _c_i32)]


def tree_params(*, theta: float = 0.5, alpha: float = 0.0, leaf_size: int = 8) -> TreeParams:
    """Opening angle, optional relative criterion and leaf size of the oct-tree."""
    return TreeParams(float(theta), float(alpha), int(leaf_size), 0)


_lock = threading.Lock()
_lib = None

_SIGS = {
    "grav_last_error_string": (ctypes.c_char_p, []),
    "grav_version": (ctypes.c_char_p, []),
    "grav_tile_config_count": (_c_i32, [_c_i32]),
    "grav_tile_config": (ctypes.c_int, [_c_i32, _c_i32, ctypes.POINTER(TileInfo)]),
    "grav_default_tile_config": (_c_i32, [_c_i32, _c_i32, _c_i32, ctypes.c_int64]),
    "grav_select_due": (ctypes.c_int, [_c_i64, _c_i64, _c_i32, _c_ptr, _c_ptr, _c_ptr, _c_dbl,
                                       _c_dbl, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr]),
    "grav_compact_workspace_bytes": (_c_i64, [_c_i64]),
    "grav_compact_active": (ctypes.c_int, [_c_i64, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr]),
    "grav_compact_active_noalloc": (ctypes.c_int, [_c_i64, _c_ptr, _c_ptr, _c_ptr, _c_ptr]),
    "grav_predict": (ctypes.c_int, [_c_i64, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_dbl, _c_ptr,
                                    _c_ptr]),
    "grav_push_history": (ctypes.c_int, [_c_i64, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                         _c_dbl, _c_ptr]),
    "grav_predict_poly": (ctypes.c_int, [_c_i64, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                         _c_dbl, _c_ptr, _c_ptr]),
    "grav_assign_bins": (ctypes.c_int, [_c_i64, _c_i64, _c_i32, _c_dbl, _c_ptr, _c_ptr, _c_ptr,
                                        _c_ptr, _c_ptr]),
    "grav_eval_workspace_bytes": (_c_i64, [ctypes.POINTER(Params), _c_i64, _c_i64]),
    "grav_eval_active": (ctypes.c_int, [ctypes.POINTER(Params), _c_i64, _c_ptr, _c_ptr, _c_ptr,
                                        _c_ptr, _c_ptr, _c_i64, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                        _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr]),
    "grav_batched_workspace_bytes": (_c_i64, [ctypes.POINTER(Params), _c_i32, _c_i64]),
    "grav_eval_batched": (ctypes.c_int, [ctypes.POINTER(Params), _c_i32, _c_ptr, _c_i64, _c_ptr,
                                         _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr, _c_ptr,
                                         _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr]),
    "grav_backward_workspace_bytes": (_c_i64, [ctypes.POINTER(Params), _c_i64]),
    "grav_eval_backward": (ctypes.c_int, [ctypes.POINTER(Params), _c_i64, _c_ptr, _c_ptr, _c_ptr,
                                          _c_dbl, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                          _c_ptr, _c_i64, _c_ptr]),
    "grav_backward_batched_workspace_bytes": (_c_i64, [ctypes.POINTER(Params), _c_i32, _c_i64]),
    "grav_eval_backward_batched": (ctypes.c_int, [ctypes.POINTER(Params), _c_i32, _c_ptr, _c_i64,
                                                  _c_ptr, _c_ptr, _c_ptr, _c_dbl, _c_ptr, _c_ptr,
                                                  _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_i64,
                                                  _c_ptr]),
    "grav_soft_workspace_bytes": (_c_i64, [_c_i64]),
    "grav_soft_solve": (ctypes.c_int, [ctypes.POINTER(SoftParams), _c_i64, _c_ptr, _c_ptr, _c_ptr,
                                       _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr]),
    "grav_eval_soft_workspace_bytes": (_c_i64, [ctypes.POINTER(Params), _c_i64, _c_i64]),
    "grav_eval_soft": (ctypes.c_int, [ctypes.POINTER(Params), _c_i64, _c_ptr, _c_ptr, _c_ptr,
                                      _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr, _c_ptr,
                                      _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr]),
    "grav_tree_workspace_bytes": (_c_i64, [_c_i64, _c_i32]),
    "grav_eval_tree": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(TreeParams), _c_i64,
                                      _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr,
                                      _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                      _c_i64, _c_ptr]),
    "grav_measure_fma_peak": (ctypes.c_int, [_c_i32, _c_dbl, ctypes.POINTER(_c_dbl), _c_ptr]),
    "grav_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_uint32, _c_ptr, _c_ptr]),
}

EXPORTED = tuple(_SIGS)


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded libgrav handle.  Raises if the library has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise GravError(GRAV_EINVAL, "libgrav",
                            f"{path} does not exist: build it first "
                            "(python -m paper_2010_13792_gb300.build)")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _err(where: str, rc: int):
    if rc != GRAV_OK:
        msg = lib().grav_last_error_string()
        raise GravError(rc, where, msg.decode() if msg else "")


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype, name, shape=None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise GravError(GRAV_EINVAL, name, "tensor required")
    if not isinstance(t, torch.Tensor):
        raise GravError(GRAV_EINVAL, name, "expected a torch.Tensor")
    if not t.is_cuda:
        raise GravError(GRAV_EINVAL, name, "tensor must live on a CUDA device")
    if t.dtype != dtype:
        raise GravError(GRAV_EINVAL, name, f"dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise GravError(GRAV_EINVAL, name, "tensor must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise GravError(GRAV_EINVAL, name, f"shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else ctypes.c_void_p(0)


def version() -> str:
    return lib().grav_version().decode()


def default_tile_config(precision: int, n_targets: int = 0, periodic: bool = False,
                        soft: bool = False) -> int:
    """Index of the tile configuration the library picks (tile_config = -1)
    for an evaluation of n_targets targets in a precision and mode."""
    r = int(lib().grav_default_tile_config(int(precision), int(bool(periodic)), int(bool(soft)),
                                           int(n_targets)))
    if r < 0:
        _err("grav_default_tile_config", r)
    return r


def tile_configs(precision: int):
    out = []
    for i in range(lib().grav_tile_config_count(precision)):
        ti = TileInfo()
        _err("grav_tile_config", lib().grav_tile_config(precision, i, ctypes.byref(ti)))
        out.append({"index": i, "threads": ti.threads, "targets_per_thread": ti.targets_per_thread,
                    "sources_per_tile": ti.sources_per_tile, "targets_per_block": ti.targets_per_block,
                    "unroll": ti.unroll, "shared_accumulators": ti.shared_accumulators})
    return out


class Workspace:
    """Caller-owned device scratch (a torch uint8 buffer, 256-byte aligned)."""

    def __init__(self, device=None):
        self.device = device
        self.buf = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        return self.buf[off: off + nbytes]


_default_ws = {}


def _ws(ws, key, device):
    if ws is not None:
        return ws
    w = _default_ws.get((key, device))
    if w is None:
        w = _default_ws[(key, device)] = Workspace()
    return w


# ---------------------------------------------------------------------------
# Selection
# ---------------------------------------------------------------------------


def select_due(tick: int, k_max: int, bin_, tf_ticks, dt_grav, q_f: float, dt_min: float,
               active_out, due_out, flags=None, stream=None, elapsed_out=None):
    n = bin_.numel()
    rc = lib().grav_select_due(
        n, int(tick), int(k_max), _ptr(bin_, torch.int8, "bin", (n,)),
        _ptr(tf_ticks, torch.int64, "tf_ticks", (n,)), _ptr(dt_grav, torch.float64, "dt_grav", (n,)),
        float(q_f), float(dt_min), _ptr(active_out, torch.uint8, "active_out", (n,)),
        _ptr(due_out, torch.uint8, "due_out", (n,)),
        _ptr(elapsed_out, torch.int64, "elapsed_out", (n,), allow_none=True),
        _ptr(flags, torch.int32, "flags", (1,), allow_none=True), _stream(stream))
    _err("grav_select_due", rc)


def compact_workspace_bytes(n: int) -> int:
    r = lib().grav_compact_workspace_bytes(int(n))
    if r < 0:
        _err("grav_compact_workspace_bytes", r)
    return r


def compact_active(flags_u8, idx_out, count_out, workspace: Workspace | None = None, stream=None):
    n = flags_u8.numel()
    dev = flags_u8.device
    nb = compact_workspace_bytes(n)
    buf = _ws(workspace, "compact", dev).get(nb, dev)
    rc = lib().grav_compact_active(
        n, _ptr(flags_u8, torch.uint8, "flags", (n,)), _ptr(idx_out, torch.int32, "idx_out", (n,)),
        _ptr(count_out, torch.int32, "count_out", (1,)), ctypes.c_void_p(buf.data_ptr()), nb,
        _stream(stream))
    _err("grav_compact_active", rc)


COMPACT_NOALLOC_MAX_N = 1 << 26


def compact_active_noalloc(flags_u8, idx_out, count_out, stream=None):
    """compact_active without a workspace (library-resident scratch; n <= 2^26).
    For callers that cannot allocate device memory.  Calls that overlap on the
    GPU share the scratch and race; make the first call on a device before
    any stream capture."""
    n = flags_u8.numel()
    rc = lib().grav_compact_active_noalloc(
        n, _ptr(flags_u8, torch.uint8, "flags", (n,)), _ptr(idx_out, torch.int32, "idx_out", (n,)),
        _ptr(count_out, torch.int32, "count_out", (1,)), _stream(stream))
    _err("grav_compact_active_noalloc", rc)


def predict(active, due, a_last, j_last, tf_ticks, dt_min: float, a_out, stream=None):
    n = active.numel()
    rc = lib().grav_predict(
        n, _ptr(active, torch.uint8, "active", (n,)), _ptr(due, torch.uint8, "due", (n,)),
        _ptr(a_last, torch.float64, "a_last", (n, 3)), _ptr(j_last, torch.float64, "j_last", (n, 3)),
        _ptr(tf_ticks, torch.int64, "tf_ticks", (n,)), float(dt_min),
        _ptr(a_out, torch.float64, "a_out", (n, 3)), _stream(stream))
    _err("grav_predict", rc)


def push_history(due, elapsed, dt_grav, a_last, a_prev, dt_prev, dt_min: float, stream=None):
    n = due.numel()
    rc = lib().grav_push_history(
        n, _ptr(due, torch.uint8, "due", (n,)), _ptr(elapsed, torch.int64, "elapsed", (n,)),
        _ptr(dt_grav, torch.float64, "dt_grav", (n,)), _ptr(a_last, torch.float64, "a_last", (n, 3)),
        _ptr(a_prev, torch.float64, "a_prev", (n, 3)), _ptr(dt_prev, torch.float64, "dt_prev", (n,)),
        float(dt_min), _stream(stream))
    _err("grav_push_history", rc)


def predict_poly(active, due, a_last, a_prev, dt_prev, tf_ticks, dt_min: float, a_out, stream=None):
    n = active.numel()
    rc = lib().grav_predict_poly(
        n, _ptr(active, torch.uint8, "active", (n,)), _ptr(due, torch.uint8, "due", (n,)),
        _ptr(a_last, torch.float64, "a_last", (n, 3)), _ptr(a_prev, torch.float64, "a_prev", (n, 3)),
        _ptr(dt_prev, torch.float64, "dt_prev", (n,)), _ptr(tf_ticks, torch.int64, "tf_ticks", (n,)),
        float(dt_min), _ptr(a_out, torch.float64, "a_out", (n, 3)), _stream(stream))
    _err("grav_predict_poly", rc)


def assign_bins(tick: int, k_max: int, dt_max: float, active, dt_grav, dt_hydro, bin_, stream=None):
    n = active.numel()
    rc = lib().grav_assign_bins(
        n, int(tick), int(k_max), float(dt_max), _ptr(active, torch.uint8, "active", (n,)),
        _ptr(dt_grav, torch.float64, "dt_grav", (n,)),
        _ptr(dt_hydro, torch.float64, "dt_hydro", (n,), allow_none=True),
        _ptr(bin_, torch.int8, "bin", (n,)), _stream(stream))
    _err("grav_assign_bins", rc)


# ---------------------------------------------------------------------------
# Force evaluation
# ---------------------------------------------------------------------------


def eval_workspace_bytes(p: Params, n_src: int, n_idx_max: int) -> int:
    r = lib().grav_eval_workspace_bytes(ctypes.byref(p), int(n_src), int(n_idx_max))
    if r < 0:
        _err("grav_eval_workspace_bytes", r)
    return r


def eval_active(p: Params, pos, vel, mass, idx, n_idx_dev, n_idx_max: int, acc, jerk, tidal,
                pot=None, dt_grav=None, flags=None, workspace: Workspace | None = None,
                stream=None):
    """Direct-sum a, jerk, tidal tensor (and pot, dt_grav) scattered to rows idx."""
    n = mass.numel()
    dev = mass.device
    nb = eval_workspace_bytes(p, n, n_idx_max)
    buf = _ws(workspace, "eval", dev).get(nb, dev)
    rc = lib().grav_eval_active(
        ctypes.byref(p), n, _ptr(pos, torch.float64, "pos", (n, 3)),
        _ptr(vel, torch.float64, "vel", (n, 3)), _ptr(mass, torch.float64, "mass", (n,)),
        _ptr(idx, torch.int32, "idx", allow_none=True),
        _ptr(n_idx_dev, torch.int32, "n_idx_dev", (1,), allow_none=True), int(n_idx_max),
        _ptr(acc, torch.float64, "acc", (n, 3)), _ptr(jerk, torch.float64, "jerk", (n, 3)),
        _ptr(tidal, torch.float64, "tidal", (n, 6)),
        _ptr(pot, torch.float64, "pot", (n,), allow_none=True),
        _ptr(dt_grav, torch.float64, "dt_grav", (n,), allow_none=True),
        _ptr(flags, torch.int32, "flags", (1,), allow_none=True),
        ctypes.c_void_p(buf.data_ptr()), nb, _stream(stream))
    _err("grav_eval_active", rc)


def soft_workspace_bytes(n: int) -> int:
    nb = int(lib().grav_soft_workspace_bytes(int(n)))
    if nb < 0:
        _err("grav_soft_workspace_bytes", nb)
    return nb


def soft_solve(sp: SoftParams, pos, mass, h, zeta=None, omega=None, iters=None, flags=None,
               workspace: Workspace | None = None, stream=None):
    """Supports h (in: guesses, out: solution) and the correction coefficients."""
    n = mass.numel()
    dev = mass.device
    nb = soft_workspace_bytes(n)
    buf = _ws(workspace, "soft", dev).get(nb, dev)
    rc = lib().grav_soft_solve(
        ctypes.byref(sp), n, _ptr(pos, torch.float64, "pos", (n, 3)),
        _ptr(mass, torch.float64, "mass", (n,)), _ptr(h, torch.float64, "h", (n,)),
        _ptr(zeta, torch.float64, "zeta", (n,), allow_none=True),
        _ptr(omega, torch.float64, "omega", (n,), allow_none=True),
        _ptr(iters, torch.int32, "iters", (n,), allow_none=True),
        _ptr(flags, torch.int32, "flags", (1,), allow_none=True),
        ctypes.c_void_p(buf.data_ptr()), nb, _stream(stream))
    _err("grav_soft_solve", rc)


def eval_soft_workspace_bytes(p: Params, n_src: int, n_idx_max: int) -> int:
    nb = int(lib().grav_eval_soft_workspace_bytes(ctypes.byref(p), int(n_src), int(n_idx_max)))
    if nb < 0:
        _err("grav_eval_soft_workspace_bytes", nb)
    return nb


def eval_soft(p: Params, pos, vel, mass, h, zeta, idx, n_idx_dev, n_idx_max: int, acc, jerk, tidal,
              pot=None, dt_grav=None, flags=None, workspace: Workspace | None = None, stream=None):
    """eval_active with per-element supports h and (zeta not None) the correction term."""
    n = mass.numel()
    dev = mass.device
    nb = eval_soft_workspace_bytes(p, n, n_idx_max)
    buf = _ws(workspace, "eval_soft", dev).get(nb, dev)
    rc = lib().grav_eval_soft(
        ctypes.byref(p), n, _ptr(pos, torch.float64, "pos", (n, 3)),
        _ptr(vel, torch.float64, "vel", (n, 3)), _ptr(mass, torch.float64, "mass", (n,)),
        _ptr(h, torch.float64, "h", (n,)), _ptr(zeta, torch.float64, "zeta", (n,), allow_none=True),
        _ptr(idx, torch.int32, "idx", allow_none=True),
        _ptr(n_idx_dev, torch.int32, "n_idx_dev", (1,), allow_none=True), int(n_idx_max),
        _ptr(acc, torch.float64, "acc", (n, 3)), _ptr(jerk, torch.float64, "jerk", (n, 3)),
        _ptr(tidal, torch.float64, "tidal", (n, 6)),
        _ptr(pot, torch.float64, "pot", (n,), allow_none=True),
        _ptr(dt_grav, torch.float64, "dt_grav", (n,), allow_none=True),
        _ptr(flags, torch.int32, "flags", (1,), allow_none=True),
        ctypes.c_void_p(buf.data_ptr()), nb, _stream(stream))
    _err("grav_eval_soft", rc)


def tree_workspace_bytes(n: int, leaf_size: int) -> int:
    nb = int(lib().grav_tree_workspace_bytes(int(n), int(leaf_size)))
    if nb < 0:
        _err("grav_tree_workspace_bytes", nb)
    return nb


def eval_tree(p: Params, tp: TreeParams, pos, vel, mass, idx, n_idx_dev, n_idx_max: int, acc, jerk,
              tidal, pot=None, dt_grav=None, a_old=None, order=None, stats=None, flags=None,
              workspace: Workspace | None = None, stream=None):
    """Oct-tree a, jerk, tidal tensor (and pot, dt_grav) scattered to rows idx."""
    n = mass.numel()
    dev = mass.device
    nb = tree_workspace_bytes(n, tp.leaf_size)
    buf = _ws(workspace, "tree", dev).get(nb, dev)
    rc = lib().grav_eval_tree(
        ctypes.byref(p), ctypes.byref(tp), n, _ptr(pos, torch.float64, "pos", (n, 3)),
        _ptr(vel, torch.float64, "vel", (n, 3)), _ptr(mass, torch.float64, "mass", (n,)),
        _ptr(a_old, torch.float64, "a_old", (n, 3), allow_none=True),
        _ptr(idx, torch.int32, "idx", allow_none=True),
        _ptr(n_idx_dev, torch.int32, "n_idx_dev", (1,), allow_none=True), int(n_idx_max),
        _ptr(acc, torch.float64, "acc", (n, 3)), _ptr(jerk, torch.float64, "jerk", (n, 3)),
        _ptr(tidal, torch.float64, "tidal", (n, 6)),
        _ptr(pot, torch.float64, "pot", (n,), allow_none=True),
        _ptr(dt_grav, torch.float64, "dt_grav", (n,), allow_none=True),
        _ptr(order, torch.int32, "order", (n,), allow_none=True),
        _ptr(stats, torch.int64, "stats", (2,), allow_none=True),
        _ptr(flags, torch.int32, "flags", (1,), allow_none=True),
        ctypes.c_void_p(buf.data_ptr()), nb, _stream(stream))
    _err("grav_eval_tree", rc)


BATCH_MAX_SYSTEMS = 16384


def batched_workspace_bytes(p: Params, n_sys: int, n_total: int) -> int:
    r = lib().grav_batched_workspace_bytes(ctypes.byref(p), int(n_sys), int(n_total))
    if r < 0:
        _err("grav_batched_workspace_bytes", r)
    return r


def systems_table(systems, h=None, device=None):
    """The device array of grav_system {offset, n, h} for eval_batched, as an
    int64 tensor [n_sys, 3] whose last column holds each h's FP64 bits.

    systems: [n_sys, 2] (offset, n); h: None (every system takes the call's
    grav_params h), one value, or one per system (0: the call's h).  A
    tensor already in this form is returned unchanged."""
    if torch.is_tensor(systems) and systems.dim() == 2 and systems.shape[1] == 3:
        return systems
    if device is None:
        device = systems.device if torch.is_tensor(systems) else torch.device("cuda")
    on = torch.as_tensor(systems, dtype=torch.int64).reshape(-1, 2).cpu()
    hs = torch.zeros(on.shape[0], dtype=torch.float64)
    if h is not None:
        hs[:] = torch.as_tensor(h, dtype=torch.float64).cpu()
    tab = torch.cat([on, hs.view(torch.int64)[:, None]], dim=1).contiguous()
    return tab.to(device)


def eval_batched(p: Params, systems, pos, vel, mass, idx, n_idx_dev, n_idx_max: int, acc, jerk,
                 tidal, pot=None, dt_grav=None, flags=None, workspace: Workspace | None = None,
                 stream=None):
    """Force evaluation over independent systems in one launch.

    systems: the int64 CUDA tensor [n_sys, 3] of systems_table (offset, n and
    the bits of each system's h); idx: ascending global target indices
    (int32), count *n_idx_dev or n_idx_max."""
    n = mass.numel()
    n_sys = systems.shape[0] if systems.dim() == 2 else 0
    dev = mass.device
    nb = batched_workspace_bytes(p, n_sys, n)
    buf = _ws(workspace, "batched", dev).get(nb, dev)
    rc = lib().grav_eval_batched(
        ctypes.byref(p), n_sys, _ptr(systems, torch.int64, "systems", (n_sys, 3)), n,
        _ptr(pos, torch.float64, "pos", (n, 3)), _ptr(vel, torch.float64, "vel", (n, 3)),
        _ptr(mass, torch.float64, "mass", (n,)), _ptr(idx, torch.int32, "idx"),
        _ptr(n_idx_dev, torch.int32, "n_idx_dev", (1,), allow_none=True), int(n_idx_max),
        _ptr(acc, torch.float64, "acc", (n, 3)), _ptr(jerk, torch.float64, "jerk", (n, 3)),
        _ptr(tidal, torch.float64, "tidal", (n, 6)),
        _ptr(pot, torch.float64, "pot", (n,), allow_none=True),
        _ptr(dt_grav, torch.float64, "dt_grav", (n,), allow_none=True),
        _ptr(flags, torch.int32, "flags", (1,), allow_none=True),
        ctypes.c_void_p(buf.data_ptr()), nb, _stream(stream))
    _err("grav_eval_batched", rc)


def backward_workspace_bytes(p: Params, n: int) -> int:
    r = lib().grav_backward_workspace_bytes(ctypes.byref(p), int(n))
    if r < 0:
        _err("grav_backward_workspace_bytes", r)
    return r


def eval_backward(p: Params, pos, mass, a_bar, w_bar: float, acc, tidal, pot, pos_bar, mass_bar,
                  flags=None, workspace: Workspace | None = None, stream=None):
    n = mass.numel()
    dev = mass.device
    nb = backward_workspace_bytes(p, n)
    buf = _ws(workspace, "backward", dev).get(nb, dev)
    rc = lib().grav_eval_backward(
        ctypes.byref(p), n, _ptr(pos, torch.float64, "pos", (n, 3)),
        _ptr(mass, torch.float64, "mass", (n,)),
        _ptr(a_bar, torch.float64, "a_bar", (n, 3), allow_none=True), float(w_bar),
        _ptr(acc, torch.float64, "acc", (n, 3), allow_none=True),
        _ptr(tidal, torch.float64, "tidal", (n, 6), allow_none=True),
        _ptr(pot, torch.float64, "pot", (n,), allow_none=True),
        _ptr(pos_bar, torch.float64, "pos_bar", (n, 3)),
        _ptr(mass_bar, torch.float64, "mass_bar", (n,)),
        _ptr(flags, torch.int32, "flags", (1,), allow_none=True),
        ctypes.c_void_p(buf.data_ptr()), nb, _stream(stream))
    _err("grav_eval_backward", rc)


def backward_batched_workspace_bytes(p: Params, n_sys: int, n_total: int) -> int:
    r = lib().grav_backward_batched_workspace_bytes(ctypes.byref(p), int(n_sys), int(n_total))
    if r < 0:
        _err("grav_backward_batched_workspace_bytes", r)
    return r


def eval_backward_batched(p: Params, systems, pos, mass, a_bar, w_bar: float, acc, tidal, pot,
                          pos_bar, mass_bar, flags=None, workspace: Workspace | None = None,
                          stream=None):
    """The adjoint over independent systems in one launch; systems: the
    int64 CUDA tensor [n_sys, 3] of systems_table."""
    n = mass.numel()
    n_sys = systems.shape[0] if systems.dim() == 2 else 0
    dev = mass.device
    nb = backward_batched_workspace_bytes(p, n_sys, n)
    buf = _ws(workspace, "backward_batched", dev).get(nb, dev)
    rc = lib().grav_eval_backward_batched(
        ctypes.byref(p), n_sys, _ptr(systems, torch.int64, "systems", (n_sys, 3)), n,
        _ptr(pos, torch.float64, "pos", (n, 3)), _ptr(mass, torch.float64, "mass", (n,)),
        _ptr(a_bar, torch.float64, "a_bar", (n, 3), allow_none=True), float(w_bar),
        _ptr(acc, torch.float64, "acc", (n, 3), allow_none=True),
        _ptr(tidal, torch.float64, "tidal", (n, 6), allow_none=True),
        _ptr(pot, torch.float64, "pot", (n,), allow_none=True),
        _ptr(pos_bar, torch.float64, "pos_bar", (n, 3)),
        _ptr(mass_bar, torch.float64, "mass_bar", (n,)),
        _ptr(flags, torch.int32, "flags", (1,), allow_none=True),
        ctypes.c_void_p(buf.data_ptr()), nb, _stream(stream))
    _err("grav_eval_backward_batched", rc)


def measure_fma_peak(precision: int, seconds: float = 0.5, stream=None) -> float:
    out = ctypes.c_double()
    rc = lib().grav_measure_fma_peak(int(precision), float(seconds), ctypes.byref(out),
                                     _stream(stream))
    _err("grav_measure_fma_peak", rc)
    return out.value


def selftest_wait_timeout(limit: int, flags, stream=None) -> int:
    """Failure-detection self-test; returns the status (GRAV_ETIMEOUT expected)."""
    return int(lib().grav_selftest_wait_timeout(int(limit), _ptr(flags, torch.int32, "flags", (1,)),
                                                _stream(stream)))
