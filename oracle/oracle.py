"""Python front end of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The product path (the CUDA library and
its binding) never imports this module, and this module imports nothing from
the product path.

Each function follows the paper passage named in ``oracle.c``; this file only
marshals NumPy arrays into the C routines and builds the shared object with
``gcc -O2 -fopenmp -ffp-contract=off`` (no FMA contraction, so selection and
binning are single correctly rounded IEEE operations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i8p = ctypes.POINTER(ctypes.c_int8)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle into a shared object (gcc, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building first if needed) the oracle library; returns the ctypes handle."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        p = path or build()
        lib = ctypes.CDLL(p)
        lib.oracle_kernel.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        lib.oracle_kernel.restype = None
        lib.oracle_tidal_dt.argtypes = [_dp, ctypes.c_double]
        lib.oracle_tidal_dt.restype = ctypes.c_double
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_eval.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_int64, _i32p,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        lib.oracle_eval.restype = ctypes.c_int
        lib.oracle_select_due.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _i8p,
                                          _i64p, _dp, ctypes.c_double, ctypes.c_double, _u8p, _u8p,
                                          _i64p]
        lib.oracle_select_due.restype = ctypes.c_int
        lib.oracle_compact.argtypes = [ctypes.c_int64, _u8p, _i32p, _i32p]
        lib.oracle_compact.restype = ctypes.c_int
        lib.oracle_predict.argtypes = [ctypes.c_int64, _u8p, _u8p, _dp, _dp, _i64p,
                                       ctypes.c_double, _dp]
        lib.oracle_predict.restype = ctypes.c_int
        lib.oracle_push_history.argtypes = [ctypes.c_int64, _u8p, _i64p, _dp, _dp, _dp, _dp,
                                            ctypes.c_double]
        lib.oracle_push_history.restype = ctypes.c_int
        lib.oracle_predict_poly.argtypes = [ctypes.c_int64, _u8p, _u8p, _dp, _dp, _dp, _i64p,
                                            ctypes.c_double, _dp]
        lib.oracle_predict_poly.restype = ctypes.c_int
        lib.oracle_assign_bins.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_double, _u8p, _dp, _dp, _i8p]
        lib.oracle_assign_bins.restype = ctypes.c_int
        lib.oracle_backward.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, _dp, _dp,
                                        _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                        _i32p, _dp, _dp, ctypes.c_int]
        lib.oracle_backward.restype = ctypes.c_int
        lib.oracle_conditioning.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_int64, _i32p,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             _dp, ctypes.c_int]
        lib.oracle_conditioning.restype = ctypes.c_int
        lib.oracle_kernel_w.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp]
        lib.oracle_kernel_w.restype = None
        lib.oracle_soft_sums.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        lib.oracle_soft_sums.restype = ctypes.c_int
        lib.oracle_soft_solve.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int32, _dp, _dp, _dp, _i32p,
                                          ctypes.c_int]
        lib.oracle_soft_solve.restype = ctypes.c_int
        lib.oracle_eval_soft.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, ctypes.c_int64,
                                         _i32p, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp,
                                         _dp, _dp, ctypes.c_int]
        lib.oracle_eval_soft.restype = ctypes.c_int
        lib.oracle_tree_eval.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_int64, _i32p,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int32, ctypes.c_double, _dp,
                                         _dp, _dp, _dp, _dp, _dp, _i64p, _i64p, _i64p, ctypes.c_int]
        lib.oracle_tree_eval.restype = ctypes.c_int
        if path is None:
            _lib = lib
        return lib


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _c(a, dtype, shape=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a


def max_threads() -> int:
    return int(load().oracle_max_threads())


def kernel(r: float, h: float, lib=None):
    """(f, g, phi) of the cubic-spline kernel at separation r, support h."""
    f, g, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    (lib or load()).oracle_kernel(float(r), float(h), ctypes.byref(f), ctypes.byref(g), ctypes.byref(p))
    return f.value, g.value, p.value


def tidal_dt(t6, eta: float, lib=None) -> float:
    t6 = _c(t6, np.float64, (6,))
    return float((lib or load()).oracle_tidal_dt(_p(t6, _dp), float(eta)))


def eval_active(pos, vel, mass, idx=None, *, G=1.0, h, eta=0.01, want_pot=True,
                nthreads: int = 0, lib=None, box=0.0):
    """Direct-sum a, jerk, tidal tensor (6), potential and dt_grav at targets
    (box > 0: nearest periodic image in a cube of that side).

    Returns a dict of arrays indexed by target slot (row t is element idx[t]).
    """
    lib = lib or load()
    pos = _c(pos, np.float64)
    vel = _c(vel, np.float64)
    mass = _c(mass, np.float64)
    n = mass.shape[0]
    if idx is not None:
        idx = _c(idx, np.int32)
        nt = idx.shape[0]
    else:
        nt = n
    out = {
        "acc": np.zeros((nt, 3)), "jerk": np.zeros((nt, 3)), "tidal": np.zeros((nt, 6)),
        "pot": np.zeros(nt) if want_pot else None, "dt_grav": np.zeros(nt),
    }
    rc = lib.oracle_eval(n, _p(pos, _dp), _p(vel, _dp), _p(mass, _dp), nt, _p(idx, _i32p),
                         float(G), float(h), float(eta), float(box), _p(out["acc"], _dp),
                         _p(out["jerk"], _dp), _p(out["tidal"], _dp), _p(out["pot"], _dp),
                         _p(out["dt_grav"], _dp), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_eval: bad arguments")
    return out


def conditioning(pos, vel, mass, idx=None, *, G=1.0, h, box=0.0, nthreads: int = 0, lib=None):
    """Per target the sums of pair magnitudes sum_j |a_ij|, sum_j |j_ij| and
    sum_j ||T_ij||_F over the pairs of eval_active; returns an [n_tgt, 3]
    array.  kappa_i = (that sum) / |a_i| (resp. |j_i|, ||T_i||_F) is the
    conditioning of target i's sum."""
    pos = _c(pos, np.float64, (-1, 3))
    vel = _c(vel, np.float64, (-1, 3))
    mass = _c(mass, np.float64)
    n = mass.shape[0]
    if idx is None:
        it, n_t = None, n
    else:
        it = _c(idx, np.int32)
        n_t = it.shape[0]
    cond = np.zeros((n_t, 3))
    rc = (lib or load()).oracle_conditioning(n, _p(pos, _dp), _p(vel, _dp), _p(mass, _dp), n_t,
                                             _p(it, _i32p), float(G), float(h), float(box),
                                             _p(cond, _dp), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_conditioning: bad arguments")
    return cond


def kernel_w(r: float, h: float, lib=None):
    """(W, dW/dr, dW/dh, dpsi/dh) of the cubic-spline kernel (psi = the
    potential kernel phi of `kernel`)."""
    v = [ctypes.c_double() for _ in range(4)]
    (lib or load()).oracle_kernel_w(float(r), float(h), *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def soft_sums(pos, mass, h, *, nthreads: int = 0, lib=None):
    """(rho, rho_h, psi_h) per element at supports h: sum_j m_j W(r_ij, h_i) and
    sum_j m_j dW/dh (j = i included), sum_{j != i} m_j dpsi(r_ij, h_i)/dh."""
    pos = _c(pos, np.float64)
    mass = _c(mass, np.float64)
    h = _c(h, np.float64)
    n = mass.shape[0]
    rho, rho_h, psi_h = np.zeros(n), np.zeros(n), np.zeros(n)
    rc = (lib or load()).oracle_soft_sums(n, _p(pos, _dp), _p(mass, _dp), _p(h, _dp), _p(rho, _dp),
                                          _p(rho_h, _dp), _p(psi_h, _dp), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_soft_sums: bad arguments")
    return rho, rho_h, psi_h


def soft_solve(pos, mass, h0, *, n_ngb: float, tol: float = 1e-13, max_iter: int = 100,
               nthreads: int = 0, lib=None):
    """Supports h_i with (4 pi/3) h_i^3 rho_i = n_ngb m_i, and the correction
    coefficients; returns a dict h, zeta, omega, iters (-1: not converged)."""
    pos = _c(pos, np.float64)
    mass = _c(mass, np.float64)
    n = mass.shape[0]
    h = np.array(np.broadcast_to(np.asarray(h0, np.float64), (n,)), dtype=np.float64, copy=True)
    zeta, omega = np.zeros(n), np.zeros(n)
    iters = np.zeros(n, np.int32)
    rc = (lib or load()).oracle_soft_solve(n, _p(pos, _dp), _p(mass, _dp), float(n_ngb), float(tol),
                                           int(max_iter), _p(h, _dp), _p(zeta, _dp),
                                           _p(omega, _dp), _p(iters, _i32p), int(nthreads))
    if rc < 0:
        raise ValueError("oracle_soft_solve: bad arguments")
    return {"h": h, "zeta": zeta, "omega": omega, "iters": iters, "converged": rc == 0}


def eval_soft(pos, vel, mass, h, zeta=None, idx=None, *, G=1.0, eta=0.01, want_pot=True,
              nthreads: int = 0, lib=None):
    """Direct sums with per-element supports h (kernels averaged over the
    pair) and, when zeta is given, the adaptive-softening correction to a."""
    lib = lib or load()
    pos = _c(pos, np.float64)
    vel = _c(vel, np.float64)
    mass = _c(mass, np.float64)
    h = _c(h, np.float64)
    zeta = None if zeta is None else _c(zeta, np.float64)
    n = mass.shape[0]
    if idx is not None:
        idx = _c(idx, np.int32)
        nt = idx.shape[0]
    else:
        nt = n
    out = {
        "acc": np.zeros((nt, 3)), "jerk": np.zeros((nt, 3)), "tidal": np.zeros((nt, 6)),
        "pot": np.zeros(nt) if want_pot else None, "dt_grav": np.zeros(nt),
    }
    rc = lib.oracle_eval_soft(n, _p(pos, _dp), _p(vel, _dp), _p(mass, _dp), _p(h, _dp),
                              _p(zeta, _dp), nt, _p(idx, _i32p), float(G), float(eta),
                              _p(out["acc"], _dp), _p(out["jerk"], _dp), _p(out["tidal"], _dp),
                              _p(out["pot"], _dp), _p(out["dt_grav"], _dp), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_eval_soft: bad arguments")
    return out


def tree_eval(pos, vel, mass, idx=None, *, G=1.0, h, eta=0.01, theta=0.5, leaf_size=8,
              alpha=0.0, a_old=None, want_pot=True, nthreads: int = 0, lib=None):
    """Oct-tree (Barnes-Hut, monopole) a, jerk, tidal, potential and dt_grav at
    targets; also returns the tree order, node count and interaction count."""
    lib = lib or load()
    pos = _c(pos, np.float64)
    vel = _c(vel, np.float64)
    mass = _c(mass, np.float64)
    a_old = None if a_old is None else _c(a_old, np.float64)
    n = mass.shape[0]
    if idx is not None:
        idx = _c(idx, np.int32)
        nt = idx.shape[0]
    else:
        nt = n
    out = {
        "acc": np.zeros((nt, 3)), "jerk": np.zeros((nt, 3)), "tidal": np.zeros((nt, 6)),
        "pot": np.zeros(nt) if want_pot else None, "dt_grav": np.zeros(nt),
        "order": np.zeros(n, np.int64),
    }
    nn = np.zeros(1, np.int64)
    ni = np.zeros(1, np.int64)
    rc = lib.oracle_tree_eval(n, _p(pos, _dp), _p(vel, _dp), _p(mass, _dp), nt, _p(idx, _i32p),
                              float(G), float(h), float(eta), float(theta), int(leaf_size),
                              float(alpha), _p(a_old, _dp), _p(out["acc"], _dp),
                              _p(out["jerk"], _dp), _p(out["tidal"], _dp), _p(out["pot"], _dp),
                              _p(out["dt_grav"], _dp), _p(out["order"], _i64p), _p(nn, _i64p),
                              _p(ni, _i64p), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_tree_eval: bad arguments")
    out["n_nodes"] = int(nn[0])
    out["interactions"] = int(ni[0])
    return out


def select_due(tick, k_max, bin_, tf_ticks, dt_grav, q_f, dt_min, lib=None, elapsed=None):
    """Counter update and due test; returns (active, due, tf_ticks_new), plus
    the elapsed ticks of due elements (a copy of `elapsed`, updated) when
    `elapsed` is given."""
    bin_ = _c(bin_, np.int8)
    tf = np.array(tf_ticks, dtype=np.int64, copy=True)
    dt_grav = _c(dt_grav, np.float64)
    n = bin_.shape[0]
    active = np.zeros(n, np.uint8)
    due = np.zeros(n, np.uint8)
    el = None if elapsed is None else np.array(elapsed, dtype=np.int64, copy=True)
    rc = (lib or load()).oracle_select_due(n, int(tick), int(k_max), _p(bin_, _i8p), _p(tf, _i64p),
                                  _p(dt_grav, _dp), float(q_f), float(dt_min),
                                  _p(active, _u8p), _p(due, _u8p), _p(el, _i64p))
    if rc != 0:
        raise ValueError("oracle_select_due: bad arguments")
    if el is not None:
        return active, due, tf, el
    return active, due, tf


def compact(flags, lib=None):
    flags = _c(flags, np.uint8)
    n = flags.shape[0]
    idx = np.zeros(max(n, 1), np.int32)
    cnt = ctypes.c_int32()
    rc = (lib or load()).oracle_compact(n, _p(flags, _u8p), _p(idx, _i32p), ctypes.byref(cnt))
    if rc != 0:
        raise ValueError("oracle_compact: bad arguments")
    return idx[: cnt.value].copy()


def predict(active, due, a_last, j_last, tf_ticks, dt_min, a_out, lib=None):
    active = _c(active, np.uint8)
    due = _c(due, np.uint8)
    a_last = _c(a_last, np.float64)
    j_last = _c(j_last, np.float64)
    tf = _c(tf_ticks, np.int64)
    out = np.array(a_out, dtype=np.float64, copy=True)
    rc = (lib or load()).oracle_predict(active.shape[0], _p(active, _u8p), _p(due, _u8p),
                               _p(a_last, _dp), _p(j_last, _dp), _p(tf, _i64p),
                               float(dt_min), _p(out, _dp))
    if rc != 0:
        raise ValueError("oracle_predict: bad arguments")
    return out


def push_history(due, elapsed, dt_grav, a_last, a_prev, dt_prev, dt_min, lib=None):
    """Log the previous evaluation of due elements; returns (a_prev, dt_prev)."""
    due = _c(due, np.uint8)
    el = _c(elapsed, np.int64)
    dtg = _c(dt_grav, np.float64)
    a_last = _c(a_last, np.float64)
    ap = np.array(a_prev, dtype=np.float64, copy=True)
    dp = np.array(dt_prev, dtype=np.float64, copy=True)
    rc = (lib or load()).oracle_push_history(due.shape[0], _p(due, _u8p), _p(el, _i64p), _p(dtg, _dp),
                                             _p(a_last, _dp), _p(ap, _dp), _p(dp, _dp), float(dt_min))
    if rc != 0:
        raise ValueError("oracle_push_history: bad arguments")
    return ap, dp


def predict_poly(active, due, a_last, a_prev, dt_prev, tf_ticks, dt_min, a_out, lib=None):
    active = _c(active, np.uint8)
    due = _c(due, np.uint8)
    a_last = _c(a_last, np.float64)
    a_prev = _c(a_prev, np.float64)
    dt_prev = _c(dt_prev, np.float64)
    tf = _c(tf_ticks, np.int64)
    out = np.array(a_out, dtype=np.float64, copy=True)
    rc = (lib or load()).oracle_predict_poly(active.shape[0], _p(active, _u8p), _p(due, _u8p),
                                             _p(a_last, _dp), _p(a_prev, _dp), _p(dt_prev, _dp),
                                             _p(tf, _i64p), float(dt_min), _p(out, _dp))
    if rc != 0:
        raise ValueError("oracle_predict_poly: bad arguments")
    return out


def assign_bins(tick, k_max, dt_max, active, dt_grav, dt_hydro, bin_, lib=None):
    active = _c(active, np.uint8)
    dt_grav = _c(dt_grav, np.float64)
    dth = None if dt_hydro is None else _c(dt_hydro, np.float64)
    out = np.array(bin_, dtype=np.int8, copy=True)
    rc = (lib or load()).oracle_assign_bins(active.shape[0], int(tick), int(k_max), float(dt_max),
                                   _p(active, _u8p), _p(dt_grav, _dp), _p(dth, _dp),
                                   _p(out, _i8p))
    if rc != 0:
        raise ValueError("oracle_assign_bins: bad arguments")
    return out


def backward(pos, mass, a_bar, w_bar, acc, tidal, pot, *, G=1.0, h, nthreads: int = 0,
             lib=None, rows=None):
    """Adjoint sums: returns (pos_bar [n,3], mass_bar [n]); with `rows` only
    those rows are computed (the others are 0)."""
    pos = _c(pos, np.float64)
    mass = _c(mass, np.float64)
    n = mass.shape[0]
    a_bar = None if a_bar is None else _c(a_bar, np.float64)
    acc = None if acc is None else _c(acc, np.float64)
    tidal = None if tidal is None else _c(tidal, np.float64)
    pot = None if pot is None else _c(pot, np.float64)
    pb = np.zeros((n, 3))
    mb = np.zeros(n)
    sel = None if rows is None else _c(rows, np.int32)
    rc = (lib or load()).oracle_backward(n, _p(pos, _dp), _p(mass, _dp), _p(a_bar, _dp), float(w_bar),
                                _p(acc, _dp), _p(tidal, _dp), _p(pot, _dp), float(G), float(h),
                                0 if sel is None else sel.size, _p(sel, _i32p),
                                _p(pb, _dp), _p(mb, _dp), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_backward: bad arguments")
    return pb, mb


def potential_energy(mass, pot) -> float:
    """W = 1/2 sum_i m_i Phi_i (self term excluded in Phi)."""
    return 0.5 * float(np.dot(np.asarray(mass, np.float64), np.asarray(pot, np.float64)))
