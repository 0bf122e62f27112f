"""Pins of the FP64 oracle to facts other than itself.

Each ``pin_*`` function takes an oracle library handle (``oracle.oracle.load``)
and raises AssertionError when the oracle disagrees with something the paper
or the mathematics fixes:

* the cubic-spline kernel functions f, g, phi against a computer-algebra
  integration of the density kernel W (M(<r) = 4 pi int s^2 W, g = f'/r,
  phi = int_r^inf s f) evaluated at 40 digits;
* the pair sums against an mpmath brute force at 40 digits that uses those
  CAS-derived kernels (tiny N, close and far pairs);
* invariants: momentum balance sum m a = 0 and sum m j = 0, trace T =
  -4 pi G sum m W (W from its own definition), the cube-symmetric
  configuration, and the scaling x -> lam x, h -> lam h;
* derivatives: jerk = central difference of a along straight-line drifts
  (Eq. 4 is d a / dt), T = central difference of a in x_i, the adjoint =
  central differences of the loss;
* the tidal timestep of Eq. (tidaltimestep) on tensors whose Frobenius norm
  is known in closed form;
* selection: update counts over a long horizon in closed form, the
  q_f <= 1/2 and q_f = 0 special cases, the counter equal to the time since
  the last update reconstructed from the update history; bins by exact
  rational enumeration; compaction by ``numpy.flatnonzero``;
* the predictor exact on a field linear in time, and equal to the paper's
  incremental update applied step by step;
* adaptive softening: W, dW/dr, dW/dh and dpsi/dh against sympy
  derivatives; the density constraint, Omega and zeta against mpmath brute
  force sums; the corrected acceleration equal to -grad U / m with every
  support re-solved (central differences), the uncorrected one not; equal
  supports reducing to the fixed-h sums bit for bit; momentum balance;
  jerk and tidal tensor as derivatives at fixed supports;
* the oct-tree: Theta = 0 equal to the direct sum; the tree order against
  Morton keys written out independently; monopole error bounds at Theta =
  0.5 shrinking with Theta; a far cluster acting as one moving point mass;
  jerk and tidal tensor as derivatives of the tree field; the relative
  criterion only opening more nodes.

The mutation test runs these pins against copies of the oracle with planted
mistakes and requires every mutant to fail at least one pin.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

from oracle import oracle as O
from paper_2010_13792_gb300 import ics

# ---------------------------------------------------------------------------
# Independent kernel: CAS integration of the cubic-spline density kernel.
# ---------------------------------------------------------------------------


@lru_cache(maxsize=1)
def cas_kernel():
    """Return mpmath callables (f, g, phi, W) in units h = 1, from sympy."""
    import sympy as sp
    s, u = sp.symbols("s u", positive=True)
    # density kernel of unit support: W = 8/pi * w(u)
    w_in = 1 - 6 * s**2 + 6 * s**3
    w_out = 2 * (1 - s) ** 3
    c = sp.Rational(8) / sp.pi
    m_in = sp.integrate(4 * sp.pi * s**2 * c * w_in, (s, 0, u))
    m_half = m_in.subs(u, sp.Rational(1, 2))
    m_out = m_half + sp.integrate(4 * sp.pi * s**2 * c * w_out, (s, sp.Rational(1, 2), u))
    f_in = sp.simplify(m_in / u**3)
    f_out = sp.simplify(m_out / u**3)
    g_in = sp.simplify(sp.diff(f_in, u) / u)
    g_out = sp.simplify(sp.diff(f_out, u) / u)
    # phi(u) = 1 + int_u^1 s f(s) ds for u < 1 (phi = 1/u beyond the support)
    phi_out = 1 + sp.integrate((s * f_out.subs(u, s)), (s, u, 1))
    phi_half = phi_out.subs(u, sp.Rational(1, 2))
    phi_in = phi_half + sp.integrate((s * f_in.subs(u, s)), (s, u, sp.Rational(1, 2)))
    mods = "mpmath"
    F = [sp.lambdify(u, e, mods) for e in (f_in, f_out, g_in, g_out, phi_in, phi_out)]
    W = [sp.lambdify(u, c * e.subs(s, u), mods) for e in (w_in, w_out)]
    total_mass = m_out.subs(u, 1)
    return F, W, sp.nsimplify(total_mass)


def kernel_mp(r, h):
    """(f, g, phi) at separation r (mpmath numbers), support h, via the CAS forms."""
    import mpmath as mp
    (f_in, f_out, g_in, g_out, p_in, p_out), _, _ = cas_kernel()
    r = mp.mpf(r)
    h = mp.mpf(h)
    u = r / h
    if u >= 1:
        return 1 / r**3, -3 / r**5, 1 / r
    if u < mp.mpf(1) / 2:
        return f_in(u) / h**3, g_in(u) / h**5, p_in(u) / h
    return f_out(u) / h**3, g_out(u) / h**5, p_out(u) / h


def W_def(r, h):
    """Cubic-spline density kernel, straight from its definition (numpy)."""
    u = np.asarray(r, np.float64) / h
    w = np.where(u < 0.5, 1 - 6 * u**2 + 6 * u**3, np.where(u < 1.0, 2 * (1 - u) ** 3, 0.0))
    return 8.0 / (np.pi * h**3) * w


# ---------------------------------------------------------------------------
# Kernel pins
# ---------------------------------------------------------------------------


def pin_kernel_vs_cas(lib):
    import mpmath as mp
    mp.mp.dps = 40
    F, W, total = cas_kernel()
    assert total == 1, "W is not normalised"
    h = 0.37
    for u in [1e-6, 0.01, 0.1, 0.25, 0.4, 0.4999, 0.5, 0.5001, 0.6, 0.75, 0.9, 0.9999, 1.0, 1.3, 4.0]:
        r = u * h
        fo, go, po = O.kernel(r, h, lib=lib)
        fr, gr, pr = kernel_mp(r, h)
        for name, a, b in (("f", fo, fr), ("g", go, gr), ("phi", po, pr)):
            assert abs(a - float(b)) <= 2e-13 * abs(float(b)) + 1e-300, (name, u, a, float(b))


def pin_kernel_limits(lib):
    h = 0.5
    f0, g0, p0 = O.kernel(0.0, h, lib=lib)
    assert abs(f0 * h**3 - 32.0 / 3.0) < 1e-13
    assert abs(p0 * h - 2.8) < 1e-13
    for u in (0.5, 1.0):
        lo = O.kernel((u - 1e-9) * h, h, lib=lib)
        hi = O.kernel((u + 1e-9) * h, h, lib=lib)
        for a, b in zip(lo, hi):
            assert abs(a - b) <= 1e-7 * abs(b), ("continuity", u, lo, hi)
    for r in (h, 1.5 * h, 10.0 * h):
        f, g, p = O.kernel(r, h, lib=lib)
        assert f == 1.0 / (r * r * r) or abs(f * r**3 - 1) < 1e-15
        assert abs(g * r**5 + 3.0) < 1e-14
        assert abs(p * r - 1.0) < 1e-15


def pin_kernel_identity_g(lib):
    """g = (4 pi W - 3 f) / r^2 (from d M/dr = 4 pi r^2 W m) with W by definition."""
    h = 0.8
    for u in np.linspace(0.02, 1.4, 37):
        r = u * h
        f, g, _ = O.kernel(r, h, lib=lib)
        want = (4 * np.pi * float(W_def(r, h)) - 3.0 * f) / (r * r)
        assert abs(g - want) <= 1e-11 * max(abs(want), 1.0 / h**5), (u, g, want)


# ---------------------------------------------------------------------------
# Pair-sum pins
# ---------------------------------------------------------------------------


def brute_mp(pos, vel, mass, G, h):
    """acc, jerk, tidal, pot by 40-digit mpmath summation with CAS kernels."""
    import mpmath as mp
    mp.mp.dps = 40
    n = len(mass)
    P = [[mp.mpf(float(x)) for x in p] for p in pos]
    V = [[mp.mpf(float(x)) for x in v] for v in vel]
    M = [mp.mpf(float(x)) for x in mass]
    acc = np.zeros((n, 3))
    jerk = np.zeros((n, 3))
    tid = np.zeros((n, 6))
    pot = np.zeros(n)
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for i in range(n):
        a = [mp.mpf(0)] * 3
        jk = [mp.mpf(0)] * 3
        T = [mp.mpf(0)] * 6
        ph = mp.mpf(0)
        for j in range(n):
            if j == i:
                continue
            d = [P[j][c] - P[i][c] for c in range(3)]
            v = [V[j][c] - V[i][c] for c in range(3)]
            r = mp.sqrt(sum(x * x for x in d))
            f, g, p = kernel_mp(r, h)
            dv = sum(d[c] * v[c] for c in range(3))
            for c in range(3):
                a[c] += M[j] * f * d[c]
                jk[c] += M[j] * (f * v[c] + g * dv * d[c])
            for t, (p1, p2) in enumerate(pairs):
                T[t] -= M[j] * ((f if p1 == p2 else 0) + g * d[p1] * d[p2])
            ph -= M[j] * p
        acc[i] = [float(G * x) for x in a]
        jerk[i] = [float(G * x) for x in jk]
        tid[i] = [float(G * x) for x in T]
        pot[i] = float(G * ph)
    return acc, jerk, tid, pot


def _tiny_system(seed, n, spread, coincident=False):
    g = ics.rng(seed)
    pos = g.uniform(-spread, spread, (n, 3))
    if coincident:
        pos[1] = pos[0]
    vel = g.normal(0.0, 1.0, (n, 3))
    mass = g.uniform(0.5, 1.5, n)
    return pos, vel, mass


def _close(a, b, rtol, what):
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.linalg.norm(b, axis=-1, keepdims=True) if b.ndim > 1 else np.abs(b)
    err = np.abs(a - b) / np.maximum(scale, 1e-300)
    assert np.all(err <= rtol), (what, float(err.max()))


def pin_brute_force(lib):
    G = 1.7
    h = 0.45
    for seed, n, coinc in ((11, 6, False), (12, 8, True), (13, 5, False)):
        pos, vel, mass = _tiny_system(seed, n, 0.6, coincident=coinc)
        o = O.eval_active(pos, vel, mass, G=G, h=h, lib=lib)
        acc, jerk, tid, pot = brute_mp(pos, vel, mass, G, h)
        _close(o["acc"], acc, 1e-13, "acc")
        _close(o["jerk"], jerk, 1e-13, "jerk")
        _close(o["tidal"], tid, 1e-13, "tidal")
        _close(o["pot"], pot, 1e-13, "pot")
        # targets given as an index subset are the same rows
        sub = np.array([n - 1, 0, 2], np.int32)
        o2 = O.eval_active(pos, vel, mass, sub, G=G, h=h, lib=lib)
        _close(o2["acc"], acc[sub], 1e-13, "acc subset")


def pin_conditioning(lib):
    """Sums of pair magnitudes (the conditioning of the error metric): against
    a 40-digit brute force over the CAS kernels, with ||T_ij||_F formed from
    the 3x3 matrix entry by entry; on two bodies (one pair) they equal |a|,
    |j| and ||T||_F of the evaluation; and they bound the evaluation's
    magnitudes from above (triangle inequality) on a larger system."""
    import mpmath as mp
    mp.mp.dps = 40
    G, h = 1.3, 0.45
    for seed, n, coinc in ((14, 7, False), (15, 6, True)):
        pos, vel, mass = _tiny_system(seed, n, 0.6, coincident=coinc)
        cond = O.conditioning(pos, vel, mass, G=G, h=h, lib=lib)
        for i in range(n):
            sa = sj = st = mp.mpf(0)
            for j in range(n):
                if j == i:
                    continue
                d = [mp.mpf(float(pos[j, c])) - mp.mpf(float(pos[i, c])) for c in range(3)]
                v = [mp.mpf(float(vel[j, c])) - mp.mpf(float(vel[i, c])) for c in range(3)]
                r = mp.sqrt(sum(x * x for x in d))
                f, g, _ = kernel_mp(r, h)
                m = mp.mpf(float(mass[j]))
                dv = sum(d[c] * v[c] for c in range(3))
                sa += m * abs(f) * r
                sj += m * mp.sqrt(sum((f * v[c] + g * dv * d[c]) ** 2 for c in range(3)))
                st += m * mp.sqrt(sum((f * (a == b) + g * d[a] * d[b]) ** 2
                                      for a in range(3) for b in range(3)))
            ref = [float(G * x) for x in (sa, sj, st)]
            for k in range(3):
                assert abs(cond[i, k] - ref[k]) <= 1e-13 * ref[k], (seed, i, k, cond[i, k], ref[k])
    x = np.array([[0.1, -0.2, 0.3], [0.4, 0.1, 0.2]])
    v = np.array([[0.2, 0.0, -0.1], [-0.3, 0.5, 0.1]])
    mass = np.array([0.7, 1.2])
    for hh in (0.1, 0.9):                       # beyond and inside the support
        o = O.eval_active(x, v, mass, G=G, h=hh, lib=lib)
        cond = O.conditioning(x, v, mass, G=G, h=hh, lib=lib)
        t = o["tidal"]
        tn = np.sqrt((t[:, :3] ** 2).sum(1) + 2 * (t[:, 3:] ** 2).sum(1))
        assert np.allclose(cond[:, 0], np.linalg.norm(o["acc"], axis=1), rtol=1e-14)
        assert np.allclose(cond[:, 1], np.linalg.norm(o["jerk"], axis=1), rtol=1e-14)
        assert np.allclose(cond[:, 2], tn, rtol=1e-14)
    pos, vel, mass = ics.plummer(300, seed=16)
    o = O.eval_active(pos, vel, mass, h=0.05, lib=lib)
    cond = O.conditioning(pos, vel, mass, h=0.05, lib=lib)
    t = o["tidal"]
    tn = np.sqrt((t[:, :3] ** 2).sum(1) + 2 * (t[:, 3:] ** 2).sum(1))
    assert np.all(cond[:, 0] >= np.linalg.norm(o["acc"], axis=1) * (1 - 1e-13))
    assert np.all(cond[:, 1] >= np.linalg.norm(o["jerk"], axis=1) * (1 - 1e-13))
    assert np.all(cond[:, 2] >= tn * (1 - 1e-13))


def pin_two_body(lib):
    """Two point masses beyond the softening: Newton's law and its derivatives."""
    G, h = 2.0, 0.1
    m1, m2 = 0.3, 1.1
    x1 = np.array([0.1, -0.2, 0.3])
    dvec = np.array([0.5, 0.4, -0.2])
    x2 = x1 + dvec
    v1 = np.array([0.0, 0.3, 0.1])
    v2 = np.array([-0.2, 0.1, 0.4])
    r = np.linalg.norm(dvec)
    o = O.eval_active(np.stack([x1, x2]), np.stack([v1, v2]), np.array([m1, m2]), G=G, h=h, lib=lib)
    a1 = G * m2 * dvec / r**3
    assert np.allclose(o["acc"][0], a1, rtol=1e-14, atol=0)
    assert np.allclose(o["acc"][1], -G * m1 * dvec / r**3, rtol=1e-14, atol=0)
    v = v2 - v1
    j1 = G * m2 * (v / r**3 - 3 * np.dot(v, dvec) * dvec / r**5)      # Eq. 4 for a point mass
    assert np.allclose(o["jerk"][0], j1, rtol=1e-13, atol=0)
    Tfull = G * m2 * (3 * np.outer(dvec, dvec) / r**5 - np.eye(3) / r**3)
    t6 = [Tfull[0, 0], Tfull[1, 1], Tfull[2, 2], Tfull[0, 1], Tfull[0, 2], Tfull[1, 2]]
    assert np.allclose(o["tidal"][0], t6, rtol=1e-13, atol=1e-15 * abs(Tfull).max())
    assert abs(o["pot"][0] + G * m2 / r) < 1e-14 * G * m2 / r


def pin_momentum_balance(lib):
    pos, vel, mass = ics.uniform_sphere(400, seed=5)
    mass = mass * ics.rng(6).uniform(0.5, 1.5, mass.size)
    o = O.eval_active(pos, vel, mass, h=0.08, lib=lib)
    for k in ("acc", "jerk"):
        tot = (mass[:, None] * o[k]).sum(axis=0)
        scale = np.abs(mass[:, None] * o[k]).sum()
        assert np.all(np.abs(tot) <= 1e-13 * scale), (k, tot, scale)


def pin_trace_density(lib):
    G, h = 1.3, 0.15
    pos, vel, mass = ics.uniform_sphere(300, seed=7)
    o = O.eval_active(pos, vel, mass, G=G, h=h, lib=lib)
    d = pos[None, :, :] - pos[:, None, :]
    r = np.linalg.norm(d, axis=-1)
    Wm = W_def(r, h) * mass[None, :]
    np.fill_diagonal(Wm, 0.0)
    want = -4 * np.pi * G * Wm.sum(axis=1)
    tr = o["tidal"][:, 0] + o["tidal"][:, 1] + o["tidal"][:, 2]
    scale = np.abs(o["tidal"][:, :3]).sum(axis=1)
    assert np.all(np.abs(tr - want) <= 1e-11 * scale + 1e-12), float(np.abs(tr - want).max())


def pin_cube_symmetry(lib):
    G, m = 1.0, 0.25
    for s, h in ((0.3, 0.2), (0.1, 0.5)):
        verts = np.array([[a, b, c] for a in (-s, s) for b in (-s, s) for c in (-s, s)])
        pos = np.vstack([[0.0, 0.0, 0.0], verts])
        vel = np.zeros_like(pos)
        mass = np.full(9, m)
        o = O.eval_active(pos, vel, mass, np.array([0], np.int32), G=G, h=h, lib=lib)
        r = s * math.sqrt(3.0)
        f, g, _ = kernel_mp(r, h)
        tdiag = -(8 * G * m / 3.0) * (3 * float(f) + r * r * float(g))
        assert np.all(np.abs(o["acc"][0]) <= 1e-15 * G * m / r**2)
        want = np.array([tdiag, tdiag, tdiag, 0, 0, 0])
        scale = max(abs(tdiag), G * m / r**3)
        assert np.all(np.abs(o["tidal"][0] - want) <= 1e-13 * scale), (o["tidal"][0], want)


def pin_scaling(lib):
    pos, vel, mass = ics.plummer(120, seed=9)
    h, lam = 0.2, 3.0
    a = O.eval_active(pos, vel, mass, h=h, lib=lib)
    b = O.eval_active(lam * pos, vel, mass, h=lam * h, lib=lib)
    _close(b["acc"], a["acc"] / lam**2, 1e-13, "acc scaling")
    _close(b["jerk"], a["jerk"] / lam**3, 1e-13, "jerk scaling")
    _close(b["tidal"], a["tidal"] / lam**3, 1e-13, "tidal scaling")
    _close(b["pot"], a["pot"] / lam, 1e-13, "pot scaling")


def pin_jerk_fd(lib):
    """Eq. 4: j = d a / dt along the straight-line drift x + v tau."""
    pos, vel, mass = ics.uniform_sphere(200, seed=21)
    h, tau = 0.12, 1e-6
    o = O.eval_active(pos, vel, mass, h=h, lib=lib)
    p = O.eval_active(pos + tau * vel, vel, mass, h=h, lib=lib)
    m = O.eval_active(pos - tau * vel, vel, mass, h=h, lib=lib)
    fd = (p["acc"] - m["acc"]) / (2 * tau)
    _close(o["jerk"], fd, 2e-6, "jerk vs FD")


def pin_tidal_fd(lib):
    """T = d a_i / d x_i by central differences of the target position."""
    pos, vel, mass = ics.uniform_sphere(150, seed=22)
    h, eps = 0.12, 1e-6
    tgt = np.array([3, 50, 149], np.int32)
    o = O.eval_active(pos, vel, mass, tgt, h=h, lib=lib)
    full = np.zeros((tgt.size, 3, 3))
    for t, i in enumerate(tgt):
        one = np.array([i], np.int32)
        for c in range(3):
            pp = pos.copy()
            pm = pos.copy()
            pp[i, c] += eps
            pm[i, c] -= eps
            ap = O.eval_active(pp, vel, mass, one, h=h, lib=lib)["acc"][0]
            am = O.eval_active(pm, vel, mass, one, h=h, lib=lib)["acc"][0]
            full[t, :, c] = (ap - am) / (2 * eps)
    t6 = np.stack([full[:, 0, 0], full[:, 1, 1], full[:, 2, 2],
                   0.5 * (full[:, 0, 1] + full[:, 1, 0]), 0.5 * (full[:, 0, 2] + full[:, 2, 0]),
                   0.5 * (full[:, 1, 2] + full[:, 2, 1])], axis=1)
    _close(o["tidal"], t6, 1e-6, "tidal vs FD")
    asym = np.abs(full - full.transpose(0, 2, 1)).max() / np.abs(full).max()
    assert asym < 1e-6


def pin_tidal_dt(lib):
    eta = 0.01
    # isotropic tensor -c I: ||T||^2 = 3 c^2
    c = 2.5
    dt = O.tidal_dt([-c, -c, -c, 0, 0, 0], eta, lib=lib)
    assert abs(dt - math.sqrt(eta) * (3 * c * c / 6) ** -0.25) <= 1e-15 * dt
    # point-mass tidal field G m (3 d d^T/r^5 - I/r^3): ||T||^2 = 6 (G m / r^3)^2,
    # so dt = sqrt(eta) * sqrt(r^3 / (G m)), the dynamical time scaled by sqrt(eta)
    G, m = 1.0, 2.0
    d = np.array([0.3, -0.4, 1.2])
    r = np.linalg.norm(d)
    T = G * m * (3 * np.outer(d, d) / r**5 - np.eye(3) / r**3)
    dt = O.tidal_dt([T[0, 0], T[1, 1], T[2, 2], T[0, 1], T[0, 2], T[1, 2]], eta, lib=lib)
    assert abs(dt - math.sqrt(eta) * math.sqrt(r**3 / (G * m))) <= 1e-14 * dt
    assert math.isinf(O.tidal_dt([0, 0, 0, 0, 0, 0], eta, lib=lib))


def _shell_ratio(pos, acc_num, acc_ref, rlo, rhi, nbins):
    r = np.linalg.norm(pos, axis=1)
    out = []
    edges = np.linspace(rlo, rhi, nbins + 1)
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        if sel.sum() < 30:
            continue
        rhat = pos[sel] / r[sel, None]
        ratio = (acc_num[sel] * rhat).sum(1) / (acc_ref[sel] * rhat).sum(1)
        out.append((ratio.mean(), ratio.std(ddof=1) / math.sqrt(sel.sum())))
    return out


def pin_uniform_sphere_field(lib, n=6000):
    """Inside a uniform ball of radius R: a = -G M x / R^3 (shell means)."""
    pos, vel, mass = ics.uniform_sphere(n, seed=31)
    o = O.eval_active(pos, vel, mass, h=0.01, lib=lib)
    ref = -pos / 1.0**3
    for mean, se in _shell_ratio(pos, o["acc"], ref, 0.2, 0.9, 7):
        assert abs(mean - 1.0) < 4 * se + 0.02, (mean, se)


def pin_plummer_field(lib, n=6000):
    """Plummer sphere: a = -G M x / (r^2 + a^2)^(3/2) (shell means)."""
    pos, vel, mass = ics.plummer(n, seed=32)
    o = O.eval_active(pos, vel, mass, h=0.01, lib=lib)
    r2 = (pos * pos).sum(1)
    ref = -pos / (r2 + 1.0)[:, None] ** 1.5
    for mean, se in _shell_ratio(pos, o["acc"], ref, 0.3, 3.0, 6):
        assert abs(mean - 1.0) < 4 * se + 0.02, (mean, se)


def _periodic_system(seed, n, L, margin):
    """Uniform points in [0, L)^3 with no pair separation (per axis) within
    `margin` of L/2, so nearest images do not switch under small moves."""
    g = ics.rng(seed)
    while True:
        pos = g.uniform(0.0, L, (n, 3))
        d = np.abs(pos[None, :, :] - pos[:, None, :])
        d = np.minimum(d, L - d)
        if not np.any(np.abs(d - 0.5 * L) < margin):
            break
    vel = g.normal(0.0, 1.0, (n, 3))
    mass = g.uniform(0.5, 1.5, n)
    return pos, vel, mass


def pin_periodic_translation(lib):
    """Nearest-image sums depend only on positions modulo the box: shifting
    every element and wrapping back into the box changes nothing."""
    L, h = 1.0, 0.08
    pos, vel, mass = _periodic_system(71, 60, L, 1e-3)
    a = O.eval_active(pos, vel, mass, h=h, box=L, lib=lib)
    shift = np.array([0.37, -0.81, 0.123])
    b = O.eval_active(np.mod(pos + shift, L), vel, mass, h=h, box=L, lib=lib)
    for k in ("acc", "jerk", "tidal", "pot"):
        _close(b[k], a[k], 1e-12, "periodic translation " + k)
    mom = (mass[:, None] * a["acc"]).sum(0)
    assert np.all(np.abs(mom) <= 1e-13 * np.abs(mass[:, None] * a["acc"]).sum())


def pin_periodic_two_body(lib):
    """Across the boundary the pair interacts through its nearest image."""
    L, G, h = 2.0, 1.5, 0.05
    x1 = np.array([0.1, 1.0, 1.9])
    x2 = np.array([1.95, 0.8, 0.2])
    d = np.array([-0.15, -0.2, 0.3])             # x2 - x1 reduced to the nearest image
    r = np.linalg.norm(d)
    m2 = 0.7
    o = O.eval_active(np.stack([x1, x2]), np.zeros((2, 3)), np.array([1.3, m2]), G=G, h=h,
                      box=L, lib=lib)
    assert np.allclose(o["acc"][0], G * m2 * d / r**3, rtol=1e-13, atol=0)
    assert abs(o["pot"][0] + G * m2 / r) <= 1e-13 * G * m2 / r


def pin_periodic_half_box_tie(lib):
    """At exactly half a box the two images are equally near; the reading
    taken keeps the separation as it is (d/L = +-1/2 rounds to image 0,
    halves to even), so each element of the pair sees the other through a
    different image, and total momentum is still conserved."""
    L, G, h = 2.0, 1.0, 0.05
    x = np.array([[0.25, 0.5, 0.5], [1.25, 0.7, 0.5]])     # x2 - x1 = (L/2, 0.2, 0)
    m = np.array([0.6, 0.9])
    o = O.eval_active(x, np.zeros((2, 3)), m, G=G, h=h, box=L, lib=lib)
    d = np.array([1.0, 0.2, 0.0])
    r = np.linalg.norm(d)
    assert np.allclose(o["acc"][0], G * m[1] * d / r**3, rtol=1e-14, atol=0)
    assert np.allclose(o["acc"][1], -G * m[0] * d / r**3, rtol=1e-14, atol=0)


def pin_periodic_open_limit(lib):
    """A box much larger than the system changes nothing, bit for bit."""
    pos, vel, mass = ics.uniform_sphere(80, seed=72)
    a = O.eval_active(pos, vel, mass, h=0.1, lib=lib)
    b = O.eval_active(pos, vel, mass, h=0.1, box=100.0, lib=lib)
    for k in ("acc", "jerk", "tidal", "pot"):
        assert np.array_equal(a[k], b[k]), k


def pin_periodic_derivatives(lib):
    """Jerk and tidal tensor are the derivatives of the nearest-image
    acceleration (central differences, no image switches nearby)."""
    L, h, tau = 1.0, 0.1, 1e-6
    pos, vel, mass = _periodic_system(73, 40, L, 2e-3)
    o = O.eval_active(pos, vel, mass, h=h, box=L, lib=lib)
    p = O.eval_active(pos + tau * vel, vel, mass, h=h, box=L, lib=lib)
    m = O.eval_active(pos - tau * vel, vel, mass, h=h, box=L, lib=lib)
    _close(o["jerk"], (p["acc"] - m["acc"]) / (2 * tau), 2e-6, "periodic jerk vs FD")
    i = 5
    one = np.array([i], np.int32)
    full = np.zeros((3, 3))
    for c in range(3):
        pp, pm = pos.copy(), pos.copy()
        pp[i, c] += tau
        pm[i, c] -= tau
        full[:, c] = (O.eval_active(pp, vel, mass, one, h=h, box=L, lib=lib)["acc"][0] -
                      O.eval_active(pm, vel, mass, one, h=h, box=L, lib=lib)["acc"][0]) / (2 * tau)
    t6 = [full[0, 0], full[1, 1], full[2, 2], full[0, 1], full[0, 2], full[1, 2]]
    _close(o["tidal"][i][None], np.array(t6)[None], 1e-6, "periodic tidal vs FD")


# ---------------------------------------------------------------------------
# Selection, binning, compaction, predictor
# ---------------------------------------------------------------------------


# ---------------------------------------------------------------------------
# Adaptive softening (per-element supports and the correction terms)
# ---------------------------------------------------------------------------


@lru_cache(maxsize=1)
def cas_kernel_h():
    """mpmath callables of (r, h) from sympy, for u = r/h < 1/2 and 1/2 <= u < 1:
    W, dW/dr, dW/dh and dpsi/dh, psi(r, h) = p(r/h)/h the potential kernel
    (p from integrating the CAS force kernel, as in cas_kernel)."""
    import sympy as sp
    s, u, r, h = sp.symbols("s u r h", positive=True)
    c = sp.Rational(8) / sp.pi
    w_in = 1 - 6 * s**2 + 6 * s**3
    w_out = 2 * (1 - s) ** 3
    m_in = sp.integrate(4 * sp.pi * s**2 * c * w_in, (s, 0, u))
    m_out = m_in.subs(u, sp.Rational(1, 2)) + sp.integrate(4 * sp.pi * s**2 * c * w_out,
                                                          (s, sp.Rational(1, 2), u))
    f_in, f_out = m_in / u**3, m_out / u**3
    p_out = 1 + sp.integrate(s * f_out.subs(u, s), (s, u, 1))
    p_in = p_out.subs(u, sp.Rational(1, 2)) + sp.integrate(s * f_in.subs(u, s),
                                                           (s, u, sp.Rational(1, 2)))
    out = []
    for w, pk in ((w_in, p_in), (w_out, p_out)):
        W = c / h**3 * w.subs(s, r / h)
        psi = pk.subs(u, r / h) / h
        exprs = (W, sp.diff(W, r), sp.diff(W, h), sp.diff(psi, h))
        out.append([sp.lambdify((r, h), sp.simplify(e), "mpmath") for e in exprs])
    return out


def kernel_h_mp(r, h):
    """(W, dW/dr, dW/dh, dpsi/dh) at (r, h) in mpmath, zero beyond the support."""
    import mpmath as mp
    r = mp.mpf(r)
    h = mp.mpf(h)
    if r >= h:
        return mp.mpf(0), mp.mpf(0), mp.mpf(0), mp.mpf(0)
    fns = cas_kernel_h()[0 if r < h / 2 else 1]
    return tuple(fn(r, h) for fn in fns)


def pin_soft_kernel_vs_cas(lib):
    """W, dW/dr, dW/dh and dpsi/dh against sympy derivatives of W and of the
    integrated potential kernel, at 40 digits."""
    import mpmath as mp
    mp.mp.dps = 40
    for h in (0.37, 2.5):
        for u in (1e-6, 0.1, 0.3, 0.4999, 0.5, 0.5001, 0.7, 0.95, 0.9999, 1.0, 1.7):
            r = u * h
            got = O.kernel_w(r, h, lib=lib)
            ref = [float(x) for x in kernel_h_mp(r, h)]
            scale = [8.0 / (np.pi * h**3), 8.0 / (np.pi * h**4), 8.0 / (np.pi * h**4), 1.0 / h**2]
            for name, a, b, sc in zip(("W", "W_r", "W_h", "psi_h"), got, ref, scale):
                assert abs(a - b) <= 1e-13 * sc, (name, h, u, a, b)


def _soft_system(seed, n):
    g = ics.rng(seed)
    pos = g.normal(0.0, 1.0, (n, 3))
    vel = g.normal(0.0, 1.0, (n, 3))
    mass = g.uniform(0.5, 1.5, n)
    return pos, vel, mass


def pin_soft_constant_h(lib):
    """Equal supports and no correction reduce to the fixed-h sums bit for bit
    (the average of two equal kernels is exact)."""
    pos, vel, mass = ics.plummer(90, seed=41)
    a = O.eval_active(pos, vel, mass, h=0.3, lib=lib)
    b = O.eval_soft(pos, vel, mass, np.full(90, 0.3), lib=lib)
    for k in ("acc", "jerk", "tidal", "pot", "dt_grav"):
        assert np.array_equal(a[k], b[k]), k


def pin_soft_two_body(lib):
    """Two elements with different supports: the pair force uses the mean of
    the two CAS kernels (Newton's third law holds with both masses)."""
    import mpmath as mp
    mp.mp.dps = 40
    G, m1, m2 = 1.3, 0.8, 0.7
    x = np.array([[0.1, 0.2, -0.1], [0.25, 0.05, 0.1]])
    h = np.array([0.5, 0.3])
    o = O.eval_soft(x, np.zeros((2, 3)), np.array([m1, m2]), h, lib=lib, G=G)
    d = x[1] - x[0]
    r = float(np.linalg.norm(d))
    k1, k2 = kernel_mp(r, h[0]), kernel_mp(r, h[1])
    f = float((k1[0] + k2[0]) / 2)
    g = float((k1[1] + k2[1]) / 2)
    p = float((k1[2] + k2[2]) / 2)
    _close(o["acc"][0], G * m2 * f * d, 1e-14, "soft two-body a1")
    _close(o["acc"][1], -G * m1 * f * d, 1e-14, "soft two-body a2")
    assert abs(o["pot"][0] + G * m2 * p) <= 1e-14 * G * m2 * p
    T = -G * m2 * (f * np.eye(3) + g * np.outer(d, d))
    t6 = np.array([T[0, 0], T[1, 1], T[2, 2], T[0, 1], T[0, 2], T[1, 2]])
    assert np.allclose(o["tidal"][0], t6, rtol=1e-13, atol=1e-13 * np.abs(t6).max())


def pin_soft_solve(lib):
    """The supports solve (4 pi/3) h^3 rho = n_ngb m with rho summed by brute
    force over the CAS kernel (self term included); Omega and zeta equal their
    definitions summed the same way."""
    import mpmath as mp
    mp.mp.dps = 30
    pos, vel, mass = _soft_system(51, 60)
    n_ngb = 20.0
    sol = O.soft_solve(pos, mass, 0.4, n_ngb=n_ngb, tol=1e-14, max_iter=200, lib=lib)
    assert sol["converged"]
    for i in (0, 7, 33, 59):
        h = sol["h"][i]
        rho = rho_h = psi_h = mp.mpf(0)
        for j in range(60):
            r = mp.sqrt(sum((mp.mpf(pos[j, c]) - mp.mpf(pos[i, c])) ** 2 for c in range(3)))
            w, _, wh, ph = kernel_h_mp(r, h)
            rho += mass[j] * w
            rho_h += mass[j] * wh
            if j != i:
                psi_h += mass[j] * ph
        F = 4 * mp.pi / 3 * mp.mpf(h) ** 3 * rho - n_ngb * mass[i]
        assert abs(float(F)) <= 1e-12 * n_ngb * mass[i], (i, float(F))
        omega = 1 + h * rho_h / (3 * rho)
        zeta = -h * psi_h / (3 * rho * omega)
        assert abs(sol["omega"][i] - float(omega)) <= 1e-11 * abs(float(omega)), i
        assert abs(sol["zeta"][i] - float(zeta)) <= 1e-11 * abs(float(zeta)), i


def pin_soft_sums(lib):
    """The per-element sums at given (unsolved) supports: rho = sum_j m_j W
    and rho_h = sum_j m_j dW/dh with the self term, psi_h = sum_{j != i} m_j
    dpsi/dh, against a 30-digit brute force over the CAS kernels; rho_h
    against a central difference of rho in h; and an isolated element, whose
    sums are its self term alone: rho = m 8/(pi h^3), rho_h = -3 rho / h,
    psi_h = 0."""
    import mpmath as mp
    mp.mp.dps = 30
    pos, vel, mass = _soft_system(53, 50)
    pos[49] = [40.0, -40.0, 40.0]                    # far from every other element
    h = ics.rng(54).uniform(0.3, 0.9, 50)
    rho, rho_h, psi_h = O.soft_sums(pos, mass, h, lib=lib)
    for i in (0, 11, 25, 48):
        r_ = rh_ = ph_ = mp.mpf(0)
        for j in range(50):
            r = mp.sqrt(sum((mp.mpf(pos[j, c]) - mp.mpf(pos[i, c])) ** 2 for c in range(3)))
            w, _, wh, ph = kernel_h_mp(r, h[i])
            r_ += mass[j] * w
            rh_ += mass[j] * wh
            if j != i:
                ph_ += mass[j] * ph
        assert abs(rho[i] - float(r_)) <= 1e-13 * float(r_), ("rho", i)
        assert abs(rho_h[i] - float(rh_)) <= 1e-12 * abs(float(rh_)), ("rho_h", i)
        assert abs(psi_h[i] - float(ph_)) <= 1e-12 * abs(float(ph_)), ("psi_h", i)
    eps = 1e-6
    up = O.soft_sums(pos, mass, h * (1 + eps), lib=lib)[0]
    dn = O.soft_sums(pos, mass, h * (1 - eps), lib=lib)[0]
    fd = (up - dn) / (2 * eps * h)
    sel = np.arange(49)
    assert np.allclose(rho_h[sel], fd[sel], rtol=1e-6, atol=1e-8 * np.abs(rho_h).max()), "rho_h vs FD"
    w0 = 8.0 / (np.pi * h[49] ** 3)
    assert abs(rho[49] - mass[49] * w0) <= 1e-15 * mass[49] * w0
    assert abs(rho_h[49] + 3.0 * mass[49] * w0 / h[49]) <= 1e-14 * 3.0 * mass[49] * w0 / h[49]
    assert psi_h[49] == 0.0


def pin_soft_energy_gradient(lib):
    """With the correction the acceleration is -grad_i U / m_i, U the potential
    energy with every support re-solved from the constraint (central
    differences); without it the difference is at the per-cent level."""
    pos, vel, mass = _soft_system(52, 40)
    n_ngb, tau = 20.0, 1e-6

    def energy(p):
        s = O.soft_solve(p, mass, 1.0, n_ngb=n_ngb, tol=1e-15, max_iter=300, lib=lib)
        assert s["converged"]
        return 0.5 * float((mass * O.eval_soft(p, vel, mass, s["h"], lib=lib)["pot"]).sum())

    sol = O.soft_solve(pos, mass, 1.0, n_ngb=n_ngb, tol=1e-15, max_iter=300, lib=lib)
    full = O.eval_soft(pos, vel, mass, sol["h"], sol["zeta"], lib=lib)["acc"]
    plain = O.eval_soft(pos, vel, mass, sol["h"], lib=lib)["acc"]
    worst_plain = 0.0
    for i in (0, 11, 25, 39):
        fd = np.zeros(3)
        for c in range(3):
            pp = pos.copy()
            pm = pos.copy()
            pp[i, c] += tau
            pm[i, c] -= tau
            fd[c] = -(energy(pp) - energy(pm)) / (2 * tau) / mass[i]
        _close(full[i], fd, 1e-6, "adaptive-softening force vs -grad U")
        worst_plain = max(worst_plain, np.linalg.norm(plain[i] - fd) / np.linalg.norm(fd))
    assert worst_plain > 1e-3, worst_plain


def pin_soft_momentum(lib):
    """The averaged pair force and the correction are antisymmetric in the pair:
    sum m a = 0 and sum m j = 0."""
    pos, vel, mass = ics.plummer(300, seed=53)
    sol = O.soft_solve(pos, mass, 0.1, n_ngb=32.0, lib=lib)
    o = O.eval_soft(pos, vel, mass, sol["h"], sol["zeta"], lib=lib)
    for k in ("acc", "jerk"):
        mom = (mass[:, None] * o[k]).sum(0)
        assert np.all(np.abs(mom) <= 1e-13 * np.abs(mass[:, None] * o[k]).sum()), k


def pin_soft_derivatives(lib):
    """At fixed supports, jerk = d a / dt along the drift and T = d a_i / d x_i
    (central differences; the correction term is not differentiated)."""
    pos, vel, mass = ics.plummer(120, seed=54)
    sol = O.soft_solve(pos, mass, 0.1, n_ngb=24.0, lib=lib)
    h, tau = sol["h"], 1e-6
    o = O.eval_soft(pos, vel, mass, h, lib=lib)
    p = O.eval_soft(pos + tau * vel, vel, mass, h, lib=lib)
    m = O.eval_soft(pos - tau * vel, vel, mass, h, lib=lib)
    _close(o["jerk"], (p["acc"] - m["acc"]) / (2 * tau), 2e-6, "soft jerk vs FD")
    i = 17
    one = np.array([i], np.int32)
    full = np.zeros((3, 3))
    for c in range(3):
        pp = pos.copy()
        pm = pos.copy()
        pp[i, c] += tau
        pm[i, c] -= tau
        full[:, c] = (O.eval_soft(pp, vel, mass, h, idx=one, lib=lib)["acc"][0]
                      - O.eval_soft(pm, vel, mass, h, idx=one, lib=lib)["acc"][0]) / (2 * tau)
    t6 = np.array([full[0, 0], full[1, 1], full[2, 2], full[0, 1], full[0, 2], full[1, 2]])
    assert np.allclose(o["tidal"][i], t6, rtol=0, atol=2e-6 * np.abs(t6).max())


# ---------------------------------------------------------------------------
# Approximate solver: oct-tree with the geometric opening criterion
# ---------------------------------------------------------------------------


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def pin_tree_theta_zero(lib):
    """Theta = 0 opens every node down to its leaves: the direct sum."""
    pos, vel, mass = ics.plummer(700, seed=61)
    d = O.eval_active(pos, vel, mass, h=0.01, lib=lib)
    t = O.tree_eval(pos, vel, mass, h=0.01, theta=0.0, leaf_size=5, lib=lib)
    assert t["interactions"] == 700 * 699
    for k in ("acc", "jerk", "tidal"):
        assert np.all(_rel(t[k], d[k]) <= 1e-13), k
    assert np.all(np.abs(t["pot"] - d["pot"]) <= 1e-13 * np.abs(d["pot"]))


def pin_tree_order(lib):
    """Tree order = elements sorted by (63-bit Morton key, index), keys from
    the bounding cube quantised to 2^21 cells per axis (written out here)."""
    pos, vel, mass = ics.uniform_sphere(500, seed=62, sort=False)
    lo = pos.min(axis=0)
    ext = float((pos.max(axis=0) - lo).max())
    q = np.clip(np.floor((pos - lo) / ext * 2.0**21), 0, 2**21 - 1).astype(np.int64)
    keys = []
    for i in range(500):
        k = 0
        for b in range(20, -1, -1):
            k = (k << 3) | (((q[i, 0] >> b) & 1) << 2) | (((q[i, 1] >> b) & 1) << 1) | ((q[i, 2] >> b) & 1)
        keys.append((k, i))
    want = [i for _, i in sorted(keys)]
    got = O.tree_eval(pos, vel, mass, h=0.01, lib=lib)["order"]
    assert list(got) == want


def pin_tree_error_bounds(lib):
    """Monopole Barnes-Hut errors: small at Theta = 0.5 and shrinking with Theta."""
    pos, vel, mass = ics.plummer(4000, seed=63)
    d = O.eval_active(pos, vel, mass, h=0.01, lib=lib)
    med = []
    for th in (0.3, 0.5, 0.7):
        t = O.tree_eval(pos, vel, mass, h=0.01, theta=th, lib=lib)
        e = _rel(t["acc"], d["acc"])
        med.append(np.median(e))
        if th == 0.5:
            assert np.median(e) < 5e-3 and np.percentile(e, 99) < 3e-2, (np.median(e), e.max())
            assert t["interactions"] < 0.3 * 4000 * 3999
    assert med[0] < med[1] < med[2], med


def pin_tree_far_cluster(lib):
    """A compact cluster B far from cluster A: every element of A sees B as
    one point mass at B's centre of mass moving with B's mean velocity, and
    the rest of A element by element."""
    g = ics.rng(64)
    na = 6                       # cluster A fits in one leaf (leaf_size 8)
    a = g.uniform(-0.05, 0.05, (na, 3))
    b = g.uniform(1.95, 3.6, (30, 3))   # fills the far octant: splits below its top node
    pos = np.vstack([a, b])
    vel = g.normal(0.0, 1.0, (na + 30, 3))
    mass = g.uniform(0.5, 1.5, na + 30)
    G, h = 1.3, 0.02
    t = O.tree_eval(pos, vel, mass, G=G, h=h, theta=0.5, leaf_size=8, lib=lib)
    MB = mass[na:].sum()
    cB = (mass[na:, None] * pos[na:]).sum(0) / MB
    vB = (mass[na:, None] * vel[na:]).sum(0) / MB
    inner = O.eval_active(pos[:na], vel[:na], mass[:na], G=G, h=h, lib=lib)
    assert t["interactions"] < (na + 30) * (na + 29)
    for i in range(na):
        dd = cB - pos[i]
        vv = vB - vel[i]
        r = np.linalg.norm(dd)
        acc = inner["acc"][i] + G * MB * dd / r**3
        jk = inner["jerk"][i] + G * MB * (vv / r**3 - 3 * np.dot(dd, vv) * dd / r**5)
        assert np.allclose(t["acc"][i], acc, rtol=1e-12, atol=0), i
        assert np.allclose(t["jerk"][i], jk, rtol=1e-11, atol=1e-11 * np.abs(jk).max()), i
    # relative criterion: B's top node (side ext/2) is accepted iff
    # G M_B L^2 <= alpha |a_old| r^4; put |a_old| just above / below that
    # (below, B is resolved into its children and the single monopole no
    # longer holds)
    ext = float((pos.max(axis=0) - pos.min(axis=0)).max())
    L = ext / 2
    alpha = 0.01
    r = np.linalg.norm(cB - pos[:na], axis=1)
    thr = G * MB * L**2 / r**4 / alpha
    for scale, monopole in ((1.5, True), (0.5, False)):
        a_old = np.zeros((na + 30, 3))
        a_old[:na, 0] = scale * thr
        tr = O.tree_eval(pos, vel, mass, G=G, h=h, theta=0.5, leaf_size=8, alpha=alpha,
                         a_old=a_old, lib=lib)
        for i in range(na):
            dd = cB - pos[i]
            acc = inner["acc"][i] + G * MB * dd / np.linalg.norm(dd) ** 3
            same = np.allclose(tr["acc"][i], acc, rtol=1e-12, atol=0)
            assert same == monopole, (scale, i)


def pin_tree_derivatives(lib):
    """Jerk = d a/dt along the drift and T = d a_i/d x_i of the tree field
    (central differences; the tree's shape does not change at this scale)."""
    pos, vel, mass = ics.plummer(300, seed=65)
    h, tau = 0.01, 1e-7
    o = O.tree_eval(pos, vel, mass, h=h, theta=0.5, lib=lib)
    p = O.tree_eval(pos + tau * vel, vel, mass, h=h, theta=0.5, lib=lib)
    m = O.tree_eval(pos - tau * vel, vel, mass, h=h, theta=0.5, lib=lib)
    _close(o["jerk"], (p["acc"] - m["acc"]) / (2 * tau), 1e-5, "tree jerk vs FD")
    i = 40
    one = np.array([i], np.int32)
    full = np.zeros((3, 3))
    for c in range(3):
        pp = pos.copy()
        pm = pos.copy()
        pp[i, c] += tau
        pm[i, c] -= tau
        full[:, c] = (O.tree_eval(pp, vel, mass, one, h=h, theta=0.5, lib=lib)["acc"][0]
                      - O.tree_eval(pm, vel, mass, one, h=h, theta=0.5, lib=lib)["acc"][0]) / (2 * tau)
    t6 = np.array([full[0, 0], full[1, 1], full[2, 2], full[0, 1], full[0, 2], full[1, 2]])
    assert np.allclose(o["tidal"][i], t6, rtol=0, atol=1e-5 * np.abs(t6).max())


def pin_tree_relative_criterion(lib):
    """The relative criterion only ever opens more nodes: a vanishing alpha
    gives the direct sum, a finite one at least the geometric-only work."""
    pos, vel, mass = ics.plummer(600, seed=66)
    d = O.eval_active(pos, vel, mass, h=0.01, lib=lib)
    geo = O.tree_eval(pos, vel, mass, h=0.01, theta=0.5, lib=lib)
    rel = O.tree_eval(pos, vel, mass, h=0.01, theta=0.5, alpha=0.0025, a_old=d["acc"], lib=lib)
    tiny = O.tree_eval(pos, vel, mass, h=0.01, theta=0.5, alpha=1e-300, a_old=d["acc"], lib=lib)
    assert rel["interactions"] >= geo["interactions"]
    assert np.median(_rel(rel["acc"], d["acc"])) <= np.median(_rel(geo["acc"], d["acc"]))
    assert tiny["interactions"] == 600 * 599
    assert np.all(_rel(tiny["acc"], d["acc"]) <= 1e-13)


def pin_update_counts(lib):
    """With fixed bins and dt_grav, an element of step s ticks is updated every
    ceil(q_f dt_grav / (s dt_min)) of its active steps (Eq. updatecondition),
    and its counter always equals the time since its last update (Eq. 3)."""
    k_max = 5
    dt_min = 2.0**-10
    g = ics.rng(41)
    n = 64
    bins = g.integers(0, k_max + 1, n).astype(np.int8)
    dtg = g.uniform(0.5, 40.0, n) * dt_min
    # exact multiples of dt_min: T_f dt_min == q_f dt_grav happens, and the
    # update condition counts equality as due (the paper's ">=")
    dtg[: n // 2] = g.integers(1, 80, n // 2) * dt_min
    for q_f in (0.0, 0.25, 0.5, 1.0, 2.0):
        tf = np.zeros(n, np.int64)
        dtg0 = np.zeros(n)               # never evaluated: due at tick 0
        last = np.zeros(n, np.int64)
        counts = np.zeros(n, np.int64)
        horizon = 4 * 2**k_max
        for tick in range(horizon):
            active, due, tf = O.select_due(tick, k_max, bins, tf, dtg if tick else dtg0, q_f,
                                           dt_min, lib=lib)
            steps = 2 ** (k_max - bins.astype(np.int64))
            assert np.array_equal(active.astype(bool), tick % steps == 0)
            assert not np.any(due & ~active)
            # the counter holds the time since the last update for active, not-due ones
            ad = (active == 1) & (due == 0)
            assert np.array_equal(tf[ad], tick - last[ad])
            assert np.all(tf[due == 1] == 0)
            last[due == 1] = tick
            counts += (due == 1) & (tick > 0)
        steps = 2 ** (k_max - bins.astype(np.int64))
        every = np.maximum(1, np.ceil(q_f * dtg / (steps * dt_min))).astype(np.int64)
        n_active = (horizon - 1) // steps       # active ticks after tick 0
        assert np.array_equal(counts, n_active // every), q_f


def pin_reverts_exactly(lib):
    """q_f <= 1/2 with the step equal to the binned dt_grav: every active
    element is due (the paper's exact reversion, with power-of-two bins)."""
    k_max = 6
    dt_max = 1.0 / 16.0
    dt_min = dt_max * 2.0**-k_max
    g = ics.rng(42)
    n = 200
    dtg = dt_max * 2.0 ** g.uniform(-k_max, 0.5, n)
    bins = np.full(n, k_max, np.int8)
    tf = np.zeros(n, np.int64)
    for tick in range(0, 3 * 2**k_max):
        active, due, tf = O.select_due(tick, k_max, bins, tf, dtg if tick else np.zeros(n),
                                       0.5, dt_min, lib=lib)
        assert np.array_equal(active, due), tick
        bins = O.assign_bins(tick, k_max, dt_max, active, dtg, None, bins, lib=lib)


def _bin_bruteforce(dt, dt_max, k_max, tick):
    if not (dt > 0):
        k = k_max
    elif math.isinf(dt):
        k = 0
    else:
        k = k_max
        for kk in range(0, k_max + 1):
            if Fraction(dt_max) / 2**kk <= Fraction(dt):
                k = kk
                break
    for kk in range(k, k_max + 1):
        if tick % (2 ** (k_max - kk)) == 0:
            return kk
    return k_max


def pin_bins(lib):
    k_max = 7
    dt_max = 0.3
    g = ics.rng(43)
    n = 300
    dtg = dt_max * 2.0 ** g.uniform(-9, 1.5, n)
    dtg[:8] = dt_max * 2.0 ** -np.arange(8)            # exactly on bin edges
    dtg[8:16] = np.nextafter(dtg[:8], 0)                # just below the edges
    dtg[16] = np.inf
    dtg[17] = 0.0
    dth = np.where(g.uniform(size=n) < 0.3, dt_max * 2.0 ** g.uniform(-9, 0, n), np.inf)
    for tick in (0, 1, 2, 4, 12, 64, 96, 128, 77):
        active = (g.uniform(size=n) < 0.7).astype(np.uint8)
        old = g.integers(0, k_max + 1, n).astype(np.int8)
        out = O.assign_bins(tick, k_max, dt_max, active, dtg, dth, old, lib=lib)
        for i in range(n):
            if not active[i]:
                assert out[i] == old[i]
            else:
                want = _bin_bruteforce(min(dtg[i], dth[i]), dt_max, k_max, tick)
                assert out[i] == want, (tick, i, dtg[i], dth[i], out[i], want)


def pin_compact(lib):
    g = ics.rng(44)
    for n, p in ((0, 0.5), (1, 1.0), (17, 0.3), (1000, 0.01), (4097, 0.9)):
        flags = (g.uniform(size=n) < p).astype(np.uint8)
        flags[flags == 1] = g.integers(1, 256, int(flags.sum()))   # any non-zero byte
        assert np.array_equal(O.compact(flags, lib=lib), np.flatnonzero(flags).astype(np.int32))


def pin_predictor(lib):
    """Exact on a field linear in time; equal to the incremental Eq. (jerkupdate)."""
    dt_min = 2.0**-10
    g = ics.rng(45)
    n = 50
    a0 = g.normal(size=(n, 3))
    j0 = g.normal(size=(n, 3))
    t_last = g.integers(0, 100, n)
    tf = g.integers(0, 64, n).astype(np.int64)
    a_last = a0 + j0 * (t_last * dt_min)[:, None]
    active = np.ones(n, np.uint8)
    due = (g.uniform(size=n) < 0.3).astype(np.uint8)
    out = O.predict(active, due, a_last, j0, tf, dt_min, np.full((n, 3), np.nan), lib=lib)
    exact = a0 + j0 * ((t_last + tf) * dt_min)[:, None]
    nd = due == 0
    assert np.allclose(out[nd], exact[nd], rtol=1e-14, atol=1e-14)
    assert np.array_equal(out[due == 1], a_last[due == 1])
    # incremental g += j dt applied over unit steps equals the closed form
    inc = a_last.copy()
    for i in range(n):
        x = a_last[i].copy()
        for _ in range(int(tf[i])):
            x = x + j0[i] * dt_min
        inc[i] = x
    assert np.allclose(out[nd], inc[nd], rtol=1e-13, atol=1e-13)
    # inactive elements are left untouched
    keep = np.full((n, 3), 7.0)
    out2 = O.predict(np.zeros(n, np.uint8), due, a_last, j0, tf, dt_min, keep, lib=lib)
    assert np.array_equal(out2, keep)


def pin_poly_history(lib):
    """The logged history equals a brute-force record of evaluation ticks:
    with the selection's elapsed ticks, dt_prev is the gap between each
    element's last two evaluations and a_prev the earlier of them."""
    g = ics.rng(46)
    n, dt_min, k_max = 40, 2.0**-10, 3
    bins = g.integers(0, k_max + 1, n).astype(np.int8)
    dtg = np.zeros(n)
    tf = np.zeros(n, np.int64)
    elapsed = np.zeros(n, np.int64)
    a_prev = np.zeros((n, 3))
    dt_prev = np.zeros(n)
    evals = [[] for _ in range(n)]                 # (tick, acceleration) per element
    a_last = np.zeros((n, 3))
    for tick in range(0, 80):
        q_f = 0.0 if tick == 0 else 1.0
        active, due, tf, elapsed = O.select_due(tick, k_max, bins, tf, dtg, q_f, dt_min, lib=lib,
                                                elapsed=elapsed)
        a_prev, dt_prev = O.push_history(due, elapsed, dtg, a_last, a_prev, dt_prev, dt_min, lib=lib)
        new = g.normal(size=(n, 3))
        a_last = np.where(due[:, None] == 1, new, a_last)
        dtg = np.where(due == 1, g.uniform(0.5, 12.0, n) * dt_min, dtg)   # "evaluated"
        for i in np.flatnonzero(due):
            evals[i].append((tick, new[i].copy()))
        for i in np.flatnonzero(due):
            if len(evals[i]) >= 2:
                (t0, a0), (t1, _) = evals[i][-2], evals[i][-1]
                assert t1 == tick and dt_prev[i] == (t1 - t0) * dt_min, (i, tick)
                assert np.array_equal(a_prev[i], a0)
            else:
                assert dt_prev[i] == 0.0


def pin_poly_predictor(lib):
    """Linear extrapolation through the last two evaluations: exact on a
    field linear in time; error c tau (tau + Delta) on a(t) = c t^2; the
    constant a_last with no history; due elements get a_last."""
    g = ics.rng(47)
    n, dt_min = 64, 2.0**-10
    gap = g.integers(1, 40, n)                         # Delta in ticks
    t1 = g.integers(40, 200, n)
    t0 = t1 - gap
    tau = g.integers(0, 50, n).astype(np.int64)        # T_f
    a0, j = g.normal(size=(n, 3)), g.normal(size=(n, 3))
    lin = lambda t: a0 + j * (t * dt_min)[:, None]
    active = np.ones(n, np.uint8)
    due = np.zeros(n, np.uint8)
    out = O.predict_poly(active, due, lin(t1), lin(t0), gap * dt_min, tau, dt_min,
                         np.zeros((n, 3)), lib=lib)
    assert np.allclose(out, lin(t1 + tau), rtol=1e-12, atol=1e-12)
    c = g.normal(size=(n, 3))
    quad = lambda t: c * ((t * dt_min) ** 2)[:, None]
    out = O.predict_poly(active, due, quad(t1), quad(t0), gap * dt_min, tau, dt_min,
                         np.zeros((n, 3)), lib=lib)
    want_err = c * ((tau * dt_min) * ((tau + gap) * dt_min))[:, None]
    assert np.allclose(quad(t1 + tau) - out, want_err, rtol=1e-9, atol=1e-15)
    out = O.predict_poly(active, due, lin(t1), lin(t0), np.zeros(n), tau, dt_min,
                         np.zeros((n, 3)), lib=lib)
    assert np.array_equal(out, lin(t1))
    due[::3] = 1
    out = O.predict_poly(active, due, lin(t1), lin(t0), gap * dt_min, tau, dt_min,
                         np.zeros((n, 3)), lib=lib)
    assert np.array_equal(out[::3], lin(t1)[::3])
    keep = np.full((n, 3), 5.0)
    out = O.predict_poly(np.zeros(n, np.uint8), due, lin(t1), lin(t0), gap * dt_min, tau, dt_min,
                         keep, lib=lib)
    assert np.array_equal(out, keep)


# ---------------------------------------------------------------------------
# Adjoint
# ---------------------------------------------------------------------------


def _loss(pos, vel, mass, w, h, lib):
    o = O.eval_active(pos, vel, mass, h=h, lib=lib)
    return float((w * (o["acc"] ** 2).sum(1)).sum()) + O.potential_energy(mass, o["pot"])


def pin_adjoint_fd(lib):
    """Gradients of L = sum w |a|^2 + W against central differences."""
    pos, vel, mass = ics.plummer(48, seed=51)
    h = 0.3
    w = ics.rng(52).uniform(0, 1, mass.size)
    o = O.eval_active(pos, vel, mass, h=h, lib=lib)
    a_bar = 2 * w[:, None] * o["acc"]
    pb, mb = O.backward(pos, mass, a_bar, 1.0, o["acc"], o["tidal"], o["pot"], h=h, lib=lib)
    eps = 1e-6
    g = ics.rng(53)
    for k, c in zip(g.integers(0, mass.size, 8), g.integers(0, 3, 8)):
        pp = pos.copy()
        pm = pos.copy()
        pp[k, c] += eps
        pm[k, c] -= eps
        fd = (_loss(pp, vel, mass, w, h, lib) - _loss(pm, vel, mass, w, h, lib)) / (2 * eps)
        assert abs(fd - pb[k, c]) <= 1e-6 * max(1.0, abs(fd)), ("pos", k, c, fd, pb[k, c])
    for k in g.integers(0, mass.size, 6):
        mp_ = mass.copy()
        mm_ = mass.copy()
        de = eps * mass[k]
        mp_[k] += de
        mm_[k] -= de
        fd = (_loss(pos, vel, mp_, w, h, lib) - _loss(pos, vel, mm_, w, h, lib)) / (2 * de)
        assert abs(fd - mb[k]) <= 1e-6 * max(1.0, abs(fd)), ("mass", k, fd, mb[k])


ALL_PINS = [
    pin_kernel_vs_cas, pin_kernel_limits, pin_kernel_identity_g, pin_brute_force, pin_conditioning,
    pin_two_body,
    pin_momentum_balance, pin_trace_density, pin_cube_symmetry, pin_scaling, pin_jerk_fd,
    pin_tidal_fd, pin_tidal_dt, pin_periodic_translation, pin_periodic_two_body,
    pin_periodic_half_box_tie, pin_periodic_open_limit, pin_periodic_derivatives,
    pin_soft_kernel_vs_cas, pin_soft_constant_h, pin_soft_two_body, pin_soft_solve, pin_soft_sums,
    pin_soft_energy_gradient, pin_soft_momentum, pin_soft_derivatives,
    pin_tree_theta_zero, pin_tree_order, pin_tree_error_bounds, pin_tree_far_cluster,
    pin_tree_derivatives, pin_tree_relative_criterion,
    pin_update_counts, pin_reverts_exactly, pin_bins, pin_compact,
    pin_predictor, pin_poly_history, pin_poly_predictor, pin_adjoint_fd,
]
