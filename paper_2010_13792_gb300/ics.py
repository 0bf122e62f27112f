"""Seeded synthetic initial conditions shaped like the paper's test problems.

This module only draws inputs: positions, velocities, masses, active subsets
and batched system layouts.  It holds none of the gravity method's arithmetic,
and it is the one module both the oracle-based tests and the CUDA path take
their inputs from.  All generators use NumPy's ``Generator(PCG64(seed))`` and
return FP64 arrays with G = M = 1 and equal masses m = M/N.

Stand-ins (the paper's own initial conditions are not published):
  * ``uniform_sphere``  -- uniform ball of radius R, isotropic Gaussian
    velocities with K/|W| = 0.5, |W| = 3 G M^2 / (5 R).
  * ``plummer``         -- Plummer sphere (scale radius a), radii truncated at
    20 a, velocities from the Plummer distribution function by the
    Aarseth-Henon-Wielen (1974) rejection sampling of q^2 (1-q^2)^(7/2).
  * ``turbulent_cloud`` -- uniform ball with a Gaussian random velocity field,
    3-D power spectrum P(k) ~ k^-4 per component on a periodic FFT grid over
    [-R, R]^3 (no Helmholtz projection), trilinearly interpolated, mean removed
    and scaled to virial parameter alpha = 2K/|W| = 2.  Stands in for the
    STARFORGE giant-molecular-cloud runs of Section 3.
  * ``zeldovich_box``   -- periodic cube [0, L)^3: a lattice displaced by one
    sinusoidal mode along x (the shape of the Zeldovich pancake of Section 3,
    without the cosmology), velocities along the displacement.
  * ``soft_inputs``     -- seeded per-element supports and correction
    coefficients for adaptive-softening parity runs at large N.
  * ``morton_order``    -- stable sort by 63-bit Morton key so that consecutive
    index ranges are spatially compact (applied once at creation time).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2010_13792


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _iso_dirs(g: np.random.Generator, n: int) -> np.ndarray:
    cz = g.uniform(-1.0, 1.0, n)
    ph = g.uniform(0.0, 2.0 * np.pi, n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)


def _morton_spread(v: np.ndarray) -> np.ndarray:
    """Spread the low 21 bits of v so that bit b lands at bit 3b."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(pos: np.ndarray) -> np.ndarray:
    """Stable permutation sorting points by 63-bit Morton key over their bbox."""
    pos = np.asarray(pos, np.float64)
    if pos.shape[0] == 0:
        return np.zeros(0, np.int64)
    lo = pos.min(axis=0)
    ext = float((pos.max(axis=0) - lo).max())
    if ext == 0.0:
        return np.arange(pos.shape[0])
    q = np.floor((pos - lo) / ext * (2**21 - 1)).astype(np.int64)
    q = np.clip(q, 0, 2**21 - 1)
    key = (_morton_spread(q[:, 0]) << np.uint64(2)) | (_morton_spread(q[:, 1]) << np.uint64(1)) \
        | _morton_spread(q[:, 2])
    return np.argsort(key, kind="stable")


def _finish(pos, vel, sort: bool):
    n = pos.shape[0]
    mass = np.full(n, 1.0 / n) if n else np.zeros(0)
    if sort and n:
        p = morton_order(pos)
        pos, vel = pos[p], vel[p]
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass


def uniform_sphere(n: int, seed: int = BASE_SEED + 0, R: float = 1.0,
                   virial_ratio: float = 0.5, sort: bool = True):
    """Uniform ball, isotropic Gaussian velocities with K/|W| = virial_ratio."""
    g = rng(seed)
    r = R * g.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    pos = r[:, None] * _iso_dirs(g, n)
    w_abs = 3.0 / (5.0 * R)                   # |W| = 3 G M^2 / (5 R), G = M = 1
    sigma = np.sqrt(2.0 * virial_ratio * w_abs / 3.0)   # K = 3/2 M sigma^2
    vel = g.normal(0.0, sigma, (n, 3))
    return _finish(pos, vel, sort)


def plummer(n: int, seed: int = BASE_SEED + 1, a: float = 1.0, r_max: float = 20.0,
            sort: bool = True):
    """Plummer sphere (G = M = 1), radii <= r_max * a, isotropic DF velocities."""
    g = rng(seed)
    r = np.empty(0)
    while r.size < n:
        u = g.uniform(0.0, 1.0, 2 * (n - r.size) + 16)
        u = u[u > 0.0]
        rr = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        r = np.concatenate([r, rr[rr <= r_max * a]])
    r = r[:n]
    pos = r[:, None] * _iso_dirs(g, n)
    q = np.empty(0)
    while q.size < n:
        x = g.uniform(0.0, 1.0, 2 * (n - q.size) + 16)
        y = g.uniform(0.0, 0.1, x.size)
        ok = y < x * x * (1.0 - x * x) ** 3.5
        q = np.concatenate([q, x[ok]])
    q = q[:n]
    v = q * np.sqrt(2.0) * (1.0 + (r / a) ** 2) ** (-0.25) / np.sqrt(a)
    vel = v[:, None] * _iso_dirs(g, n)
    return _finish(pos, vel, sort)


def _grf_component(g: np.random.Generator, ng: int, index: float) -> np.ndarray:
    """Real Gaussian random field on ng^3 with |f(k)|^2 ~ k^index (k != 0)."""
    kx = np.fft.fftfreq(ng) * ng
    kz = np.fft.rfftfreq(ng) * ng
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (index / 4.0)        # sqrt(P) with P ~ k^index
    noise = g.normal(size=k2.shape) + 1j * g.normal(size=k2.shape)
    return np.fft.irfftn(noise * amp, s=(ng, ng, ng), axes=(0, 1, 2))


def _trilinear(field: np.ndarray, pos: np.ndarray, lo: float, hi: float) -> np.ndarray:
    ng = field.shape[0]
    x = (pos - lo) / (hi - lo) * ng            # periodic cell-centred grid
    i0 = np.floor(x).astype(np.int64)
    t = x - i0
    out = np.zeros(pos.shape[0])
    for dx in (0, 1):
        wx = t[:, 0] if dx else 1.0 - t[:, 0]
        ix = (i0[:, 0] + dx) % ng
        for dy in (0, 1):
            wy = t[:, 1] if dy else 1.0 - t[:, 1]
            iy = (i0[:, 1] + dy) % ng
            for dz in (0, 1):
                wz = t[:, 2] if dz else 1.0 - t[:, 2]
                iz = (i0[:, 2] + dz) % ng
                out += wx * wy * wz * field[ix, iy, iz]
    return out


def turbulent_cloud(n: int, seed: int = BASE_SEED + 2, R: float = 1.0, grid: int = 128,
                    spectral_index: float = -4.0, alpha_vir: float = 2.0, sort: bool = True):
    """Uniform ball with a k^-4 Gaussian random velocity field, alpha = 2K/|W|."""
    g = rng(seed)
    r = R * g.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    pos = r[:, None] * _iso_dirs(g, n)
    vel = np.zeros((n, 3))
    for c in range(3):
        fld = _grf_component(g, grid, spectral_index)
        vel[:, c] = _trilinear(fld, pos, -R, R)
    vel -= vel.mean(axis=0)
    w_abs = 3.0 / (5.0 * R)
    k = 0.5 * (1.0 / max(n, 1)) * float((vel * vel).sum())
    if k > 0:
        vel *= np.sqrt(0.5 * alpha_vir * w_abs / k)
    return _finish(pos, vel, sort)


def zeldovich_box(n_side: int = 64, L: float = 1.0, amplitude: float = 0.1, jitter: float = 0.01,
                  seed: int = BASE_SEED + 6, sort: bool = True):
    """n_side^3 equal masses in the periodic cube [0, L)^3: a cubic lattice,
    displaced along x by amplitude * L / (2 pi) * sin(2 pi q_x / L) (one
    sinusoidal mode; amplitude < 1 before shell crossing) plus a small random
    jitter (fraction of the lattice spacing), with velocities along the
    displacement; positions wrapped into the box."""
    g = rng(seed)
    n = n_side**3
    spacing = L / n_side
    k = (np.arange(n_side) + 0.5) * spacing
    qx, qy, qz = np.meshgrid(k, k, k, indexing="ij")
    q = np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)
    disp = amplitude * L / (2.0 * np.pi) * np.sin(2.0 * np.pi * q[:, 0] / L)
    pos = q.copy()
    pos[:, 0] += disp
    pos += g.uniform(-0.5, 0.5, (n, 3)) * jitter * spacing
    pos = np.mod(pos, L)
    vel = np.zeros((n, 3))
    vel[:, 0] = -disp                      # converging flow toward the pancake plane
    vel += g.normal(0.0, 1e-3, (n, 3))
    return _finish(pos, vel, sort)


def soft_inputs(pos: np.ndarray, h0: float, seed: int = BASE_SEED + 7):
    """Seeded per-element supports and correction coefficients for parity runs
    of the adaptive-softening sums at sizes where solving the supports on the
    CPU is out of reach: h_i = h0 * (1 + |x_i|^2)^(1/2) * U(0.7, 1.3) (larger
    supports in sparser outskirts) and zeta_i = U(0.02, 0.3) * h_i^2 (the
    coefficient's scale, h^2).  Inputs only: neither is solved here."""
    g = rng(seed)
    n = pos.shape[0]
    h = h0 * np.sqrt(1.0 + (np.asarray(pos) ** 2).sum(axis=1)) * g.uniform(0.7, 1.3, n)
    zeta = g.uniform(0.02, 0.3, n) * h * h
    return h, zeta


def active_subset(n: int, fraction: float, seed: int) -> np.ndarray:
    """Seeded random subset of round(fraction*n) indices, ascending, int32."""
    m = int(round(fraction * n))
    m = max(0, min(n, m))
    sel = rng(seed).choice(n, size=m, replace=False)
    return np.sort(sel).astype(np.int32)


def batched_systems(n_systems: int = 256, n_min: int = 512, n_max: int = 65536,
                    seed: int = BASE_SEED + 4, frac_lo: float = 0.01, frac_hi: float = 0.5):
    """Independent systems, half Plummer half uniform, sizes log-uniform.

    Returns (pos, vel, mass, offsets, sizes, active_idx_list), systems packed
    contiguously; active_idx_list[s] holds local ascending indices of system s.
    """
    g = rng(seed)
    sizes = np.exp(g.uniform(np.log(n_min), np.log(n_max), n_systems)).astype(np.int64)
    sizes = np.clip(sizes, n_min, n_max)
    fracs = g.uniform(frac_lo, frac_hi, n_systems)
    pos, vel, mass, act = [], [], [], []
    for s in range(n_systems):
        ns = int(sizes[s])
        if s % 2 == 0:
            p, v, m = plummer(ns, seed=seed * 1000 + s)
        else:
            p, v, m = uniform_sphere(ns, seed=seed * 1000 + s)
        pos.append(p)
        vel.append(v)
        mass.append(m)
        act.append(active_subset(ns, max(1.0 / ns, fracs[s]), seed * 7 + s))
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return (np.concatenate(pos), np.concatenate(vel), np.concatenate(mass), offsets, sizes, act)
