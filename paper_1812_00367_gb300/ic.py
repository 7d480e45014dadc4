"""Seeded synthetic initial conditions for the Hermite-6 N-body workloads.

This module is the only code that both the CUDA path and the CPU oracle
consume.  It draws particle masses, positions and velocities; it holds none of
the integration method (no force, predictor, corrector or time step).

The paper (Sec. 4) measures "as a function of the number of particles" on
unstated inputs; these generators are the synthetic stand-ins:

* Plummer spheres sampled after Aarseth, Henon & Wielen (1974), mass cut at
  0.999 of the total (reading), scaled analytically to Henon units
  (G = M = 1, E = -1/4 for the untruncated model: length scale 3 pi / 16),
  then moved to the centre-of-mass frame.
* A Kroupa (2001)-like two-segment power law mass spectrum (slopes 1.3 below
  and 2.3 above a break at five times the minimum; masses in [0.1, 100] before
  rescaling the total to 1).
* Hernquist (1990) spheres: radii from the inverse cumulative mass (cut at
  0.99 of the mass), speeds from the closed-form isotropic distribution
  function by rejection.
* A pair of Hernquist spheres on a parabolic two-point-mass orbit.
* Batches of independent Plummer clusters with log-uniform sizes.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
Layout: ``m (n,)``, ``x (n,3)``, ``v (n,3)``, float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

HENON_PLUMMER_SCALE = 3.0 * math.pi / 16.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere."""
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def _to_com_frame(m: np.ndarray, x: np.ndarray, v: np.ndarray):
    mt = m.sum()
    x = x - (m[:, None] * x).sum(axis=0) / mt
    v = v - (m[:, None] * v).sum(axis=0) / mt
    return x, v


def plummer(n: int, seed: int = 1, masses: np.ndarray | None = None,
            mass_cut: float = 0.999):
    """Plummer sphere in Henon units (Aarseth, Henon & Wielen 1974 sampling).

    ``masses`` (optional, length n, any positive values) replaces equal masses;
    they are rescaled to sum to 1.  Returns (m, x, v).
    """
    rng = _rng(seed)
    if masses is None:
        m = np.full(n, 1.0 / n)
    else:
        m = np.asarray(masses, dtype=np.float64).copy()
        m /= m.sum()
    # radius from the cumulative mass fraction X: M(r) = r^3 / (1 + r^2)^{3/2}
    X = rng.uniform(0.0, mass_cut, n)
    X = np.maximum(X, 1e-300)
    r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _isotropic(rng, n)
    # speed fraction q = v / v_esc from g(q) = q^2 (1 - q^2)^{7/2} by rejection
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        q4 = rng.uniform(0.0, 1.0, todo.size)
        q5 = rng.uniform(0.0, 0.1, todo.size)
        ok = q5 < q4 * q4 * (1.0 - q4 * q4) ** 3.5
        q[todo[ok]] = q4[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    v = (q * vesc)[:, None] * _isotropic(rng, n)
    # Henon units: total energy -1/4 for G = M = 1
    x *= HENON_PLUMMER_SCALE
    v /= math.sqrt(HENON_PLUMMER_SCALE)
    x, v = _to_com_frame(m, x, v)
    return m, x, v


def kroupa_masses(n: int, seed: int = 1, m_min: float = 0.1, m_max: float = 100.0):
    """Kroupa-like two-segment IMF: dN/dm ~ m^-1.3 on [m_min, 5 m_min],
    m^-2.3 on [5 m_min, m_max], continuous at the break.  Sum rescaled to 1."""
    rng = _rng(seed)
    mb = 5.0 * m_min
    a1, a2 = 1.3, 2.3

    def seg_int(lo, hi, a):  # integral of m^-a
        return (hi ** (1 - a) - lo ** (1 - a)) / (1 - a)

    # continuity: c2 mb^-a2 = mb^-a1  ->  c2 = mb^(a2 - a1)
    w1 = seg_int(m_min, mb, a1)
    w2 = mb ** (a2 - a1) * seg_int(mb, m_max, a2)
    u = rng.uniform(0.0, 1.0, n)
    pick1 = rng.uniform(0.0, 1.0, n) < w1 / (w1 + w2)

    def inv(lo, hi, a, uu):
        e = 1 - a
        return (lo ** e + uu * (hi ** e - lo ** e)) ** (1.0 / e)

    m = np.where(pick1, inv(m_min, mb, a1, u), inv(mb, m_max, a2, u))
    return m / m.sum()


def hernquist_df(E: np.ndarray, M: float = 1.0, a: float = 1.0) -> np.ndarray:
    """Isotropic distribution function of the Hernquist (1990) model, G = 1.

    E is the specific energy (negative for bound orbits)."""
    vg = math.sqrt(M / a)
    q = np.sqrt(np.clip(-a * E / M, 0.0, 1.0 - 1e-15))
    pref = M / (8.0 * math.sqrt(2.0) * math.pi ** 3 * a ** 3 * vg ** 3)
    body = (3.0 * np.arcsin(q)
            + q * np.sqrt(1.0 - q * q) * (1.0 - 2.0 * q * q) * (8.0 * q ** 4 - 8.0 * q * q - 3.0))
    return pref * body / (1.0 - q * q) ** 2.5


def hernquist(n: int, seed: int = 1, M: float = 1.0, a: float = 1.0,
              mass_cut: float = 0.99):
    """Hernquist sphere: equal masses M/n, isotropic velocities from its DF."""
    rng = _rng(seed)
    m = np.full(n, M / n)
    X = rng.uniform(0.0, mass_cut, n)
    sX = np.sqrt(X)
    r = a * sX / (1.0 - sX)
    x = r[:, None] * _isotropic(rng, n)
    phi = -M / (r + a)
    vesc = np.sqrt(-2.0 * phi)
    # rejection in speed with target density ~ v^2 f(phi + v^2/2) on [0, vesc]
    grid = np.linspace(0.0, 1.0, 65)[1:-1]
    vv = grid[None, :] * vesc[:, None]
    dens = vv * vv * hernquist_df(phi[:, None] + 0.5 * vv * vv, M, a)
    fmax = 1.2 * dens.max(axis=1)
    speed = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        vt = rng.uniform(0.0, 1.0, todo.size) * vesc[todo]
        ft = vt * vt * hernquist_df(phi[todo] + 0.5 * vt * vt, M, a)
        ok = rng.uniform(0.0, 1.0, todo.size) * fmax[todo] < ft
        speed[todo[ok]] = vt[ok]
        todo = todo[~ok]
    v = speed[:, None] * _isotropic(rng, n)
    x, v = _to_com_frame(m, x, v)
    return m, x, v


def parabolic_pair(m1: float, m2: float, separation: float, pericentre: float):
    """Relative position and velocity of two point masses on a parabolic
    (e = 1) orbit, approaching, at the given separation; barycentric offsets.

    Returns (dx1, dv1, dx2, dv2) to add to the two bodies."""
    mu = m1 + m2
    d = float(separation)
    speed = math.sqrt(2.0 * mu / d)
    h = math.sqrt(2.0 * mu * pericentre)           # specific angular momentum
    vt = h / d
    vr = -math.sqrt(max(0.0, speed * speed - vt * vt))
    rel_x = np.array([d, 0.0, 0.0])
    rel_v = np.array([vr, vt, 0.0])
    f1, f2 = m2 / mu, m1 / mu
    return -f1 * rel_x, -f1 * rel_v, f2 * rel_x, f2 * rel_v


def hernquist_merger(n_each: int, seed: int = 1, separation: float = 20.0,
                     pericentre: float = 1.0):
    """Two equal Hernquist spheres (M = 1, a = 1 each) on a parabolic orbit."""
    m1, x1, v1 = hernquist(n_each, seed=seed)
    m2, x2, v2 = hernquist(n_each, seed=seed + 1_000_003)
    dx1, dv1, dx2, dv2 = parabolic_pair(m1.sum(), m2.sum(), separation, pericentre)
    m = np.concatenate([m1, m2])
    x = np.concatenate([x1 + dx1, x2 + dx2])
    v = np.concatenate([v1 + dv1, v2 + dv2])
    return m, x, v


@dataclass
class Batch:
    m: np.ndarray
    x: np.ndarray
    v: np.ndarray
    offsets: np.ndarray  # int64, length n_clusters + 1

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)


def cluster_sizes(n_clusters: int, seed: int, n_min: int = 256, n_max: int = 16384):
    rng = _rng(seed)
    u = rng.uniform(math.log(n_min), math.log(n_max), n_clusters)
    return np.floor(np.exp(u)).astype(np.int64)


def plummer_batch(n_clusters: int = 512, seed: int = 1, n_min: int = 256,
                  n_max: int = 16384, sizes=None) -> Batch:
    """Independent Plummer clusters (Henon units each), concatenated."""
    if sizes is None:
        sizes = cluster_sizes(n_clusters, seed, n_min, n_max)
    sizes = np.asarray(sizes, dtype=np.int64)
    parts = [plummer(int(nk), seed=seed * 100_003 + k) for k, nk in enumerate(sizes)]
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return Batch(np.concatenate([p[0] for p in parts]),
                 np.concatenate([p[1] for p in parts]),
                 np.concatenate([p[2] for p in parts]), offsets)
