"""Seeded synthetic particle sets for the SFMM gravity solver and its oracle.

This module is the only code shared by the CUDA path and the CPU oracle: it
draws particle positions, masses and smoothing lengths and holds none of the
method's arithmetic (no tree, no softening kernel, no expansion).  Every
generator returns ``(pos, mass, h)`` as float64 NumPy arrays of shapes
``(N, 3)``, ``(N,)`` and ``(N,)``.

Workloads follow the test problems of the paper (Sect. 4.1: Plummer and
homogeneous spheres of equal-mass particles; Sect. 4.2: a binary of n = 1.5
polytropes) plus two stress cases (a batched ensemble and a clustered
cloud).  Smoothing lengths come from the analytic density,
``h = 1.2 (m / rho)^(1/3)``, the usual SPH relation between particle mass,
density and smoothing length.
"""
from __future__ import annotations

import math

import numpy as np

HFACT = 1.2


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere (cos(theta) and phi uniform)."""
    mu = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return np.stack([s * np.cos(phi), s * np.sin(phi), mu], axis=1)


def _hsml(m: np.ndarray, rho: np.ndarray) -> np.ndarray:
    return HFACT * np.cbrt(m / rho)


def uniform_sphere(n: int, seed: int, radius: float = 1.0, mass: float = 1.0):
    """Homogeneous sphere: r = R u^(1/3), isotropic directions, equal masses."""
    rng = np.random.default_rng(seed)
    r = radius * np.cbrt(rng.uniform(0.0, 1.0, n))
    pos = r[:, None] * _isotropic(rng, n)
    m = np.full(n, mass / n)
    rho = np.full(n, 3.0 * mass / (4.0 * math.pi * radius ** 3))
    return pos, m, _hsml(m, rho)


def plummer_density(r, a: float = 1.0, mass: float = 1.0):
    """Plummer density 3 M a^2 / (4 pi (a^2 + r^2)^(5/2)) (Sect. 4.1; the
    printed exponent sign is a typesetting slip, the profile is Plummer's)."""
    return 3.0 * mass * a * a / (4.0 * math.pi * (a * a + np.asarray(r) ** 2) ** 2.5)


def _plummer_radii(rng, n, a, rtrunc):
    umax = (rtrunc * rtrunc / (a * a + rtrunc * rtrunc)) ** 1.5
    u = rng.uniform(0.0, umax, n)
    u = np.maximum(u, np.finfo(float).tiny)
    return a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)


def plummer(n: int, seed: int, a: float = 1.0, mass: float = 1.0, rtrunc: float = 20.0):
    """Plummer sphere truncated at ``rtrunc``: inverse-CDF radii, isotropic
    directions, equal masses ``mass / n``."""
    rng = np.random.default_rng(seed)
    r = _plummer_radii(rng, n, a, rtrunc)
    pos = r[:, None] * _isotropic(rng, n)
    m = np.full(n, mass / n)
    return pos, m, _hsml(m, plummer_density(r, a, mass))


def lane_emden(npoly: float = 1.5, dxi: float = 1e-4):
    """Lane-Emden solution theta(xi) by classical RK4 from a series start.

    Returns (xi, theta, mu) tabulated up to the first zero xi_1, where
    mu(xi) = -xi^2 theta'(xi) is the dimensionless enclosed mass.
    """
    xi0 = 1e-3
    th = 1.0 - xi0 ** 2 / 6.0 + npoly * xi0 ** 4 / 120.0
    dth = -xi0 / 3.0 + npoly * xi0 ** 3 / 30.0

    def f(x, y):
        t, dt = y
        return np.array([dt, -max(t, 0.0) ** npoly - 2.0 * dt / x])

    xs, ts, mus = [0.0, xi0], [1.0, th], [0.0, -xi0 * xi0 * dth]
    x, y = xi0, np.array([th, dth])
    while True:
        k1 = f(x, y)
        k2 = f(x + dxi / 2, y + dxi / 2 * k1)
        k3 = f(x + dxi / 2, y + dxi / 2 * k2)
        k4 = f(x + dxi, y + dxi * k3)
        yn = y + dxi / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        if yn[0] <= 0.0:
            # linear interpolation to the zero crossing
            frac = y[0] / (y[0] - yn[0])
            x1 = x + frac * dxi
            d1 = y[1] + frac * (yn[1] - y[1])
            xs.append(x1)
            ts.append(0.0)
            mus.append(-x1 * x1 * d1)
            break
        x, y = x + dxi, yn
        xs.append(x)
        ts.append(y[0])
        mus.append(-x * x * y[1])
    return np.array(xs), np.array(ts), np.array(mus)


_LE_CACHE: dict = {}


def _lane_emden_cached():
    if "le" not in _LE_CACHE:
        _LE_CACHE["le"] = lane_emden()
    return _LE_CACHE["le"]


def polytrope_star(rng, n, mass, radius, centre, npoly=1.5):
    """One n=1.5 polytrope: radii by inverse cumulative Lane-Emden mass,
    random angles; returns positions and the analytic density at each."""
    xi, th, mu = _lane_emden_cached()
    xi1, mu1 = xi[-1], mu[-1]
    rho_c = mass * xi1 ** 3 / (4.0 * math.pi * radius ** 3 * mu1)
    u = rng.uniform(0.0, 1.0, n)
    u = np.minimum(u, 1.0 - 0.5 / n)
    xq = np.interp(u * mu1, mu, xi)
    r = radius * xq / xi1
    pos = r[:, None] * _isotropic(rng, n) + np.asarray(centre)[None, :]
    rho = rho_c * np.maximum(np.interp(xq, xi, th), 0.0) ** npoly
    rho = np.maximum(rho, 1e-6 * rho_c)
    return pos, rho


def binary_polytrope(n: int, seed: int, q: float = 0.3, r1: float = 1.0, r2: float = 0.6,
                     sep: float = 3.0):
    """Two n=1.5 polytropes of mass 1/(1+q) and q/(1+q), radii r1 and r2,
    centres ``sep`` apart on x with the centre of mass at the origin;
    particle numbers in mass proportion, equal particle masses."""
    rng = np.random.default_rng(seed)
    m1, m2 = 1.0 / (1.0 + q), q / (1.0 + q)
    n1 = int(round(n * m1))
    n2 = n - n1
    x1 = -sep * m2
    x2 = sep * m1
    p1, rho1 = polytrope_star(rng, n1, m1, r1, (x1, 0.0, 0.0))
    p2, rho2 = polytrope_star(rng, n2, m2, r2, (x2, 0.0, 0.0))
    pos = np.concatenate([p1, p2])
    m = np.full(n, 1.0 / n)
    rho = np.concatenate([rho1, rho2])
    return pos, m, _hsml(m, rho)


def binary_orbit(n: int, seed: int, q: float = 0.3, r1: float = 1.0, r2: float = 0.6, sep: float = 3.0,
                 G: float = 1.0):
    """The binary polytrope set moving on a circular orbit: every particle of
    a star gets that star's orbital velocity (along y, perpendicular to the
    separation on x), v_rel = sqrt(G M / sep) with M the total mass and the
    centre of mass at rest.  Returns (pos, vel, m, h); the orbital period is
    2 pi sqrt(sep^3 / (G M))."""
    pos, m, h = binary_polytrope(n, seed, q, r1, r2, sep)
    n1 = int(round(n * (1.0 / (1.0 + q))))
    m1, m2 = m[:n1].sum(), m[n1:].sum()
    mt = m1 + m2
    v_rel = math.sqrt(G * mt / sep)
    vel = np.zeros((n, 3))
    vel[:n1, 1] = -v_rel * m2 / mt
    vel[n1:, 1] = v_rel * m1 / mt
    return pos, vel, m, h


def orbital_period(sep: float = 3.0, mass: float = 1.0, G: float = 1.0) -> float:
    return 2.0 * math.pi * math.sqrt(sep ** 3 / (G * mass))


def clustered_cloud(n: int, seed: int, nclump: int = 64, clump_scale: float = 0.02,
                    halo_frac: float = 0.7, sigma: float = 1.0):
    """Plummer halo (a=1, truncated at 20a) holding ``halo_frac`` of the mass
    plus ``nclump`` Plummer clumps (scale 0.02, truncated at 20 scales) with
    log-normal masses normalised to the rest; clump centres follow the halo
    profile truncated at 5a; equal particle masses; h from the summed
    analytic density, each clump's term truncated at its 20 scales."""
    rng = np.random.default_rng(seed)
    cm = rng.lognormal(0.0, sigma, nclump)
    cm *= (1.0 - halo_frac) / cm.sum()
    counts = np.floor(cm * n).astype(np.int64)
    nh = n - counts.sum()
    centres = _plummer_radii(rng, nclump, 1.0, 5.0)[:, None] * _isotropic(rng, nclump)
    parts = []
    rh = _plummer_radii(rng, nh, 1.0, 20.0)
    parts.append(rh[:, None] * _isotropic(rng, nh))
    for c in range(nclump):
        rc = _plummer_radii(rng, counts[c], clump_scale, 20.0 * clump_scale)
        parts.append(rc[:, None] * _isotropic(rng, counts[c]) + centres[c][None, :])
    pos = np.concatenate(parts)
    m = np.full(n, 1.0 / n)
    rho = plummer_density(np.linalg.norm(pos, axis=1), 1.0, halo_frac)
    # each clump's density is truncated like its particles (at 20 scales): only
    # particles inside that ball receive it; they are found from an x-sorted slab
    rcut = 20.0 * clump_scale
    xorder = np.argsort(pos[:, 0], kind="stable")
    xs, ys, zs = pos[xorder, 0], pos[xorder, 1], pos[xorder, 2]
    for c in range(nclump):
        cx, cy, cz = centres[c]
        lo, hi = np.searchsorted(xs, [cx - rcut, cx + rcut])
        box = np.flatnonzero((np.abs(ys[lo:hi] - cy) < rcut) & (np.abs(zs[lo:hi] - cz) < rcut)) + lo
        dx, dy, dz = xs[box] - cx, ys[box] - cy, zs[box] - cz
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        inside = d < rcut
        rho[xorder[box[inside]]] += plummer_density(d[inside], clump_scale, cm[c])
    return pos, m, _hsml(m, rho)


def ensemble_sizes(seed: int, nsys: int = 256, lo: float = 3.0, hi: float = 5.0):
    """System sizes N_s = floor(10^U(lo, hi)) for the batched ensemble."""
    rng = np.random.default_rng(seed)
    return np.floor(10.0 ** rng.uniform(lo, hi, nsys)).astype(np.int64)


def ensemble(seed: int, nsys: int = 256, lo: float = 3.0, hi: float = 5.0):
    """Batched ensemble: even systems Plummer, odd systems uniform spheres,
    sizes log-uniform in [10^lo, 10^hi].  Returns (pos, m, h, offsets) with
    the systems packed back to back and offsets of length nsys + 1."""
    sizes = ensemble_sizes(seed, nsys, lo, hi)
    ps, ms, hs = [], [], []
    for s, ns in enumerate(sizes):
        gen = plummer if s % 2 == 0 else uniform_sphere
        p, m, h = gen(int(ns), seed * 1000 + s)
        ps.append(p)
        ms.append(m)
        hs.append(h)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(ps), np.concatenate(ms), np.concatenate(hs), offsets


# Named workloads: the sizes and parameters of the solver's benchmark
# configurations (seed = 1000 + index).
WORKLOADS = {
    "uniform_1e4": dict(gen="uniform_sphere", n=10_000, seed=1001, theta=0.5, leaf_size=10),
    "plummer_1e6": dict(gen="plummer", n=1_000_000, seed=1002, theta=0.5, leaf_size=16),
    "binary_polytrope_2e6": dict(gen="binary_polytrope", n=2_000_000, seed=1003, theta=0.5, leaf_size=16),
    "ensemble_256": dict(gen="ensemble", n=None, seed=1004, theta=0.5, leaf_size=None),
    "clustered_1.6e7": dict(gen="clustered_cloud", n=16_000_000, seed=1005, theta=0.5, leaf_size=16),
}


def make(name: str, n: int | None = None, seed: int | None = None):
    """Generate a named workload (optionally at another size or seed)."""
    w = WORKLOADS[name]
    gen = globals()[w["gen"]]
    s = w["seed"] if seed is None else seed
    if w["gen"] == "ensemble":
        return gen(s)
    return gen(w["n"] if n is None else n, s)
