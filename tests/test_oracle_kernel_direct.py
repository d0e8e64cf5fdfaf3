"""Pins of the oracle's softening kernel and direct sum (CPU only).

The kernel is checked against values derived independently from the M4
density (tests/golden/m4_softening.txt), against Poisson's equation by
finite differences, and against its limits; the direct sum against the
two-body law, Newton's third law and the closed-form potential and
acceleration of the homogeneous and Plummer spheres (Sect. 4.1 workloads).
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kernel():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "m4_softening.txt")) if l.strip() and l[0] != "#"]
    return np.array(rows, dtype=float)


def test_kernel_golden_values():
    g = _golden_kernel()
    for h in (1.0, 0.37):
        phi, gg = oracle.kernel(g[:, 0] * h, np.full(len(g), h))
        np.testing.assert_allclose(phi, g[:, 1] / h, rtol=1e-14, atol=0)
        np.testing.assert_allclose(gg, g[:, 2] / h**3, rtol=1e-14, atol=0)


def test_kernel_newtonian_outside_support():
    r = np.array([2.0, 2.5, 7.0, 100.0]) * 0.3
    phi, g = oracle.kernel(r, np.full(4, 0.3))
    np.testing.assert_allclose(phi, -1.0 / r, rtol=1e-15, atol=0)
    np.testing.assert_allclose(g, 1.0 / r**3, rtol=1e-15, atol=0)


def test_kernel_continuous_at_breaks():
    h = 0.7
    for q in (1.0, 2.0):
        r = np.array([q * h * (1 - 1e-12), q * h * (1 + 1e-12)])
        phi, g = oracle.kernel(r, np.full(2, h))
        assert abs(phi[0] - phi[1]) < 1e-10 * abs(phi[0])
        assert abs(g[0] - g[1]) < 1e-10 * abs(g[0])


def test_kernel_poisson_density_is_m4_and_normalised():
    """rho = (1/4 pi r^2) d/dr (r^3 g) must equal the M4 density and
    integrate to one (unit point mass smoothed over 2h)."""
    h = 1.0
    r = np.linspace(0.01, 2.5, 2000)
    eps = 1e-6
    _, gp = oracle.kernel(r + eps, np.full_like(r, h))
    _, gm = oracle.kernel(r - eps, np.full_like(r, h))
    d = ((r + eps) ** 3 * gp - (r - eps) ** 3 * gm) / (2 * eps)
    rho = d / (4 * math.pi * r**2)
    q = r / h
    w = np.where(q < 1, 1 - 1.5 * q**2 + 0.75 * q**3, np.where(q < 2, 0.25 * (2 - q) ** 3, 0.0)) / math.pi
    np.testing.assert_allclose(rho, w, atol=1e-6)
    # consistency of phi and g: phi' = g r
    phip, _ = oracle.kernel(r + eps, np.full_like(r, h))
    phim, _ = oracle.kernel(r - eps, np.full_like(r, h))
    _, g0 = oracle.kernel(r, np.full_like(r, h))
    np.testing.assert_allclose((phip - phim) / (2 * eps), g0 * r, rtol=1e-6, atol=1e-8)
    rr = np.linspace(0, 2, 200001)
    qq = rr
    ww = np.where(qq < 1, 1 - 1.5 * qq**2 + 0.75 * qq**3, 0.25 * (2 - qq) ** 3) / math.pi
    assert abs(np.trapezoid(4 * math.pi * rr**2 * ww, rr) - 1.0) < 1e-9


def test_direct_two_body():
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    m = np.array([2.0, 5.0])
    h = np.array([0.1, 0.2])
    acc, pot = oracle.direct(pos, m, h, G=1.5)
    # outside the kernel: Newton, attractive, equal and opposite
    np.testing.assert_allclose(acc[0], 1.5 * 5.0 * np.array([3.0, 4.0, 0.0]) / 125.0, rtol=1e-15)
    np.testing.assert_allclose(acc[1], -1.5 * 2.0 * np.array([3.0, 4.0, 0.0]) / 125.0, rtol=1e-15)
    np.testing.assert_allclose(pot, [-1.5 * 5.0 / 5.0, -1.5 * 2.0 / 5.0], rtol=1e-15)
    # inside the kernel: r = 0.5 h_j for h_j = 1, mean of the two kernels
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    h = np.array([1.0, 1.0])
    acc, pot = oracle.direct(pos, np.array([1.0, 1.0]), h)
    gk = _golden_kernel()
    row = gk[np.isclose(gk[:, 0], 0.5)][0]
    np.testing.assert_allclose(acc[0, 0], row[2] * 0.5, rtol=1e-14)
    np.testing.assert_allclose(pot[0], row[1], rtol=1e-14)
    # self potential option adds G m phi(0, h) = -7/5 G m / h
    _, pot2 = oracle.direct(pos, np.array([1.0, 1.0]), h, self_potential=True)
    np.testing.assert_allclose(pot2 - pot, -1.4, rtol=1e-14)


def test_direct_newton_third_law():
    pos, m, h = workloads.plummer(1500, 7)
    m = m * np.random.default_rng(1).uniform(0.5, 1.5, len(m))
    acc, _ = oracle.direct(pos, m, h)
    mom = (m[:, None] * acc).sum(0)
    assert np.linalg.norm(mom) <= 1e-15 * np.abs(m[:, None] * acc).sum()


def _radial_bins(r, vals, edges):
    out = []
    for a, b in zip(edges[:-1], edges[1:]):
        sel = (r >= a) & (r < b)
        out.append((sel.sum(), vals[sel].mean() if sel.any() else np.nan))
    return out


def test_direct_uniform_sphere_closed_form():
    n = 6000
    pos, m, h = workloads.uniform_sphere(n, 11)
    acc, pot = oracle.direct(pos, m, h)
    r = np.linalg.norm(pos, axis=1)
    ar = -(acc * pos).sum(1) / r  # inward radial acceleration
    edges = np.array([0.3, 0.5, 0.7, 0.9])
    for (cnt, mean_a), (cnt2, mean_p), a, b in zip(_radial_bins(r, ar, edges), _radial_bins(r, pot, edges),
                                                   edges[:-1], edges[1:]):
        rm = r[(r >= a) & (r < b)]
        exact_a = rm.mean()                     # |a| = r for M = R = 1
        exact_p = (-(3 - rm**2) / 2).mean()     # Phi = -(3 - r^2)/2
        assert abs(mean_a - exact_a) < 4.0 / math.sqrt(cnt) * exact_a + 0.02
        assert abs(mean_p - exact_p) < 0.02 * abs(exact_p)
    W = 0.5 * (m * pot).sum()
    assert abs(W - (-0.6)) < 0.01


def test_direct_plummer_closed_form():
    n = 6000
    pos, m, h = workloads.plummer(n, 12)
    acc, pot = oracle.direct(pos, m, h)
    r = np.linalg.norm(pos, axis=1)
    ar = -(acc * pos).sum(1) / r
    edges = np.array([0.5, 1.0, 1.5, 2.5])
    for (cnt, mean_a), (cnt2, mean_p), a, b in zip(_radial_bins(r, ar, edges), _radial_bins(r, pot, edges),
                                                   edges[:-1], edges[1:]):
        rm = r[(r >= a) & (r < b)]
        exact_a = (rm / (rm**2 + 1) ** 1.5).mean()
        exact_p = (-1 / np.sqrt(rm**2 + 1)).mean()
        assert abs(mean_a - exact_a) < 4.0 / math.sqrt(cnt) * exact_a + 0.02 * exact_a
        assert abs(mean_p - exact_p) < 0.03 * abs(exact_p)
    # W of the Plummer sphere truncated at 20a: -3 pi / 32 for the untruncated
    # model; truncation changes it by well under 1 %
    W = 0.5 * (m * pot).sum()
    assert abs(W - (-3 * math.pi / 32)) < 0.02 * 3 * math.pi / 32


def test_direct_targets_subset():
    pos, m, h = workloads.uniform_sphere(500, 3)
    acc, pot = oracle.direct(pos, m, h)
    t = np.array([0, 17, 499, 250])
    a2, p2 = oracle.direct(pos, m, h, targets=t)
    np.testing.assert_array_equal(a2, acc[t])
    np.testing.assert_array_equal(p2, pot[t])
