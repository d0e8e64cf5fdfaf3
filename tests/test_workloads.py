"""Checks of the seeded input generators (CPU only)."""
import math

import numpy as np

import workloads


def test_lane_emden_n15_constants():
    """Lane-Emden n = 1.5: first zero xi_1 = 3.65375 and
    -xi_1^2 theta'(xi_1) = 2.71406 (Chandrasekhar 1939, Table 4)."""
    xi, th, mu = workloads.lane_emden(1.5)
    assert abs(xi[-1] - 3.65375) < 2e-4
    assert abs(mu[-1] - 2.71406) < 2e-4


def test_reproducible_and_shapes():
    for gen in (workloads.uniform_sphere, workloads.plummer, workloads.binary_polytrope):
        a = gen(1000, 4)
        b = gen(1000, 4)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
        pos, m, h = a
        assert pos.shape == (1000, 3) and m.shape == (1000,) and h.shape == (1000,)
        assert (h > 0).all() and (m > 0).all() and np.isfinite(pos).all()
        assert abs(m.sum() - 1.0) < 1e-12


def test_plummer_mass_profile():
    pos, m, h = workloads.plummer(200_000, 1)
    r = np.linalg.norm(pos, axis=1)
    assert r.max() <= 20.0 + 1e-9
    for R in (0.5, 1.0, 3.0):
        exact = (R**3 / (1 + R**2) ** 1.5) / (400 / 401) ** 1.5
        assert abs((r < R).mean() - exact) < 0.005


def test_uniform_profile_and_h():
    pos, m, h = workloads.uniform_sphere(100_000, 2)
    r = np.linalg.norm(pos, axis=1)
    assert r.max() <= 1.0
    assert abs((r < 0.5).mean() - 0.125) < 0.005
    np.testing.assert_allclose(h, 1.2 * (m / (3 / (4 * math.pi))) ** (1 / 3))


def test_binary_polytrope_masses_and_com():
    pos, m, h = workloads.binary_polytrope(100_000, 3)
    n1 = int(round(100_000 / 1.3))
    com = (m[:, None] * pos).sum(0)
    assert np.linalg.norm(com) < 0.02
    c1 = pos[:n1].mean(0)
    c2 = pos[n1:].mean(0)
    assert abs(c1[0] - (-3.0 * 0.3 / 1.3)) < 0.01 and abs(c2[0] - 3.0 / 1.3) < 0.01
    assert np.linalg.norm(pos[:n1] - c1, axis=1).max() <= 1.0 + 1e-3
    assert np.linalg.norm(pos[n1:] - c2, axis=1).max() <= 0.6 + 1e-3


def test_ensemble_and_clustered():
    pos, m, h, off = workloads.ensemble(4, nsys=6)
    assert off[0] == 0 and off[-1] == len(m) and len(off) == 7
    sizes = np.diff(off)
    assert (sizes >= 1000).all() and (sizes < 100_000).all()
    pos, m, h = workloads.clustered_cloud(50_000, 5)
    assert len(m) == 50_000 and (h > 0).all()
