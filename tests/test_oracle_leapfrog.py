"""Oracle leapfrog (the integration of the binary-polytrope test, Sect. 4)
pinned against properties fixed by the mathematics, independent of the
oracle's own code: exact time reversal of kick-drift-kick, a Kepler orbit
that closes with a second-order energy error, and linear momentum constant
to round-off because every SFMM pair force is antisymmetric."""
import math

import numpy as np

import oracle
import workloads


def test_kick_drift_kick_is_time_reversible():
    rng = np.random.default_rng(3)
    pos, m, h = workloads.uniform_sphere(300, 4)
    vel = 0.3 * rng.standard_normal((300, 3))
    x1, v1, _ = oracle.leapfrog(pos, vel, m, h, theta=0.5, p=2, leaf_size=8, dt=0.01, nsteps=12)
    # run back: same steps with -dt from the final state
    x0, v0, _ = oracle.leapfrog(x1, v1, m, h, theta=0.5, p=2, leaf_size=8, dt=-0.01, nsteps=12)
    np.testing.assert_allclose(x0, pos, rtol=0, atol=1e-11)
    np.testing.assert_allclose(v0, vel, rtol=0, atol=1e-10)


def test_two_body_kepler_orbit_closes():
    # two point masses far outside each other's kernel, circular orbit of
    # radius 1 (separation 1, total mass 1): period 2 pi; E = -1/(2 a) ...
    m = np.array([0.5, 0.5])
    h = np.array([1e-4, 1e-4])
    pos = np.array([[-0.5, 0.0, 0.0], [0.5, 0.0, 0.0]])
    v = math.sqrt(1.0 / 1.0) / 2.0  # each body moves at half the relative speed
    vel = np.array([[0.0, -v, 0.0], [0.0, v, 0.0]])
    T = 2.0 * math.pi
    errs = []
    for steps in (400, 800):
        x, u, _ = oracle.leapfrog(pos, vel, m, h, theta=0.5, p=2, leaf_size=1, dt=T / steps, nsteps=steps)
        sep = np.linalg.norm(x[1] - x[0])
        kin = 0.5 * (m[:, None] * u * u).sum()
        e = kin - m[0] * m[1] / sep
        errs.append(abs(e - (-0.125)) / 0.125)  # E0 = 1/2 (1/2)(1/4)*... = -G m1 m2 / (2 r) = -0.125
        assert np.linalg.norm(x - pos) < 2e-3 * (400 / steps) ** 2  # orbit closes
    assert errs[1] < errs[0] / 3.0  # energy error falls as dt^2
    assert errs[0] < 1e-3


def test_linear_momentum_is_constant_to_round_off():
    pos, vel, m, h = workloads.binary_orbit(2000, 11)
    _, _, rec = oracle.leapfrog(pos, vel, m, h, theta=0.5, p=2, leaf_size=16, dt=0.02, nsteps=40, record_every=4)
    scale = rec[:, 7].max()
    drift = np.abs(rec[:, 1:4] - rec[0, 1:4]).max()
    assert drift <= 1e-14 * scale, drift / scale
    # the binary set starts with its centre of mass at rest (to the rounding
    # of a sum of n mixed-sign terms)
    assert np.abs(rec[0, 1:4]).max() <= 1e-13 * scale


def test_binary_orbit_initial_conditions():
    pos, vel, m, h = workloads.binary_orbit(5000, 2)
    p = m[:, None] * vel
    assert np.abs(p.sum(0)).max() < 1e-13 * np.abs(p).sum()
    com = (m[:, None] * pos).sum(0) / m.sum()
    assert np.abs(com).max() < 0.05  # sampling noise of the two stars
    assert abs(workloads.orbital_period() - 2 * math.pi * math.sqrt(27.0)) < 1e-12
