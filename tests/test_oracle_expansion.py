"""Pins of the oracle's expansion pieces (CPU only).

D_gamma: closed forms to order 2, the Laplace trace identity, and finite
differences to order 5.  Moments: brute force and the shift identity of
App. A.1.  M2L: exact for single particles and whenever a_i = b_j (Sect. 2.2),
geometric convergence in p for well-separated clusters.  L2L: translation
invariance of the evaluated expansion (App. A.2).
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def multi_indices(P):
    return [(a, b, c) for n in range(P + 1) for a in range(n, -1, -1) for b in range(n - a, -1, -1)
            for c in [n - a - b]]


def test_derivs_closed_forms():
    r = np.array([0.3, -1.1, 0.7])
    R = np.linalg.norm(r)
    g = multi_indices(2)
    D = dict(zip(g, oracle.derivs(2, r, g)))
    assert D[(0, 0, 0)] == pytest.approx(1 / R, rel=1e-15)
    for i, e in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        assert D[e] == pytest.approx(-r[i] / R**3, rel=1e-14)
    for i in range(3):
        for j in range(3):
            gam = [0, 0, 0]
            gam[i] += 1
            gam[j] += 1
            exact = 3 * r[i] * r[j] / R**5 - (1.0 if i == j else 0.0) / R**3
            assert D[tuple(gam)] == pytest.approx(exact, rel=1e-13, abs=1e-15)


def test_derivs_laplace_trace():
    r = np.array([0.8, 0.2, -0.5])
    g = multi_indices(5)
    D = dict(zip(g, oracle.derivs(5, r, g)))
    for gam in multi_indices(3):
        s = sum(D[tuple(np.add(gam, 2 * np.eye(3, dtype=int)[i]))] for i in range(3))
        scale = max(abs(D[tuple(np.add(gam, 2 * np.eye(3, dtype=int)[i]))]) for i in range(3))
        assert abs(s) < 1e-12 * scale


def test_derivs_finite_differences():
    """D_{gamma + e_i} = d/dr_i D_gamma, by a Richardson-extrapolated
    central difference, for |gamma| <= 4."""
    r = np.array([0.9, -0.4, 0.6])
    gs = multi_indices(5)
    D = dict(zip(gs, oracle.derivs(5, r, gs)))
    for gam in multi_indices(4):
        for i in range(3):
            e = np.zeros(3)
            e[i] = 1.0

            def cd(step):
                dp = oracle.derivs(5, r + step * e, [gam])[0]
                dm = oracle.derivs(5, r - step * e, [gam])[0]
                return (dp - dm) / (2 * step)

            h = 1e-3
            est = (4 * cd(h / 2) - cd(h)) / 3
            target = D[tuple(np.add(gam, np.eye(3, dtype=int)[i]))]
            assert abs(est - target) < 1e-7 * max(1.0, abs(target))


def test_p2m_brute_force():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(7, 3))
    m = rng.uniform(0.5, 2.0, 7)
    s = np.array([0.1, -0.2, 0.3])
    Q = oracle.p2m(3, x, m, s)
    b = x - s
    for n in range(4):
        off = oracle.rank_offset(n)
        for idx in itertools.product(range(3), repeat=n):
            flat = 0
            for a in idx:
                flat = flat * 3 + a
            exact = sum(m[j] * np.prod([b[j, a] for a in idx]) for j in range(7))
            assert Q[off + flat] == pytest.approx(exact, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_m2m_equals_direct_p2m(p):
    """App. A.1: moments of a child about its centre, shifted to the parent
    centre, equal the direct moments about the parent centre."""
    rng = np.random.default_rng(10 + p)
    x = rng.normal(size=(20, 3)) * 0.3 + 1.0
    m = rng.uniform(0.5, 2.0, 20)
    sc = np.array([1.05, 0.97, 1.02])
    sp = np.array([0.7, 1.4, 0.9])
    Qc = oracle.p2m(p, x, m, sc)
    Qp = oracle.m2m(p, Qc, sc - sp)
    Qd = oracle.p2m(p, x, m, sp)
    np.testing.assert_allclose(Qp, Qd, rtol=1e-13, atol=1e-14 * np.abs(Qd).max())


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_m2l_exact_single_particles(p):
    """Point nodes (a = b = 0): every order reproduces Newton exactly."""
    xA = np.array([[0.2, 0.1, -0.3]])
    xB = np.array([[2.0, -1.0, 0.5]])
    mB = np.array([3.0])
    acc, pot = oracle.m2l_eval(p, xA[0], xB[0], xB, mB, xA, G=2.0)
    d = xA[0] - xB[0]
    r = np.linalg.norm(d)
    np.testing.assert_allclose(acc[0], -2.0 * 3.0 * d / r**3, rtol=1e-14)
    assert pot[0] == pytest.approx(-2.0 * 3.0 / r, rel=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_m2l_exact_when_a_equals_b(p):
    """Sect. 2.2: the expansion is exact when a_i = b_j (here one particle
    per node, both displaced by the same vector from their centres)."""
    sA = np.array([0.0, 0.0, 0.0])
    sB = np.array([1.5, 0.5, -0.7])
    off = np.array([0.11, -0.07, 0.05])
    acc, pot = oracle.m2l_eval(p, sA, sB, (sB + off)[None], np.array([1.0]), (sA + off)[None])
    d = sA - sB
    r = np.linalg.norm(d)
    np.testing.assert_allclose(acc[0], -d / r**3, rtol=1e-13)
    assert pot[0] == pytest.approx(-1 / r, rel=1e-13)


def test_m2l_converges_geometrically_in_p():
    rng = np.random.default_rng(3)
    xA = rng.uniform(-0.5, 0.5, (30, 3)) * 0.4
    xB = rng.uniform(-0.5, 0.5, (40, 3)) * 0.4 + np.array([2.0, 0.7, -0.4])
    mB = rng.uniform(0.5, 1.5, 40)
    sA = xA.mean(0)
    sB = (mB[:, None] * xB).sum(0) / mB.sum()
    exact_a = np.zeros((30, 3))
    exact_p = np.zeros(30)
    for j in range(40):
        d = xA - xB[j]
        r = np.linalg.norm(d, axis=1)
        exact_a += -mB[j] * d / r[:, None] ** 3
        exact_p += -mB[j] / r
    errs = []
    for p in range(5):
        acc, pot = oracle.m2l_eval(p, sA, sB, xB, mB, xA)
        errs.append((np.abs(acc - exact_a).max() / np.abs(exact_a).max(),
                     np.abs(pot - exact_p).max() / np.abs(exact_p).max()))
    errs = np.array(errs)
    # each order gains at least a factor ~ (size/d) ~ 0.2 in accuracy
    for p in range(4):
        assert errs[p + 1, 0] < 0.5 * errs[p, 0]
        assert errs[p + 1, 1] < 0.5 * errs[p, 1]
    assert errs[4, 0] < 1e-4


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_l2l_translation_invariance(p):
    """App. A.2: translating the coefficients to a new centre and evaluating
    there equals evaluating about the old centre (a polynomial identity)."""
    rng = np.random.default_rng(20 + p)
    xB = rng.uniform(-0.2, 0.2, (10, 3)) + np.array([3.0, 1.0, 0.0])
    mB = rng.uniform(0.5, 1.5, 10)
    xA = rng.uniform(-0.3, 0.3, (12, 3))
    sA = np.zeros(3)
    sA2 = np.array([0.12, -0.05, 0.08])
    sB = (mB[:, None] * xB).sum(0) / mB.sum()
    a1, p1 = oracle.m2l_eval(p, sA, sB, xB, mB, xA)
    a2, p2 = oracle.m2l_l2l_eval(p, sA, sA2, sB, xB, mB, xA)
    np.testing.assert_allclose(a2, a1, rtol=1e-13, atol=1e-15 * np.abs(a1).max())
    np.testing.assert_allclose(p2, p1, rtol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_m2l_pairwise_antisymmetry(p):
    """Newton's third law for one node pair (the SFMM property, Sect. 2.2):
    the total force of B on A equals minus that of A on B."""
    rng = np.random.default_rng(40 + p)
    xA = rng.uniform(-0.2, 0.2, (9, 3))
    mA = rng.uniform(0.5, 1.5, 9)
    xB = rng.uniform(-0.2, 0.2, (11, 3)) + np.array([1.5, -0.4, 0.6])
    mB = rng.uniform(0.5, 1.5, 11)
    sA = (mA[:, None] * xA).sum(0) / mA.sum()
    sB = (mB[:, None] * xB).sum(0) / mB.sum()
    aA, _ = oracle.m2l_eval(p, sA, sB, xB, mB, xA)
    aB, _ = oracle.m2l_eval(p, sB, sA, xA, mA, xB)
    FA = (mA[:, None] * aA).sum(0)
    FB = (mB[:, None] * aB).sum(0)
    np.testing.assert_allclose(FA, -FB, rtol=1e-12, atol=1e-14 * np.abs(FA).max())


def test_dipole_about_centre_of_mass_vanishes_to_rounding():
    """The FP32 form leaves the dipole term out of its M2L because moments
    are taken about each node's centre of mass (Eq. massmom with s the
    centre of mass), where Q_1 = sum m (x - s) = 0.  In FP64 the oracle's
    directly summed dipoles are at rounding level: at most a few n eps of
    M max|x| for a node of n particles."""
    import workloads

    eps = np.finfo(float).eps
    for gen in (workloads.plummer, workloads.uniform_sphere, workloads.binary_polytrope):
        pos, m, h = gen(20000, 5)
        t = oracle.Tree(pos, m, h, 8, p=2)
        q1 = np.abs(t.Q[:, oracle.rank_offset(1):oracle.rank_offset(2)]).max(axis=1)
        xmax = np.abs(pos).max()
        assert np.all(q1 <= 4 * t.count * eps * t.mass * xmax), q1.max()
