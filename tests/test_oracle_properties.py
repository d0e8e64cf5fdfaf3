"""Property tests of the oracle on random tiny systems (CPU only).

Exact invariants of the method as the oracle implements it:
- scaling every position and smoothing length by 2 scales every rounding
  step by a power of two, so accelerations come out exactly /4 and
  potentials exactly /2 (Morton keys or kd pivots, opening decisions, kernel
  pieces and expansions all unchanged);
- scaling every mass by 2 scales accelerations and potentials exactly by 2;
- permuting the input particles leaves the tree, and so every result,
  unchanged (distinct keys);
- theta = 0 is the direct sum (Algorithm 2 opens every pair), and linear
  momentum is conserved to round-off for any theta and order (Sect. 2).
"""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SETTINGS = settings(max_examples=60, deadline=None)


def _system(seed, n, spread):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1.0, 1.0, (n, 3)) * spread
    m = rng.uniform(0.5, 1.5, n) / n
    h = rng.uniform(0.05, 0.4, n) * spread
    return pos, m, h


systems = st.tuples(st.integers(0, 2**31 - 1), st.integers(2, 40), st.sampled_from([0.5, 1.0, 3.0]))
thetas = st.sampled_from([0.0, 0.3, 0.5, 0.8])
trees = st.sampled_from(["morton", "kd"])
orders = st.integers(0, 4)
leaf_sizes = st.integers(1, 8)


@SETTINGS
@given(systems, thetas, orders, leaf_sizes, trees)
def test_length_scaling_is_exact(sysargs, theta, p, ls, tree):
    pos, m, h = _system(*sysargs)
    a1, p1, _ = oracle.sfmm(pos, m, h, theta=theta, p=p, leaf_size=ls, tree=tree)
    a2, p2, _ = oracle.sfmm(2.0 * pos, m, 2.0 * h, theta=theta, p=p, leaf_size=ls, tree=tree)
    np.testing.assert_array_equal(a2, a1 / 4.0)
    np.testing.assert_array_equal(p2, p1 / 2.0)


@SETTINGS
@given(systems, thetas, orders, leaf_sizes, trees)
def test_mass_scaling_is_exact(sysargs, theta, p, ls, tree):
    pos, m, h = _system(*sysargs)
    a1, p1, _ = oracle.sfmm(pos, m, h, theta=theta, p=p, leaf_size=ls, tree=tree)
    a2, p2, _ = oracle.sfmm(pos, 2.0 * m, h, theta=theta, p=p, leaf_size=ls, tree=tree)
    np.testing.assert_array_equal(a2, 2.0 * a1)
    np.testing.assert_array_equal(p2, 2.0 * p1)


@SETTINGS
@given(systems, thetas, orders, leaf_sizes, st.integers(0, 2**31 - 1))
def test_input_order_does_not_matter(sysargs, theta, p, ls, pseed):
    pos, m, h = _system(*sysargs)
    perm = np.random.default_rng(pseed).permutation(len(m))
    a1, p1, _ = oracle.sfmm(pos, m, h, theta=theta, p=p, leaf_size=ls)
    a2, p2, _ = oracle.sfmm(pos[perm], m[perm], h[perm], theta=theta, p=p, leaf_size=ls)
    np.testing.assert_array_equal(a2, a1[perm])
    np.testing.assert_array_equal(p2, p1[perm])


@SETTINGS
@given(systems, orders, leaf_sizes)
def test_theta_zero_is_the_direct_sum(sysargs, p, ls):
    pos, m, h = _system(*sysargs)
    a, pot, st_ = oracle.sfmm(pos, m, h, theta=0.0, p=p, leaf_size=ls)
    ad, pd = oracle.direct(pos, m, h)
    n = len(m)
    assert st_["m2l"] == 0 and st_["p2p_pairs"] == n * (n - 1)
    np.testing.assert_allclose(a, ad, rtol=0, atol=1e-13 * np.abs(ad).max())
    np.testing.assert_allclose(pot, pd, rtol=1e-13)


@SETTINGS
@given(systems, thetas, orders, leaf_sizes, trees)
def test_momentum_is_conserved(sysargs, theta, p, ls, tree):
    pos, m, h = _system(*sysargs)
    a, _, _ = oracle.sfmm(pos, m, h, theta=theta, p=p, leaf_size=ls, tree=tree)
    ma = m[:, None] * a
    assert np.linalg.norm(ma.sum(0)) <= 1e-13 * np.abs(ma).sum()
