"""Pins of the oracle's centre-of-mass-pivot kd tree (Sect. 3) and of the
SFMM walk over it (CPU only).

Tree: every internal node's children split its particles along the axis of
largest extent at the node's centre of mass (recomputed here with an
exactly rounded sum), each child keeps a contiguous range, leaves hold at
most leaf_size particles and internal nodes more, the layout is pre-order.
SFMM over the kd tree: theta = 0 reduces to the direct sum, every particle
pair is covered once per leaf and the pair set equals that of an
independent recursive dual-tree walk, momentum is conserved to round-off.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from test_oracle_tree_sfmm import _recursive_pairs


@pytest.fixture(scope="module", params=[("uniform", 3000, 10), ("plummer", 4000, 16), ("plummer", 700, 1),
                                        ("uniform", 1200, 64)])
def kd(request):
    kind, n, ls = request.param
    gen = workloads.uniform_sphere if kind == "uniform" else workloads.plummer
    pos, m, h = gen(n, 78)
    m = m * np.random.default_rng(4).uniform(0.5, 1.5, n)  # unequal masses: the pivot is not the mean
    return oracle.Tree(pos, m, h, ls, p=2, tree="kd"), pos, m, h, ls


def test_layout_partition_and_leaf_sizes(kd):
    t, pos, m, h, ls = kd
    assert sorted(t.perm.tolist()) == list(range(t.n))
    assert t.first[0] == 0 and t.count[0] == t.n
    for v in range(t.nnodes):
        if t.left[v] < 0:
            assert 1 <= t.count[v] <= ls
            continue
        assert t.count[v] > ls
        L, R = t.left[v], t.right[v]
        assert L == v + 1  # pre-order
        assert t.parent[L] == v and t.parent[R] == v
        assert t.first[L] == t.first[v] and t.first[R] == t.first[v] + t.count[L]
        assert t.count[L] + t.count[R] == t.count[v]
        assert t.count[L] >= 1 and t.count[R] >= 1
    leaves = np.sort(t.first[t.leaves])
    assert np.array_equal(t.first[t.leaves], leaves)  # leaves in pre-order = range order


def test_split_rule_centre_of_mass_pivot(kd):
    """Left child: coordinate below the pivot on the widest axis; right: the
    rest.  The pivot is recomputed with math.fsum (exact sums), so only
    particles within rounding of it may be classified either way."""
    t, pos, m, h, ls = kd
    xs, ms = pos[t.perm], m[t.perm]
    checked = 0
    for v in range(t.nnodes):
        if t.left[v] < 0:
            continue
        f, c = t.first[v], t.count[v]
        x, mm = xs[f:f + c], ms[f:f + c]
        ext = x.max(0) - x.min(0)
        axis = int(np.argmax(ext))  # first maximum: ties go to the lowest axis
        M = math.fsum(mm)
        piv = math.fsum(mm * x[:, axis]) / M
        nl = t.count[t.left[v]]
        below = x[:, axis] < piv
        tol = 1e-12 * (abs(piv) + ext[axis])
        near = np.abs(x[:, axis] - piv) <= tol
        if below.sum() in (0, c):  # degenerate pivot: middle split
            assert nl == c // 2
            continue
        left = np.zeros(c, bool)
        left[:nl] = True
        assert np.all(left[~near] == below[~near]), v
        checked += 1
    assert checked > 10


def test_degenerate_pivot_splits_in_the_middle():
    pos = np.zeros((40, 3))
    pos[:, 0] = 1.0  # all particles at one point
    m = np.full(40, 0.025)
    h = np.full(40, 0.1)
    t = oracle.Tree(pos, m, h, 4, p=0, tree="kd")
    for v in range(t.nnodes):
        if t.left[v] >= 0:
            assert t.count[t.left[v]] == t.count[v] // 2
    assert np.array_equal(t.perm, np.arange(40))


def test_theta_zero_equals_direct_on_kd_tree():
    pos, m, h = workloads.plummer(1500, 6)
    acc_d, pot_d = oracle.direct(pos, m, h)
    acc, pot, st = oracle.sfmm(pos, m, h, theta=0.0, p=2, leaf_size=10, tree="kd")
    assert st["m2l"] == 0 and st["p2p_pairs"] == 1500 * 1499
    np.testing.assert_allclose(acc, acc_d, rtol=0, atol=1e-14 * np.abs(acc_d).max())
    np.testing.assert_allclose(pot, pot_d, rtol=1e-14)


@pytest.mark.parametrize("theta", [0.4, 0.7])
def test_kd_walk_equals_recursive_dual_walk(kd, theta):
    t = kd[0]
    mo, lv, src, po, ps = t.lists(theta)
    m2l, p2p = set(), set()
    for q in range(t.nleaves):
        chain = []
        v = t.leaves[q]
        while v >= 0:
            chain.append(v)
            v = t.parent[v]
        chain = chain[::-1]
        cover = np.zeros(t.n, int)
        for e in range(mo[q], mo[q + 1]):
            m2l.add((chain[lv[e]], src[e]))
            B = src[e]
            cover[t.first[B]:t.first[B] + t.count[B]] += 1
        for e in range(po[q], po[q + 1]):
            p2p.add((t.leaves[q], ps[e]))
            S = ps[e]
            cover[t.first[S]:t.first[S] + t.count[S]] += 1
        assert (cover == 1).all()
    rm, rp = _recursive_pairs(t, theta)
    assert m2l == rm and p2p == rp


@pytest.mark.parametrize("p", [0, 2, 4])
def test_momentum_conserved_on_kd_tree(p):
    pos, m, h = workloads.plummer(3000, 32)
    acc, _, _ = oracle.sfmm(pos, m, h, theta=0.6, p=p, leaf_size=8, tree="kd")
    ma = m[:, None] * acc
    assert np.linalg.norm(ma.sum(0)) / np.abs(ma).sum() <= 1e-14
