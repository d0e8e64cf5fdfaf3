"""Pins of the oracle's tree and SFMM walk (CPU only).

Tree: Morton keys and the split rule recomputed by brute force in Python
integers, leaf partition, pre-order layout, node centre / size / h_max /
moments recomputed by hand.  SFMM: theta = 0 reduces to the direct sum,
every particle pair is covered exactly once, the interaction set is
symmetric and equals the one of an independent recursive dual-tree walk,
momentum is conserved to round-off, and the error falls with theta and p.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads


def brute_key(x, mn, scale):
    k = [min(2**21 - 1, int(np.floor((x[c] - mn[c]) * scale))) for c in range(3)]
    key = 0
    for b in range(21):
        key |= ((k[0] >> b) & 1) << (3 * b + 2)
        key |= ((k[1] >> b) & 1) << (3 * b + 1)
        key |= ((k[2] >> b) & 1) << (3 * b)
    return key


@pytest.fixture(scope="module", params=[("uniform", 3000, 10), ("plummer", 4000, 16), ("plummer", 2500, 1),
                                        ("uniform", 1200, 64)])
def tree(request):
    kind, n, ls = request.param
    gen = workloads.uniform_sphere if kind == "uniform" else workloads.plummer
    pos, m, h = gen(n, 77)
    return oracle.Tree(pos, m, h, ls, p=2), pos, m, h, ls


def test_keys_and_sort(tree):
    t, pos, m, h, ls = tree
    mn = pos.min(0)
    E = (pos.max(0) - mn).max()
    scale = 2**21 / E
    assert t.bbox[4] == scale
    for i in range(0, t.n, max(1, t.n // 300)):
        j = t.perm[i]
        assert int(t.keys[i]) == brute_key(pos[j], mn, scale)
    aug = [(int(k), int(p)) for k, p in zip(t.keys, t.perm)]
    assert aug == sorted(aug)
    assert sorted(t.perm.tolist()) == list(range(t.n))


def test_partition_and_split_rule(tree):
    t, pos, m, h, ls = tree
    aug = [(int(k) << 32) | i for i, k in enumerate(t.keys)]
    covered = np.zeros(t.n, int)
    for v in range(t.nnodes):
        f, c = t.first[v], t.count[v]
        if t.left[v] < 0:
            assert 1 <= c <= ls
            covered[f:f + c] += 1
            continue
        assert c > ls
        L, R = t.left[v], t.right[v]
        assert L == v + 1                       # pre-order layout
        assert t.first[L] == f and t.first[R] == f + t.count[L]
        assert t.count[L] + t.count[R] == c
        assert t.parent[L] == v and t.parent[R] == v
        assert t.depth[L] == t.depth[v] + 1
        # split at the highest differing bit of the augmented keys
        b = (aug[f] ^ aug[f + c - 1]).bit_length() - 1
        split = next(i for i in range(f, f + c) if (aug[i] >> b) & 1)
        assert t.first[R] == split
    assert (covered == 1).all()
    order = sorted(range(t.nnodes), key=lambda v: (t.first[v], t.depth[v]))
    assert order == list(range(t.nnodes))
    assert (np.diff(t.first[t.leaves]) > 0).all()


def test_node_properties_brute_force(tree):
    t, pos, m, h, ls = tree
    xs, ms, hs = pos[t.perm], m[t.perm], h[t.perm]
    for v in list(range(0, t.nnodes, max(1, t.nnodes // 60))) + [0]:
        f, c = t.first[v], t.count[v]
        x, mm = xs[f:f + c], ms[f:f + c]
        M = mm.sum()
        s = (mm[:, None] * x).sum(0) / M
        np.testing.assert_allclose(t.centre[v], s, rtol=1e-13, atol=1e-15)
        assert t.mass[v] == pytest.approx(M, rel=1e-13)
        assert t.size[v] == pytest.approx(np.linalg.norm(x - t.centre[v], axis=1).max(), rel=1e-14)
        assert t.hmax[v] == hs[f:f + c].max()
        Q = oracle.p2m(2, x, mm, t.centre[v])
        np.testing.assert_allclose(t.Q[v], Q, rtol=1e-12, atol=1e-13 * np.abs(Q).max())


@pytest.mark.parametrize("kind,n,ls,p", [("uniform", 1500, 10, 2), ("plummer", 2000, 16, 0),
                                         ("plummer", 1000, 1, 4), ("uniform", 800, 64, 3)])
def test_theta_zero_equals_direct(kind, n, ls, p):
    gen = workloads.uniform_sphere if kind == "uniform" else workloads.plummer
    pos, m, h = gen(n, 5)
    acc_d, pot_d = oracle.direct(pos, m, h)
    acc, pot, st = oracle.sfmm(pos, m, h, theta=0.0, p=p, leaf_size=ls)
    assert st["m2l"] == 0
    assert st["p2p_pairs"] == n * (n - 1)
    np.testing.assert_allclose(acc, acc_d, rtol=0, atol=1e-14 * np.abs(acc_d).max())
    np.testing.assert_allclose(pot, pot_d, rtol=1e-14)


def _leaf_of(t):
    lid = np.empty(t.n, np.int64)
    for q, v in enumerate(t.leaves):
        lid[t.first[v]:t.first[v] + t.count[v]] = q
    return lid


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.8])
def test_walk_covers_every_pair_once_and_is_symmetric(tree, theta):
    t = tree[0]
    mo, lv, src, po, ps = t.lists(theta)
    nl = t.nleaves
    directed = {}
    for q in range(nl):
        L = t.leaves[q]
        cover = np.zeros(t.n, int)
        chain = []
        v = L
        while v >= 0:
            chain.append(v)
            v = t.parent[v]
        chain = chain[::-1]
        for e in range(mo[q], mo[q + 1]):
            A, B = chain[lv[e]], src[e]
            cover[t.first[B]:t.first[B] + t.count[B]] += 1
            directed[(A, B)] = directed.get((A, B), 0) + 1
        for e in range(po[q], po[q + 1]):
            S = ps[e]
            assert t.left[S] < 0
            cover[t.first[S]:t.first[S] + t.count[S]] += 1
        assert (cover == 1).all(), "every source particle exactly once per leaf"
    # an (A,B) entry appears once for each leaf under A, and (B,A) exists
    nleaves_under = {}
    for v in range(t.nnodes - 1, -1, -1):
        nleaves_under[v] = 1 if t.left[v] < 0 else nleaves_under[t.left[v]] + nleaves_under[t.right[v]]
    for (A, B), cnt in directed.items():
        assert cnt == nleaves_under[A]
        assert (B, A) in directed
    p2p = {(t.leaves[q], ps[e]) for q in range(nl) for e in range(po[q], po[q + 1])}
    for (L, S) in p2p:
        assert (S, L) in p2p


def _recursive_pairs(t, theta):
    """Independent serial dual-tree walk from (root, root): the directed
    pair set that the replay of Algorithms 1-2 must reproduce."""
    m2l, p2p = set(), set()
    leaf = lambda v: t.left[v] < 0
    kids = lambda v: (t.left[v], t.right[v])
    stack = [(0, 0)]
    while stack:
        A, B = stack.pop()
        if A != B and t.accept(A, B, theta):
            m2l.add((A, B))
            continue
        if leaf(A) and leaf(B):
            p2p.add((A, B))
        elif leaf(B):
            stack += [(a, B) for a in kids(A)]
        elif leaf(A):
            stack += [(A, b) for b in kids(B)]
        else:
            stack += [(a, b) for a in kids(A) for b in kids(B)]
    return m2l, p2p


@pytest.mark.parametrize("theta", [0.4, 0.7])
def test_replay_equals_recursive_dual_walk(tree, theta):
    t = tree[0]
    mo, lv, src, po, ps = t.lists(theta)
    m2l, p2p = set(), set()
    for q in range(t.nleaves):
        chain = []
        v = t.leaves[q]
        while v >= 0:
            chain.append(v)
            v = t.parent[v]
        chain = chain[::-1]
        for e in range(mo[q], mo[q + 1]):
            m2l.add((chain[lv[e]], src[e]))
        for e in range(po[q], po[q + 1]):
            p2p.add((t.leaves[q], ps[e]))
    rm, rp = _recursive_pairs(t, theta)
    assert m2l == rm
    assert p2p == rp


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("theta", [0.3, 0.6, 0.9])
def test_momentum_conserved_to_roundoff(p, theta):
    pos, m, h = workloads.plummer(3000, 31)
    m = m * np.random.default_rng(2).uniform(0.5, 1.5, len(m))
    acc, _, st = oracle.sfmm(pos, m, h, theta=theta, p=p, leaf_size=8)
    assert st["m2l"] > 0
    ma = m[:, None] * acc
    assert np.linalg.norm(ma.sum(0)) / np.abs(ma).sum() < 1e-14


def test_error_falls_with_theta_and_order():
    pos, m, h = workloads.plummer(4000, 8)
    acc_d, pot_d = oracle.direct(pos, m, h)
    an = np.linalg.norm(acc_d, axis=1)

    def err(theta, p):
        a, _, _ = oracle.sfmm(pos, m, h, theta=theta, p=p, leaf_size=8)
        return (np.linalg.norm(a - acc_d, axis=1) / an).mean()

    e = {(th, p): err(th, p) for th in (0.3, 0.5, 0.7) for p in (1, 2, 3)}
    for p in (1, 2, 3):
        assert e[(0.3, p)] < e[(0.5, p)] < e[(0.7, p)]
    for th in (0.3, 0.5, 0.7):
        assert e[(th, 3)] < e[(th, 2)] < e[(th, 1)]
    assert e[(0.5, 2)] < 1e-2


def test_leaf_sample_matches_full_run():
    pos, m, h = workloads.uniform_sphere(3000, 9)
    t = oracle.Tree(pos, m, h, 10, p=2)
    acc, pot, _ = t.sfmm(0.5)
    sel = np.array([0, 5, t.nleaves - 1, t.nleaves // 2])
    a2, p2, _ = t.sfmm(0.5, leaf_sample=sel)
    for q in sel:
        v = t.leaves[q]
        idx = t.perm[t.first[v]:t.first[v] + t.count[v]]
        np.testing.assert_array_equal(a2[idx], acc[idx])
        np.testing.assert_array_equal(p2[idx], pot[idx])


def test_duplicate_positions_and_tiny_systems():
    # coincident particles: equal keys, split on the sorted position
    pos = np.zeros((40, 3))
    pos[20:] = 1.0
    m = np.full(40, 1.0 / 40)
    h = np.full(40, 0.05)
    acc_d, pot_d = oracle.direct(pos, m, h)
    for theta in (0.0, 0.5):
        acc, pot, _ = oracle.sfmm(pos, m, h, theta=theta, p=2, leaf_size=4)
        np.testing.assert_allclose(acc, acc_d, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(pot, pot_d, rtol=1e-13)
    # a single particle: one leaf, no force, zero potential
    acc, pot, st = oracle.sfmm(np.zeros((1, 3)), np.ones(1), np.ones(1), 0.5, 2, 10)
    assert (acc == 0).all() and (pot == 0).all()
