"""Centre-of-mass-pivot kd tree on the GPU (option tree = 1) against the
oracle's kd tree, and the SFMM over it (needs a GB300; marked gpu)."""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_FP32_RMS, TOL_FP64, TOL_MOM_FP64, acc_rel, momentum_residual, pot_rel, solver

pytestmark = pytest.mark.gpu


def _set(kind, n, seed):
    return {"uniform": workloads.uniform_sphere, "plummer": workloads.plummer,
            "binary": workloads.binary_polytrope}[kind](n, seed)


CASES = [("uniform", 4000, 10), ("plummer", 5003, 16), ("plummer", 3001, 1), ("binary", 2999, 64),
         ("uniform", 777, 8), ("plummer", 40000, 16)]


@pytest.mark.parametrize("kind,n,ls", CASES)
def test_kd_tree_matches_oracle(kind, n, ls):
    pos, m, h = _set(kind, n, 22)
    t = oracle.Tree(pos, m, h, ls, p=2, tree="kd")
    s = solver("fp64", tree=1)
    s.build(pos, m, h, ls)
    g = s.tree()
    assert g["first"].shape[0] == t.nnodes
    np.testing.assert_array_equal(g["perm"], t.perm)
    np.testing.assert_array_equal(g["first"], t.first)
    np.testing.assert_array_equal(g["count"], t.count)
    np.testing.assert_array_equal(g["right"], t.right)
    np.testing.assert_array_equal(g["parent"], t.parent)
    np.testing.assert_array_equal(g["depth"], t.depth)
    np.testing.assert_array_equal(g["leaves"], t.leaves)
    np.testing.assert_array_equal(g["hmax"], t.hmax)
    scale = np.abs(pos).max()
    np.testing.assert_allclose(g["centre"], t.centre, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(g["size"], t.size, rtol=0, atol=2e-12 * scale)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("walk", [0, 1, 3, 4])
@pytest.mark.parametrize("theta", [0.3, 0.6])
def test_sfmm_on_kd_tree_matches_oracle(prec, walk, theta):
    pos, m, h = workloads.plummer(6000, 23)
    acc_o, pot_o, st_o = oracle.sfmm(pos, m, h, theta=theta, p=2, leaf_size=16, tree="kd")
    s = solver(prec, walk=walk, tree=1)
    s.build(pos, m, h, 16)
    acc, pot = s.gravity(theta, 2)
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    st = s.stats()
    for k in ("m2l", "m2l_unique", "p2p_pairs", "p2p_leaves"):
        assert st[k] == st_o[k], k
    e = acc_rel(acc, acc_o)
    if prec == "fp64":
        assert e.max() <= TOL_FP64
        assert pot_rel(pot, pot_o).max() <= TOL_FP64
        assert momentum_residual(m, acc) <= TOL_MOM_FP64
    else:
        assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS


def test_kd_degenerate_pivots_split_in_the_middle():
    pos = np.zeros((60, 3))
    pos[30:, 1] = 2.0
    m = np.full(60, 1.0 / 60)
    h = np.full(60, 0.05)
    t = oracle.Tree(pos, m, h, 4, p=2, tree="kd")
    s = solver("fp64", tree=1)
    s.build(pos, m, h, 4)
    g = s.tree()
    np.testing.assert_array_equal(g["perm"], t.perm)
    np.testing.assert_array_equal(g["first"], t.first)
    np.testing.assert_array_equal(g["count"], t.count)
    acc, pot = s.gravity(0.5, 2)
    acc_d, pot_d = oracle.direct(pos, m, h)
    np.testing.assert_allclose(acc.cpu().numpy(), acc_d, rtol=1e-12, atol=1e-14)


def test_kd_tree_is_refused_for_batches():
    from paper_2602_05804_gb300 import sfmm

    pos, m, h = workloads.uniform_sphere(200, 1)
    s = solver("fp32", tree=1)
    with pytest.raises(sfmm.SFMMError) as e:
        s.build_batch(np.array([0, 100, 200]), pos, m, h)
    assert e.value.code == sfmm.SFMM_ENOTIMPL


def test_kd_full_size_sampled_leaves():
    """Plummer 10^6 on the kd tree, FP32 form: sampled leaves against the
    oracle's kd tree and walk."""
    w = workloads.WORKLOADS["plummer_1e6"]
    pos, m, h = workloads.make("plummer_1e6")
    t = oracle.Tree(pos, m, h, 16, p=2, tree="kd")
    s = solver("fp32", tree=1)
    s.build(pos, m, h, 16)
    g = s.tree()
    np.testing.assert_array_equal(g["perm"], t.perm)
    np.testing.assert_array_equal(g["count"][g["leaves"]], t.count[t.leaves])
    acc, pot = s.gravity(w["theta"], 2)
    acc = acc.cpu().numpy()
    sel = np.random.default_rng(9).choice(t.nleaves, 96, replace=False).astype(np.int32)
    a_o, _, _ = t.sfmm(w["theta"], leaf_sample=sel)
    idx = np.concatenate([t.perm[t.first[L]:t.first[L] + t.count[L]] for L in t.leaves[sel]])
    e = acc_rel(acc[idx], a_o[idx])
    assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS
