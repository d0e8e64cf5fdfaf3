"""Parity at the full benchmark sizes, in the launch configuration the
benchmark times (needs a GB300; marked gpu).

The GPU solves the whole system; the oracle builds the same tree on the host
and runs Algorithms 1-2 for a seeded sample of leaves only (every leaf's
result depends on the read-only tree alone, so sampled leaves are exact).
Sampled particles are compared element by element; the momentum residual is
checked over all particles (it holds at any size).
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import (TOL_FP32_MAX, TOL_FP32_RMS, TOL_FP64, TOL_MOM_FP32, TOL_MOM_FP64, acc_rel, momentum_residual,
                         pot_rel, solver)

pytestmark = pytest.mark.gpu

_CACHE = {}


def _system(name):
    if name not in _CACHE:
        _CACHE.clear()
        pos, m, h = workloads.make(name)
        w = workloads.WORKLOADS[name]
        t = oracle.Tree(pos, m, h, w["leaf_size"], p=2)
        _CACHE[name] = (pos, m, h, w, t)
    return _CACHE[name]


def _sample(t, k, seed):
    """k seeded leaves plus the first and the last leaf of the tree."""
    rng = np.random.default_rng(seed)
    sel = rng.choice(t.nleaves, size=min(k, t.nleaves), replace=False)
    return np.unique(np.concatenate([sel, [0, t.nleaves - 1]])).astype(np.int32)


def _sampled_particles(t, sel):
    return np.concatenate([t.perm[t.first[L]:t.first[L] + t.count[L]] for L in t.leaves[sel]])


def test_full_size_tree_leaves_match_oracle():
    """The GPU tree of the 10^6 Plummer sphere has the oracle's leaves."""
    pos, m, h, w, t = _system("plummer_1e6")
    s = solver("fp32")
    s.build(pos, m, h, w["leaf_size"])
    g = s.tree()
    s.close()
    np.testing.assert_array_equal(g["perm"], t.perm)
    np.testing.assert_array_equal(g["first"][g["leaves"]], t.first[t.leaves])
    np.testing.assert_array_equal(g["count"][g["leaves"]], t.count[t.leaves])


@pytest.mark.parametrize("name,prec,theta", [
    ("plummer_1e6", "fp32", 0.5),
    ("plummer_1e6", "fp64", 0.5),
    ("plummer_1e6", "fp32", 0.3),
    ("plummer_1e6", "fp64", 0.3),
    ("plummer_1e6", "fp32", 0.7),
    ("plummer_1e6", "fp64", 0.7),
    ("binary_polytrope_2e6", "fp32", 0.5),
    ("binary_polytrope_2e6", "fp64", 0.5),
    ("clustered_1.6e7", "fp32", 0.5),
])
def test_full_size_sampled_leaves_match_oracle(name, prec, theta):
    pos, m, h, w, t = _system(name)
    s = solver(prec)  # the library's defaults, as the benchmark runs it
    s.build(pos, m, h, w["leaf_size"])
    acc, pot = s.gravity(theta, 2)
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    s.close()

    res = momentum_residual(m, acc)
    assert res <= (TOL_MOM_FP64 if prec == "fp64" else TOL_MOM_FP32), res

    sel = _sample(t, 96 if theta >= 0.5 else 48, seed=len(name) + int(100 * theta))
    a_o, p_o, _ = t.sfmm(theta, leaf_sample=sel)
    idx = _sampled_particles(t, sel)
    assert len(idx) > 0
    e = acc_rel(acc[idx], a_o[idx])
    ep = pot_rel(pot[idx], p_o[idx])
    print("%s %s theta %.1f: acc rel rms %.3e max %.3e, pot rel rms %.3e max %.3e, momentum %.3e (%d particles)"
          % (name, prec, theta, math.sqrt((e**2).mean()), e.max(), math.sqrt((ep**2).mean()), ep.max(), res,
             len(idx)))
    if prec == "fp64":
        assert e.max() <= TOL_FP64, e.max()
        assert ep.max() <= TOL_FP64, ep.max()
    else:
        assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS, math.sqrt((e**2).mean())
        assert math.sqrt((ep**2).mean()) <= TOL_FP32_RMS, math.sqrt((ep**2).mean())
        assert e.max() <= TOL_FP32_MAX, e.max()


def test_uniform_sphere_1e4_fp64_matches_oracle_and_direct():
    """The small configuration (uniform sphere, N = 10^4, theta 0.5, leaf 10,
    FP64 form): every particle against the full oracle to 1e-10, the same
    interaction counts, and the same error against the softened direct sum
    as the oracle's own (the truncation error of the method, stated)."""
    name = "uniform_1e4"
    pos, m, h = workloads.make(name)
    w = workloads.WORKLOADS[name]
    a_o, p_o, st_o = oracle.sfmm(pos, m, h, theta=w["theta"], p=2, leaf_size=w["leaf_size"])
    a_d, p_d = oracle.direct(pos, m, h)
    for prec in ("fp64", "fp32"):
        s = solver(prec)
        s.build(pos, m, h, w["leaf_size"])
        acc, pot = s.gravity(w["theta"], 2)
        acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
        st = s.stats()
        s.close()
        assert st["m2l"] == st_o["m2l"] and st["p2p_pairs"] == st_o["p2p_pairs"]
        e = acc_rel(acc, a_o)
        ep = pot_rel(pot, p_o)
        an = np.linalg.norm(a_d, axis=1)
        ed = np.linalg.norm(acc - a_d, axis=1) / an
        ed_o = np.linalg.norm(a_o - a_d, axis=1) / an
        print("uniform 1e4 %s: vs oracle acc max %.3e rms %.3e, pot max %.3e; vs direct mean %.3e max %.3e "
              "(oracle: mean %.3e max %.3e)" % (prec, e.max(), math.sqrt((e**2).mean()), ep.max(), ed.mean(),
                                                ed.max(), ed_o.mean(), ed_o.max()))
        if prec == "fp64":
            assert e.max() <= TOL_FP64 and ep.max() <= TOL_FP64
            assert abs(ed.mean() - ed_o.mean()) <= 1e-8 * ed_o.mean()
            assert momentum_residual(m, acc) <= TOL_MOM_FP64
        else:
            assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS and e.max() <= TOL_FP32_MAX
            assert abs(ed.mean() - ed_o.mean()) <= 1e-3 * ed_o.mean()
            assert momentum_residual(m, acc) <= TOL_MOM_FP32
        # the method's own truncation error at theta 0.5, p 2 (homogeneous
        # sphere: the paper's Sect. 4.1 finds errors well below the Plummer
        # sphere's); a loose sanity bound, the value is printed above
        assert ed.mean() < 3e-3


@pytest.mark.parametrize("name", ["plummer_1e6", "clustered_1.6e7"])
def test_full_size_schedules_agree_bitwise(name):
    """One launch per depth and both readiness queues give bitwise the same
    result at full size (the automatic choice takes the queue of nodes for
    the first tree and the queue of sibling pairs for the second)."""
    pos, m, h, w, t = _system(name)
    out = []
    for sched in (1, 2, 3):
        s = solver("fp32", walk=1, schedule=sched)
        s.build(pos, m, h, w["leaf_size"])
        acc, pot = s.gravity(w["theta"], 2)
        out.append((acc.cpu().numpy(), pot.cpu().numpy(), s.stats()["m2l"]))
        s.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
