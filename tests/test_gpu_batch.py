"""Batched ensemble (many independent systems in the same launches) against
the oracle run on each system alone (needs a GB300; marked gpu)."""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_FP32_RMS, TOL_FP64, TOL_MOM_FP64, acc_rel, momentum_residual, pot_rel, solver

pytestmark = pytest.mark.gpu


def _batch(seed=5):
    sizes = [700, 2500, 31, 1, 4000, 1200, 17, 3333]
    gens = [workloads.plummer, workloads.uniform_sphere]
    ps, ms, hs = [], [], []
    for s, n in enumerate(sizes):
        p, m, h = gens[s % 2](n, seed * 100 + s)
        p = p + np.array([100.0 * s, 0.0, 0.0])  # far apart: must still not interact
        ps.append(p)
        ms.append(m)
        hs.append(h)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lsz = np.array([8, 16, 32, 64, 16, 10, 4, 1], np.int32)
    return ps, ms, hs, off, lsz


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("walk", [0, 1, 3, 4])
def test_batch_matches_oracle_per_system(prec, walk):
    ps, ms, hs, off, lsz = _batch()
    s = solver(prec, walk=walk)
    s.build_batch(off, np.concatenate(ps), np.concatenate(ms), np.concatenate(hs), lsz)
    acc, pot = s.gravity(0.5, 2)
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    st = s.stats()
    tot = {"m2l": 0, "m2l_unique": 0, "p2p_pairs": 0}
    sums = s.batch_sums()
    for k in range(len(ps)):
        a_o, p_o, st_o = oracle.sfmm(ps[k], ms[k], hs[k], theta=0.5, p=2, leaf_size=int(lsz[k]))
        for key in tot:
            tot[key] += st_o[key]
        a, p = acc[off[k]:off[k + 1]], pot[off[k]:off[k + 1]]
        if len(ms[k]) == 1:
            assert np.all(a == 0) and np.all(p == 0)
            continue
        e = acc_rel(a, a_o)
        if prec == "fp64":
            assert e.max() <= TOL_FP64, (k, e.max())
            assert pot_rel(p, p_o).max() <= TOL_FP64
            assert momentum_residual(ms[k], a) <= TOL_MOM_FP64
        else:
            assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS, (k, math.sqrt((e**2).mean()))
        ma = ms[k][:, None] * a
        np.testing.assert_allclose(sums[k, :3], ma.sum(0), rtol=0, atol=1e-10 * np.abs(ma).sum())
        np.testing.assert_allclose(sums[k, 3], np.abs(ma).sum(), rtol=1e-10)
        np.testing.assert_allclose(sums[k, 4], 0.5 * (ms[k] * p).sum(), rtol=1e-10)
    for key in tot:
        assert st[key] == tot[key], key


def test_batch_tree_partitions_each_system_like_its_own_build():
    ps, ms, hs, off, lsz = _batch(seed=9)
    s = solver("fp64")
    s.build_batch(off, np.concatenate(ps), np.concatenate(ms), np.concatenate(hs), lsz)
    g = s.tree()
    leaves = g["leaves"]
    lf, lc = g["first"][leaves], g["count"][leaves]
    for k in range(len(ps)):
        t = oracle.Tree(ps[k], ms[k], hs[k], int(lsz[k]), p=0)
        sel = (lf >= off[k]) & (lf < off[k + 1])
        assert np.all(lf[sel] + lc[sel] <= off[k + 1])
        np.testing.assert_array_equal(lf[sel] - off[k], t.first[t.leaves])
        np.testing.assert_array_equal(lc[sel], t.count[t.leaves])
        np.testing.assert_array_equal(g["perm"][off[k]:off[k + 1]] - off[k], t.perm)


def test_batch_of_one_equals_single_build():
    pos, m, h = workloads.plummer(6000, 3)
    s1 = solver("fp32")
    s1.build(pos, m, h, 16)
    a1, p1 = s1.gravity(0.5, 2)
    s2 = solver("fp32")
    s2.build_batch(np.array([0, 6000]), pos, m, h, np.array([16], np.int32))
    a2, p2 = s2.gravity(0.5, 2)
    np.testing.assert_array_equal(a1.cpu().numpy(), a2.cpu().numpy())
    np.testing.assert_array_equal(p1.cpu().numpy(), p2.cpu().numpy())


def test_batch_rejects_bad_offsets():
    from paper_2602_05804_gb300 import sfmm

    pos, m, h = workloads.uniform_sphere(100, 1)
    s = solver("fp32")
    for off in ([1, 100], [0, 50, 50, 100], [0, 60, 40, 100]):
        with pytest.raises(sfmm.SFMMError) as e:
            s.build_batch(np.array(off), pos, m, h)
        assert e.value.code == sfmm.SFMM_EINVAL


def _ensemble(nsys=16, seed=11):
    rng = np.random.default_rng(seed)
    sizes = np.floor(10 ** rng.uniform(2.7, 3.9, nsys)).astype(np.int64)
    gens = [workloads.plummer, workloads.uniform_sphere]
    ps, ms, hs = [], [], []
    for s, n in enumerate(sizes):
        p, m, h = gens[s % 2](int(n), seed * 1000 + s)
        ps.append(p)
        ms.append(m)
        hs.append(h)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return ps, ms, hs, off


def test_autotuned_batch_and_null_leaf_sizes(tmp_path):
    """sfmm_autotune_batch picks leaf sizes in {8, 16, 32, 64} and launch
    knobs from timed trials and caches them; a fresh context loading the
    cache builds with NULL leaf sizes exactly the tree the explicit sizes
    give, and the per-system results match the oracle."""
    import json

    from paper_2602_05804_gb300 import sfmm

    ps, ms, hs, off = _ensemble()
    pos, m, h = np.concatenate(ps), np.concatenate(ms), np.concatenate(hs)
    cache = str(tmp_path / "tune.json")
    s = solver("fp32")
    sfmm.sfmm_autotune_cache(s.ctx, cache)
    leaf = s.autotune_batch(off, pos, m, h, 0.5, 2)
    assert set(leaf.tolist()) <= {8, 16, 32, 64}
    acc1, pot1 = s.gravity(0.5, 2)
    s.close()
    table = json.load(open(cache))
    assert len(table["leaf"]) >= 2 and len(table["knobs"]) == 1
    assert all(e["leaf_size"] in (8, 16, 32, 64) for e in table["leaf"])
    # the two profiles fall in different classes
    assert {e["key"].split("|")[1] for e in table["leaf"]} == {"c0", "c2"}

    s2 = solver("fp32")
    sfmm.sfmm_autotune_cache(s2.ctx, cache)
    s2.set_option("autotune_theta", 0.5)
    s2.build_batch(off, pos, m, h, None)  # NULL: the cached table
    g2 = s2.tree()
    acc2, pot2 = s2.gravity(0.5, 2)
    s3 = solver("fp32")
    s3.build_batch(off, pos, m, h, leaf)  # explicit sizes
    g3 = s3.tree()
    for k in ("first", "count", "right"):
        np.testing.assert_array_equal(g2[k], g3[k])
    assert json.load(open(cache)) == table  # nothing new was timed
    a2 = acc2.cpu().numpy()
    np.testing.assert_array_equal(a2, acc1.cpu().numpy())
    for k in (0, 1, len(ps) - 1):
        a_o, _, _ = oracle.sfmm(ps[k], ms[k], hs[k], theta=0.5, p=2, leaf_size=int(leaf[k]))
        e = acc_rel(a2[off[k]:off[k + 1]], a_o)
        assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS


def test_null_leaf_sizes_without_cache_run_trials():
    """With no table at all, NULL leaf sizes run the leaf-size trials inline."""
    ps, ms, hs, off = _ensemble(nsys=6, seed=12)
    s = solver("fp64")
    s.build_batch(off, np.concatenate(ps), np.concatenate(ms), np.concatenate(hs), None)
    acc, _ = s.gravity(0.5, 2)
    acc = acc.cpu().numpy()
    g = s.tree()
    leaves = g["leaves"]
    assert g["count"][leaves].max() <= 64
    for k in (0, 3):
        a_o, _, _ = oracle.sfmm(ps[k], ms[k], hs[k], theta=0.5, p=2, leaf_size=16)
        # leaf sizes may differ from 16: compare against the direct sum's scale instead
        e = acc_rel(acc[off[k]:off[k + 1]], a_o)
        assert np.median(e) < 1e-2
