"""Build + gravity captured as one CUDA graph per shape class
(sfmm_solve_graph; needs a GB300; marked gpu).

The replayed graph must give bitwise the results of the ordinary calls
(sfmm_build_batch + sfmm_gravity_batch) on the same inputs, match the FP64
oracle within the forms' tolerances, follow particle values that change
between calls (its kernels read each rebuild's node and leaf counts on the
device), and be recaptured after anything that invalidates it.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_FP32_RMS, TOL_FP64, TOL_MOM_FP64, acc_rel, momentum_residual, pot_rel, solver

pytestmark = pytest.mark.gpu


def _dev(*arrays):
    import torch

    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _out(n):
    import torch

    return (torch.empty((n, 3), dtype=torch.float64, device="cuda"),
            torch.empty(n, dtype=torch.float64, device="cuda"))


def _ordinary(prec, off, pd, md, hd, leaf, theta=0.5, order=2):
    from paper_2602_05804_gb300 import sfmm

    s = solver(prec)
    n = int(off[-1])
    a, p = _out(n)
    sfmm.sfmm_build_batch(s.ctx, off, pd, md, hd, leaf)
    sfmm.sfmm_gravity_batch(s.ctx, theta, order, a, p)
    st = s.stats()
    s.close()
    return a.cpu().numpy(), p.cpu().numpy(), st


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replays_equal_ordinary_calls_and_oracle(prec):
    from paper_2602_05804_gb300 import sfmm

    pos, m, h = workloads.plummer(20_000, 81)
    n = len(m)
    off = np.array([0, n], np.int64)
    leaf = np.array([16], np.int32)
    pd, md, hd = _dev(pos, m, h)
    a0, p0, st0 = _ordinary(prec, off, pd, md, hd, leaf)
    s = solver(prec)
    a, p = _out(n)
    for call in range(3):
        a.fill_(float("nan"))
        sfmm.sfmm_solve_graph(s.ctx, off, pd, md, hd, leaf, 0.5, 2, a, p)
        np.testing.assert_array_equal(a.cpu().numpy(), a0)
        np.testing.assert_array_equal(p.cpu().numpy(), p0)
        st = s.stats()
        assert st["graph_replays"] == call
        for k in ("nnodes", "nleaves", "m2l", "m2l_unique", "p2p_pairs"):
            assert st[k] == st0[k], k
        assert st["momentum"] == st0["momentum"] and st["W"] == st0["W"]
    s.close()
    a_o, p_o, _ = oracle.sfmm(pos, m, h, theta=0.5, p=2, leaf_size=16)
    e = acc_rel(a0, a_o)
    if prec == "fp64":
        assert e.max() <= TOL_FP64 and pot_rel(p0, p_o).max() <= TOL_FP64
        assert momentum_residual(m, a0) <= TOL_MOM_FP64
    else:
        assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS


def test_graph_follows_particles_that_move():
    """The same buffers with new positions (a drift step): the replay builds
    the new tree (its node count differs) and equals the ordinary calls."""
    from paper_2602_05804_gb300 import sfmm

    pos, m, h = workloads.plummer(30_000, 82)
    n = len(m)
    off = np.array([0, n], np.int64)
    leaf = np.array([16], np.int32)
    pd, md, hd = _dev(pos, m, h)
    s = solver("fp32")
    a, p = _out(n)
    sfmm.sfmm_solve_graph(s.ctx, off, pd, md, hd, leaf, 0.5, 2, a, p)
    nodes = {s.stats()["nnodes"]}
    rng = np.random.default_rng(3)
    for step in range(3):
        pd.add_(pd.new_tensor(rng.normal(0.0, 0.05, (n, 3))))  # in place: same address
        sfmm.sfmm_solve_graph(s.ctx, off, pd, md, hd, leaf, 0.5, 2, a, p)
        st = s.stats()
        assert st["graph_replays"] == step + 1
        a0, p0, st0 = _ordinary("fp32", off, pd, md, hd, leaf)
        assert st["nnodes"] == st0["nnodes"] and st["p2p_pairs"] == st0["p2p_pairs"]
        np.testing.assert_array_equal(a.cpu().numpy(), a0)
        np.testing.assert_array_equal(p.cpu().numpy(), p0)
        nodes.add(st["nnodes"])
    assert len(nodes) > 1  # the trees really differed
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_batch_matches_oracle_per_system(prec):
    from paper_2602_05804_gb300 import sfmm

    sizes = [700, 2500, 31, 4000, 1200, 17, 3333]
    gens = [workloads.plummer, workloads.uniform_sphere]
    ps, ms, hs = [], [], []
    for k, nk in enumerate(sizes):
        pk, mk, hk = gens[k % 2](nk, 900 + k)
        ps.append(pk + np.array([50.0 * k, 0.0, 0.0]))
        ms.append(mk)
        hs.append(hk)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    leaf = np.array([8, 16, 32, 16, 10, 4, 16], np.int32)
    pd, md, hd = _dev(np.concatenate(ps), np.concatenate(ms), np.concatenate(hs))
    s = solver(prec)
    a, p = _out(int(off[-1]))
    for _ in range(2):
        sfmm.sfmm_solve_graph(s.ctx, off, pd, md, hd, leaf, 0.5, 2, a, p)
    assert s.stats()["graph_replays"] == 1
    sums = sfmm.sfmm_batch_sums(s.ctx, len(sizes))
    s.close()
    acc, pot = a.cpu().numpy(), p.cpu().numpy()
    for k in range(len(sizes)):
        a_o, p_o, _ = oracle.sfmm(ps[k], ms[k], hs[k], theta=0.5, p=2, leaf_size=int(leaf[k]))
        ak, pk = acc[off[k]:off[k + 1]], pot[off[k]:off[k + 1]]
        e = acc_rel(ak, a_o)
        if prec == "fp64":
            assert e.max() <= TOL_FP64 and pot_rel(pk, p_o).max() <= TOL_FP64, k
        else:
            assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS, k
        ma = ms[k][:, None] * ak
        np.testing.assert_allclose(sums[k, 3], np.abs(ma).sum(), rtol=1e-12)


def test_graph_is_recaptured_after_an_option_change():
    from paper_2602_05804_gb300 import sfmm

    pos, m, h = workloads.uniform_sphere(8000, 83)
    n = len(m)
    off = np.array([0, n], np.int64)
    pd, md, hd = _dev(pos, m, h)
    s = solver("fp32")
    a, p = _out(n)
    for _ in range(2):
        sfmm.sfmm_solve_graph(s.ctx, off, pd, md, hd, None, 0.5, 2, a, p)
    assert s.stats()["graph_replays"] == 1
    s.set_option("G", 2.0)  # invalidates the graph
    sfmm.sfmm_solve_graph(s.ctx, off, pd, md, hd, None, 0.5, 2, a, p)
    assert s.stats()["graph_replays"] == 1
    a2 = a.cpu().numpy()
    sfmm.sfmm_solve_graph(s.ctx, off, pd, md, hd, None, 0.5, 2, a, p)
    assert s.stats()["graph_replays"] == 2
    np.testing.assert_array_equal(a.cpu().numpy(), a2)
    s.close()


def test_graph_rejects_what_it_cannot_capture():
    from paper_2602_05804_gb300 import sfmm

    pos, m, h = workloads.uniform_sphere(500, 84)
    pd, md, hd = _dev(pos, m, h)
    a, p = _out(500)
    s = solver("fp32", tree=1)
    with pytest.raises(sfmm.SFMMError) as e:
        sfmm.sfmm_solve_graph(s.ctx, np.array([0, 500]), pd, md, hd, None, 0.5, 2, a, p)
    assert e.value.code == sfmm.SFMM_ENOTIMPL
    s.close()
    s = solver("fp32")
    with pytest.raises(sfmm.SFMMError) as e:
        sfmm.sfmm_solve_graph(s.ctx, np.array([0, 1]), pd, md, hd, None, 0.5, 2, a, p)
    assert e.value.code == sfmm.SFMM_EINVAL
    s.close()
