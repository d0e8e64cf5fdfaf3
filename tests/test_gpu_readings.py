"""Tests of the precision and reduction readings (needs a GB300; marked gpu).

- Compensated sums: the momentum sums the gravity call reports (and the
  allocation-free reduction) are Neumaier-compensated FP64 sums, so they
  equal the exactly rounded sum of the returned m a far below the error of a
  plain sum, even where the momentum cancels to 1e-18 of sum |m a|; the
  same-sign sums (sum |m a|, W) are plain FP64 sums, accurate to a few tens
  of eps of themselves.
- FP32 form, dipole term: moments are taken about each node's centre of mass,
  where the dipole vanishes; the FP32 M2L leaves it out.  At p = 1 (monopole
  and dipole only) the FP32 form still matches the oracle, which keeps it.
- FP32 form, inherited coefficients: accumulated in double-float down each
  branch, so the error does not grow with the depth of the tree.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_FP32_RMS, acc_rel, solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_reported_sums_are_compensated(prec):
    pos, m, h = workloads.plummer(200_000, 71)
    s = solver(prec)
    s.build(pos, m, h, 16)
    acc, pot = s.gravity(0.5, 2)
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    st = s.stats()
    s.close()
    ma = m[:, None] * acc  # the same products the device forms (one rounding each)
    scale = np.abs(ma).sum()
    for d in range(3):
        exact = math.fsum(ma[:, d])
        # compensated: |err| <= 2 eps |S| + n eps^2 sum|x|; a plain sum errs by ~log2(n) eps sum|x|
        assert abs(st["momentum"][d] - exact) <= 4e-16 * abs(exact) + 1e-25 * scale, (d, st["momentum"][d], exact)
    # same-sign sums are plain FP64 sums in a fixed tree: a few tens of eps at most
    assert abs(st["abs_momentum"] - math.fsum(np.abs(ma).ravel())) <= 1e-14 * scale
    W = 0.5 * math.fsum(m * pot)
    assert abs(st["W"] - W) <= 1e-14 * abs(W)


def test_noalloc_sums_are_compensated_on_cancelling_input():
    """Crafted input whose plain sum loses most digits: large values in
    cancelling pairs plus small ones.  The compensated result equals the
    exactly rounded sum (math.fsum) to far below the plain sum's error."""
    import torch

    from paper_2602_05804_gb300 import sfmm

    rng = np.random.default_rng(5)
    big = rng.normal(0.0, 1e10, 100_000)
    a = np.concatenate([big, -big[::-1]]) + rng.normal(0.0, 1.0, 200_000)
    acc = np.stack([a, np.roll(a, 7), np.roll(a, 11)], axis=1)
    m = np.ones(len(a))
    pot = -np.abs(a)
    exact = [math.fsum(acc[:, d]) for d in range(3)]
    plain_err = max(abs(float(np.sum(acc[:, d])) - exact[d]) for d in range(3))
    dev = "cuda"
    out = torch.empty(5, dtype=torch.float64, device=dev)
    md, ad, pd = (torch.from_numpy(x).to(dev) for x in (m, np.ascontiguousarray(acc), pot))
    sfmm.sfmm_reduce_noalloc(len(m), md, ad, pd, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for d in range(3):
        assert abs(got[d] - exact[d]) <= 4e-16 * abs(exact[d]) + 1e-9, (d, got[d], exact[d])
    assert plain_err > 1e-6  # the input really defeats a plain sum
    assert abs(got[3] - math.fsum(np.abs(acc).ravel())) <= 5e-14 * got[3]
    assert abs(got[4] - 0.5 * math.fsum(pot)) <= 5e-14 * abs(got[4])


@pytest.mark.parametrize("theta", [0.5, 0.9])
def test_fp32_form_without_dipole_matches_oracle_at_order_one(theta):
    """p = 1: the far field is monopole + dipole only, so a dipole that did
    not vanish about the centre of mass would show at once."""
    pos, m, h = workloads.plummer(20_000, 72)
    a_o, _, st_o = oracle.sfmm(pos, m, h, theta=theta, p=1, leaf_size=16)
    s = solver("fp32")
    s.build(pos, m, h, 16)
    acc, _ = s.gravity(theta, 1)
    st = s.stats()
    s.close()
    assert st["m2l"] == st_o["m2l"]
    e = acc_rel(acc.cpu().numpy(), a_o)
    rms = math.sqrt((e**2).mean())
    print("fp32 p 1 theta %.1f: rms %.3e max %.3e" % (theta, rms, e.max()))
    assert rms <= TOL_FP32_RMS


def test_fp32_error_does_not_grow_with_branch_depth():
    """Leaf size 1 on a clustered set gives branches of 30+ levels; the
    double-float accumulation of the inherited coefficients keeps the FP32
    form's error at the level of a shallow tree's."""
    pos, m, h = workloads.clustered_cloud(20_000, 73)
    out = {}
    for leaf in (1, 32):
        t = oracle.Tree(pos, m, h, leaf, p=2)
        a_o, _, _ = t.sfmm(0.5)
        s = solver("fp32")
        s.build(pos, m, h, leaf)
        acc, _ = s.gravity(0.5, 2)
        depth = int(s.tree()["depth"].max())
        s.close()
        e = acc_rel(acc.cpu().numpy(), a_o)
        out[leaf] = (math.sqrt((e**2).mean()), e.max(), depth)
        print("fp32 clustered 2e4 leaf %d: depth %d rms %.3e max %.3e" % (leaf, depth, out[leaf][0], out[leaf][1]))
    assert out[1][2] >= 30
    assert out[1][0] <= TOL_FP32_RMS and out[32][0] <= TOL_FP32_RMS
