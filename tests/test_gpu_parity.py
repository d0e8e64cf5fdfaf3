"""GPU parity against the FP64 CPU oracle (needs a GB300; marked gpu).

Every test calls the CUDA library through the C ABI (ctypes binding) on
seeded inputs and compares element by element with the oracle:
  - the tree: keys, permutation, node ranges, links, depths, leaves exactly;
    centres/sizes to rounding, h_max exactly;
  - the mass moments to rounding;
  - the interaction lists of Algorithm 2 exactly (per leaf, as multisets);
  - accelerations and potentials: FP64 form <= 1e-10 relative per particle,
    FP32 form <= 1e-5 rms relative, momentum residual <= 1e-14 / 1e-6.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import (TOL_FP32_MAX, TOL_FP32_RMS, TOL_FP64, TOL_MOM_FP32, TOL_MOM_FP64, acc_rel,
                         momentum_residual, pot_rel, solver)

pytestmark = pytest.mark.gpu


def _set(kind, n, seed):
    return {"uniform": workloads.uniform_sphere, "plummer": workloads.plummer,
            "binary": workloads.binary_polytrope}[kind](n, seed)


CASES = [("uniform", 4000, 10), ("plummer", 5003, 16), ("plummer", 3001, 1), ("binary", 2999, 64),
         ("uniform", 777, 8)]


@pytest.mark.parametrize("kind,n,ls", CASES)
def test_tree_matches_oracle(kind, n, ls):
    pos, m, h = _set(kind, n, 21)
    t = oracle.Tree(pos, m, h, ls, p=2)
    s = solver("fp64")
    s.build(pos, m, h, ls)
    g = s.tree()
    assert g["first"].shape[0] == t.nnodes
    np.testing.assert_array_equal(g["keys"], t.keys)
    np.testing.assert_array_equal(g["perm"], t.perm)
    np.testing.assert_array_equal(g["first"], t.first)
    np.testing.assert_array_equal(g["count"], t.count)
    np.testing.assert_array_equal(g["right"], t.right)
    np.testing.assert_array_equal(g["parent"], t.parent)
    np.testing.assert_array_equal(g["depth"], t.depth)
    np.testing.assert_array_equal(g["leaves"], t.leaves)
    np.testing.assert_array_equal(g["hmax"], t.hmax)
    np.testing.assert_allclose(g["mass"], t.mass, rtol=1e-13)
    # centres: bottom-up (GPU) vs direct (oracle) sums of n terms of size
    # <= scale differ by at most ~ n eps scale; 1e-12 scale covers n <= 9000
    scale = np.abs(pos).max()
    np.testing.assert_allclose(g["centre"], t.centre, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(g["size"], t.size, rtol=0, atol=2e-12 * scale)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_moments_match_oracle(p, prec):
    """FP64 moments against the oracle's.  In the FP32 form the build keeps
    FP32 rows only; the export recomputes the FP64 moments."""
    pos, m, h = workloads.plummer(3000, 5)
    t = oracle.Tree(pos, m, h, 12, p=p)
    s = solver(prec)
    s.build(pos, m, h, 12)
    Q, mi = s.moments(p)
    fact = np.array([math.factorial(a) * math.factorial(b) * math.factorial(c) for a, b, c in mi])
    for k, (a, b, c) in enumerate(mi):
        n = a + b + c
        ref = t.Q[:, oracle.rank_offset(n) + oracle.full_index((a, b, c))]
        got = Q[:, k] * fact[k]
        scale = np.abs(t.Q[:, oracle.rank_offset(n):oracle.rank_offset(n + 1)]).max(axis=1) + t.mass * t.size**n
        if n == 1:  # dipole about the centre of mass: rounding level only
            assert np.all(np.abs(got - ref) <= 1e-12 * (t.mass * np.abs(pos).max() + scale))
        else:
            assert np.all(np.abs(got - ref) <= 1e-12 * scale), (a, b, c)


def _per_leaf_sets(mo, lv, src, po, ps):
    """Per leaf, the sorted multiset of its M2L entries (level, source) and
    of its neighbour leaves: a duplicated or missing entry changes it."""
    m2l = [sorted(zip(lv[mo[q]:mo[q + 1]].tolist(), src[mo[q]:mo[q + 1]].tolist())) for q in range(len(mo) - 1)]
    p2p = [sorted(ps[po[q]:po[q + 1]].tolist()) for q in range(len(po) - 1)]
    return m2l, p2p


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
@pytest.mark.parametrize("kind,n,ls", [("uniform", 4000, 10), ("plummer", 6000, 16), ("binary", 3000, 4)])
def test_lists_match_oracle(kind, n, ls, theta):
    pos, m, h = _set(kind, n, 33)
    t = oracle.Tree(pos, m, h, ls, p=0)
    s = solver("fp32")
    s.build(pos, m, h, ls)
    om, op = _per_leaf_sets(*t.lists(theta))
    gm, gp = _per_leaf_sets(*s.lists(theta))
    assert len(om) == len(gm)
    diff = [q for q in range(len(om)) if om[q] != gm[q] or op[q] != gp[q]]
    assert not diff, "lists differ for %d leaves (first %s)" % (len(diff), diff[:5])
    # the GPU's own list counts equal the oracle's
    mo = t.lists(theta)[0]
    assert sum(len(x) for x in gm) == mo[-1]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind,n,ls", [("uniform", 1500, 10), ("plummer", 2001, 3)])
def test_theta_zero_equals_direct(prec, kind, n, ls):
    pos, m, h = _set(kind, n, 9)
    acc_d, pot_d = oracle.direct(pos, m, h)
    s = solver(prec)
    s.build(pos, m, h, ls)
    acc, pot = s.gravity(0.0, 2)
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    st = s.stats()
    assert st["m2l"] == 0 and st["p2p_pairs"] == n * (n - 1)
    e = acc_rel(acc, acc_d)
    if prec == "fp64":
        assert e.max() <= 1e-12 and pot_rel(pot, pot_d).max() <= 1e-12
    else:
        assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS


PARITY = [("uniform", 6000, 10, 0.5, 2), ("plummer", 8001, 16, 0.5, 2), ("plummer", 5000, 16, 0.3, 3),
          ("plummer", 5000, 8, 0.7, 1), ("uniform", 3000, 32, 0.6, 4), ("binary", 6000, 16, 0.5, 0),
          ("plummer", 2500, 1, 0.5, 2), ("uniform", 1000, 64, 0.9, 2)]


@pytest.mark.parametrize("walk", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("kind,n,ls,theta,p", PARITY)
def test_fp64_form_matches_oracle(kind, n, ls, theta, p, walk):
    pos, m, h = _set(kind, n, 17)
    acc_o, pot_o, st_o = oracle.sfmm(pos, m, h, theta=theta, p=p, leaf_size=ls)
    s = solver("fp64", walk=walk)
    s.build(pos, m, h, ls)
    acc, pot = s.gravity(theta, p)
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    st = s.stats()
    assert st["m2l"] == st_o["m2l"] and st["p2p_pairs"] == st_o["p2p_pairs"]
    assert st["m2l_unique"] == st_o["m2l_unique"]
    assert acc_rel(acc, acc_o).max() <= TOL_FP64
    assert pot_rel(pot, pot_o).max() <= TOL_FP64
    assert momentum_residual(m, acc) <= TOL_MOM_FP64
    mom = np.linalg.norm(st["momentum"]) / st["abs_momentum"]
    assert mom <= TOL_MOM_FP64
    assert abs(st["W"] - 0.5 * (m * pot_o).sum()) <= 1e-10 * abs(st["W"])


@pytest.mark.parametrize("walk", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("kind,n,ls,theta,p", PARITY)
def test_fp32_form_matches_oracle(kind, n, ls, theta, p, walk):
    pos, m, h = _set(kind, n, 17)
    acc_o, pot_o, st_o = oracle.sfmm(pos, m, h, theta=theta, p=p, leaf_size=ls)
    s = solver("fp32", walk=walk)
    s.build(pos, m, h, ls)
    acc, pot = s.gravity(theta, p)
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    st = s.stats()
    assert st["m2l"] == st_o["m2l"] and st["p2p_pairs"] == st_o["p2p_pairs"]
    e = acc_rel(acc, acc_o)
    print("fp32 %s n %d leaf %d theta %.1f p %d walk %d: acc rel rms %.3e max %.3e" % (
        kind, n, ls, theta, p, walk, math.sqrt((e**2).mean()), e.max()))
    assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS, (math.sqrt((e**2).mean()), e.max())
    assert e.max() <= TOL_FP32_MAX, e.max()
    pe = pot_rel(pot, pot_o)
    assert math.sqrt((pe**2).mean()) <= TOL_FP32_RMS
    assert momentum_residual(m, acc) <= TOL_MOM_FP32


def test_self_potential_and_G():
    pos, m, h = workloads.uniform_sphere(2000, 3)
    acc_o, pot_o, _ = oracle.sfmm(pos, m, h, theta=0.5, p=2, leaf_size=10, G=2.5, self_potential=True)
    s = solver("fp64", G=2.5, self_potential=1)
    s.build(pos, m, h, 10)
    acc, pot = s.gravity(0.5, 2)
    assert acc_rel(acc.cpu().numpy(), acc_o).max() <= TOL_FP64
    assert pot_rel(pot.cpu().numpy(), pot_o).max() <= TOL_FP64


def test_solve_host_equals_device_path():
    import torch

    pos, m, h = workloads.plummer(5000, 4)
    s = solver("fp32")
    s.build(pos, m, h, 16)
    acc_d, pot_d = s.gravity(0.5, 2)
    acc_h = torch.empty((5000, 3), dtype=torch.float64).pin_memory()
    pot_h = torch.empty(5000, dtype=torch.float64).pin_memory()
    pos_h = torch.from_numpy(pos).pin_memory()
    for call in range(2):  # the first call runs and captures the step, the second replays it
        acc_h.fill_(float("nan"))
        s.solve_host(pos_h, torch.from_numpy(m), torch.from_numpy(h), 16, 0.5, 2, acc_h, pot_h)
        np.testing.assert_array_equal(acc_h.numpy(), acc_d.cpu().numpy())
        np.testing.assert_array_equal(pot_h.numpy(), pot_d.cpu().numpy())
        assert s.stats()["graph_replays"] == call


@pytest.mark.parametrize("n", [4001, 2])
def test_solve_host_odd_sizes_and_pinned_buffers(n):
    """All host buffers pinned (the device copies them by a kernel), odd
    counts (the copies' last element) and the smallest captured step."""
    import torch

    pos, m, h = workloads.plummer(n, 7) if n > 2 else (np.array([[0.0, 0, 0], [1.0, 0, 0]]), np.ones(2), np.ones(2))
    s = solver("fp64")
    s.build(pos, m, h, 16)
    acc_d, pot_d = s.gravity(0.5, 2)
    pin = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (pos, m, h)]
    acc_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    pot_h = torch.empty(n, dtype=torch.float64).pin_memory()
    for _ in range(2):
        acc_h.fill_(float("nan"))
        pot_h.fill_(float("nan"))
        s.solve_host(pin[0], pin[1], pin[2], 16, 0.5, 2, acc_h, pot_h)
        np.testing.assert_array_equal(acc_h.numpy(), acc_d.cpu().numpy())
        np.testing.assert_array_equal(pot_h.numpy(), pot_d.cpu().numpy())
    s.close()


@pytest.mark.parametrize("opts", [{"tree": 1}, {"walk": 0}])
def test_solve_host_without_capture_equals_device_path(opts):
    """Options the captured step does not run (kd tree, per-leaf replay walk):
    the host-buffer solve takes the separate calls, with the same results."""
    import torch

    pos, m, h = workloads.uniform_sphere(3000, 6)
    s = solver("fp32", **opts)
    s.build(pos, m, h, 16)
    acc_d, pot_d = s.gravity(0.5, 2)
    acc_h = torch.empty((3000, 3), dtype=torch.float64).pin_memory()
    pot_h = torch.empty(3000, dtype=torch.float64).pin_memory()
    s.solve_host(torch.from_numpy(pos).pin_memory(), torch.from_numpy(m), torch.from_numpy(h), 16, 0.5, 2, acc_h,
                 pot_h)
    np.testing.assert_array_equal(acc_h.numpy(), acc_d.cpu().numpy())
    np.testing.assert_array_equal(pot_h.numpy(), pot_d.cpu().numpy())
    assert s.stats()["graph_replays"] == 0
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_deterministic_rerun(prec):
    pos, m, h = workloads.plummer(6000, 8)
    s = solver(prec)
    s.build(pos, m, h, 16)
    a1, p1 = s.gravity(0.5, 2)
    a1, p1 = a1.cpu().numpy(), p1.cpu().numpy()
    s.build(pos, m, h, 16)
    a2, p2 = s.gravity(0.5, 2)
    np.testing.assert_array_equal(a1, a2.cpu().numpy())
    np.testing.assert_array_equal(p1, p2.cpu().numpy())


def test_capacity_regrow_retry():
    pos, m, h = workloads.plummer(6000, 12)
    acc_o, pot_o, _ = oracle.sfmm(pos, m, h, theta=0.3, p=2, leaf_size=16)
    s = solver("fp64", ring_capacity=256, list_capacity=64)
    s.build(pos, m, h, 16)
    acc, pot = s.gravity(0.3, 2)
    assert acc_rel(acc.cpu().numpy(), acc_o).max() <= TOL_FP64


def test_edge_cases_small_systems():
    from paper_2602_05804_gb300 import sfmm

    # one particle: no force; two particles: Newton; fewer than leaf_size
    for n in (1, 2, 7):
        pos, m, h = workloads.uniform_sphere(n, 2)
        for prec in ("fp64", "fp32"):
            s = solver(prec)
            s.build(pos, m, h, 10)
            acc, pot = s.gravity(0.5, 2)
            acc_d, pot_d = oracle.direct(pos, m, h)
            np.testing.assert_allclose(acc.cpu().numpy(), acc_d, rtol=1e-5, atol=1e-12)
            np.testing.assert_allclose(pot.cpu().numpy(), pot_d, rtol=1e-5, atol=1e-12)
    # coincident particles (equal keys)
    pos = np.zeros((50, 3))
    pos[25:] = 1.0
    m = np.full(50, 0.02)
    h = np.full(50, 0.05)
    acc_d, pot_d = oracle.direct(pos, m, h)
    s = solver("fp64")
    s.build(pos, m, h, 4)
    acc, pot = s.gravity(0.5, 2)
    np.testing.assert_allclose(acc.cpu().numpy(), acc_d, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(pot.cpu().numpy(), pot_d, rtol=1e-12)


def test_errors_are_reported():
    import torch

    from paper_2602_05804_gb300 import sfmm

    s = solver("fp32")
    with pytest.raises(sfmm.SFMMError) as e:
        s.gravity(0.5, 2, acc=torch.empty((1, 3), dtype=torch.float64, device="cuda"))
    assert e.value.code == sfmm.SFMM_ESTATE
    pos, m, h = workloads.uniform_sphere(100, 1)
    for bad in ("nan", "h0", "m0"):
        p2, m2, h2 = pos.copy(), m.copy(), h.copy()
        if bad == "nan":
            p2[5, 1] = np.nan
        elif bad == "h0":
            h2[7] = 0.0
        else:
            m2[3] = -1.0
        with pytest.raises(sfmm.SFMMError) as e:
            s.build(p2, m2, h2, 10)
        assert e.value.code == sfmm.SFMM_ENONFINITE
    for ls in (0, 65):
        with pytest.raises(sfmm.SFMMError) as e:
            s.build(pos, m, h, ls)
        assert e.value.code == sfmm.SFMM_EINVAL
    s.build(pos, m, h, 10)
    for theta, p in ((1.0, 2), (-0.1, 2), (0.5, 5), (0.5, -1)):
        with pytest.raises(sfmm.SFMMError) as e:
            s.gravity(theta, p)
        assert e.value.code == sfmm.SFMM_EINVAL
    with pytest.raises(sfmm.SFMMError):
        s.set_option("nonsense", 1.0)
    with pytest.raises(sfmm.SFMMError):
        s.set_option("ring_capacity", 1000)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", TOL_FP32_RMS)])
def test_shared_walk_equals_replay(prec, tol):
    """Per-node shared pairs and the per-leaf replay evaluate the same
    interactions: equal counts, results equal up to summation order (in the
    FP32 form the M2L terms are accumulated in FP32 in a walk-dependent
    order, so the bound is the FP32 form's own tolerance)."""
    pos, m, h = workloads.plummer(20000, 44)
    out = []
    for walk in (0, 1):
        s = solver(prec, walk=walk)
        s.build(pos, m, h, 16)
        acc, pot = s.gravity(0.5, 2)
        out.append((acc.cpu().numpy(), pot.cpu().numpy(), s.stats()))
    (a0, p0, s0), (a1, p1, s1) = out
    for k in ("m2l", "m2l_unique", "p2p_pairs", "p2p_leaves"):
        assert s0[k] == s1[k], k
    assert acc_rel(a1, a0).max() <= tol
    assert pot_rel(p1, p0).max() <= tol


@pytest.mark.parametrize("walk", [1, 3, 4])
def test_shared_walk_capacity_regrow(walk):
    pos, m, h = workloads.plummer(6000, 12)
    acc_o, pot_o, _ = oracle.sfmm(pos, m, h, theta=0.3, p=2, leaf_size=16)
    s = solver("fp64", walk=walk, ring_capacity=256, list_capacity=64)
    s.build(pos, m, h, 16)
    acc, pot = s.gravity(0.3, 2)
    assert acc_rel(acc.cpu().numpy(), acc_o).max() <= TOL_FP64


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("walk", [0, 1, 3, 4])
def test_long_lists_split_into_chunks(prec, walk):
    """Neighbour lists longer than one chunk are evaluated as several work
    items and recombined in chunk order: the result still matches the
    oracle, and a rerun is bitwise identical."""
    pos, m, h = workloads.uniform_sphere(6000, 31)
    acc_o, pot_o, st_o = oracle.sfmm(pos, m, h, theta=0.1, p=2, leaf_size=4)
    s = solver(prec, walk=walk)
    s.build(pos, m, h, 4)
    acc, pot = s.gravity(0.1, 2)
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    st = s.stats()
    assert st["p2p_leaves"] == st_o["p2p_leaves"] and st["p2p_pairs"] == st_o["p2p_pairs"]
    assert st["p2p_leaves"] > 2 * 256 * st["nleaves"] // 4  # most lists span several chunks
    e = acc_rel(acc, acc_o)
    if prec == "fp64":
        assert e.max() <= TOL_FP64
        assert pot_rel(pot, pot_o).max() <= TOL_FP64
        assert momentum_residual(m, acc) <= TOL_MOM_FP64
    else:
        assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS
        assert momentum_residual(m, acc) <= TOL_MOM_FP32
    s.build(pos, m, h, 4)
    acc2, pot2 = s.gravity(0.1, 2)
    np.testing.assert_array_equal(acc, acc2.cpu().numpy())
    np.testing.assert_array_equal(pot, pot2.cpu().numpy())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", TOL_FP32_RMS)])
def test_one_sided_symmetric_pairs_equal_shared_walk(prec, tol):
    """Walk mode 2 evaluates D once per pair for both sides (Sect. 5): same
    interaction counts as the shared walk, same results up to summation
    order, momentum to round-off in the FP64 form."""
    pos, m, h = workloads.plummer(30000, 45)
    out = []
    for walk in (1, 2):
        s = solver(prec, walk=walk)
        s.build(pos, m, h, 16)
        acc, pot = s.gravity(0.5, 2)
        out.append((acc.cpu().numpy(), pot.cpu().numpy(), s.stats()))
    (a1, p1, s1), (a2, p2, s2) = out
    for k in ("m2l", "m2l_unique", "p2p_pairs", "p2p_leaves"):
        assert s1[k] == s2[k], k
    assert acc_rel(a2, a1).max() <= tol
    assert pot_rel(p2, p1).max() <= tol
    if prec == "fp64":
        assert momentum_residual(m, a2) <= TOL_MOM_FP64


@pytest.mark.parametrize("walk", [0, 1, 2, 3, 4])
def test_small_theta_grows_buffers_and_matches_oracle(walk):
    """theta = 0.1: almost every pair is done pairwise, lists are long and
    several work buffers must grow (regrow and retry inside the call)."""
    pos, m, h = workloads.plummer(20000, 46)
    acc_o, pot_o, st_o = oracle.sfmm(pos, m, h, theta=0.1, p=2, leaf_size=16)
    s = solver("fp32", walk=walk)
    s.build(pos, m, h, 16)
    acc, pot = s.gravity(0.1, 2)
    st = s.stats()
    assert st["p2p_pairs"] == st_o["p2p_pairs"] and st["m2l"] == st_o["m2l"]
    e = acc_rel(acc.cpu().numpy(), acc_o)
    assert math.sqrt((e**2).mean()) <= TOL_FP32_RMS


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind,n,theta", [("plummer", 40000, 0.5), ("binary", 30000, 0.3)])
def test_queue_walk_equals_level_walk(prec, kind, n, theta):
    """The readiness queues run the per-node shared walk as one launch over
    nodes (or sibling pairs) whose parents are done, instead of one launch
    per depth: every node does the same arithmetic on the same inherited
    list in the same order, so the results are bitwise the same, and so are
    those of the automatic choice."""
    pos, m, h = _set(kind, n, 47)
    out = []
    for walk in (1, 3, 4):
        s = solver(prec, walk=walk)
        s.build(pos, m, h, 16)
        acc, pot = s.gravity(theta, 2)
        out.append((acc.cpu().numpy(), pot.cpu().numpy(), s.stats()))
    s = solver(prec)  # automatic schedule
    s.build(pos, m, h, 16)
    acc, pot = s.gravity(theta, 2)
    out.append((acc.cpu().numpy(), pot.cpu().numpy(), s.stats()))
    (a1, p1, s1) = out[0]
    for a3, p3, s3 in out[1:]:
        for k in ("m2l", "m2l_unique", "p2p_pairs", "p2p_leaves", "mac_fallbacks"):
            assert s1[k] == s3[k], k
        np.testing.assert_array_equal(a3, a1)
        np.testing.assert_array_equal(p3, p1)


def test_schedule_option_is_checked():
    from paper_2602_05804_gb300 import sfmm

    s = solver("fp32")
    for bad in (-1, 4, 0.5):
        with pytest.raises(sfmm.SFMMError) as e:
            s.set_option("schedule", bad)
        assert e.value.code == sfmm.SFMM_EINVAL
    with pytest.raises(sfmm.SFMMError):
        s.set_option("walk", 3)
