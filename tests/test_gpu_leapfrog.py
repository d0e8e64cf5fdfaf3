"""Gravity-only leapfrog on the GPU (the binary-polytrope test of Sect. 4)
against the oracle leapfrog, and linear momentum conservation over many
steps (needs a GB300; marked gpu)."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import solver

pytestmark = pytest.mark.gpu


def test_fp64_leapfrog_matches_oracle():
    pos, vel, m, h = workloads.binary_orbit(3000, 5)
    steps, dt = 6, 0.02
    xo, vo, ro = oracle.leapfrog(pos, vel, m, h, theta=0.5, p=2, leaf_size=16, dt=dt, nsteps=steps, record_every=2)
    s = solver("fp64")
    x, v, r = s.leapfrog(pos, vel, m, h, 16, 0.5, 2, dt, steps, record_every=2)
    x, v = x.cpu().numpy(), v.cpu().numpy()
    # per-step forces agree to 1e-10 relative: trajectories agree far below the step
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-12 * np.abs(xo).max())
    np.testing.assert_allclose(v, vo, rtol=0, atol=1e-10 * np.abs(vo).max())
    assert r.shape == ro.shape
    np.testing.assert_array_equal(r[:, 0], ro[:, 0])
    scale = ro[:, 7].max()
    np.testing.assert_allclose(r[:, 1:7], ro[:, 1:7], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(r[:, 7], ro[:, 7], rtol=1e-12)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_linear_momentum_is_conserved_over_many_steps(prec, tol):
    """Symmetric pair forces: sum m v stays at its initial value to rounding
    (FP64 form; the FP32 form to its own momentum tolerance) over one
    hundred and fifty steps of the orbiting binary."""
    pos, vel, m, h = workloads.binary_orbit(20000, 6)
    s = solver(prec)
    _, _, r = s.leapfrog(pos, vel, m, h, 16, 0.5, 2, 0.05, 150, record_every=10)
    scale = r[:, 7].max()
    drift = np.abs(r[:, 1:4] - r[0, 1:4]).max() / scale
    assert drift <= tol, drift


def test_leapfrog_rejects_bad_arguments():
    from paper_2602_05804_gb300 import sfmm

    pos, vel, m, h = workloads.binary_orbit(100, 1)
    s = solver("fp64")
    for dt, steps, every in ((float("nan"), 1, 1), (0.1, -1, 1), (0.1, 1, 0)):
        with pytest.raises(sfmm.SFMMError) as e:
            s.leapfrog(pos, vel, m, h, 16, 0.5, 2, dt, steps, record_every=every)
        assert e.value.code == sfmm.SFMM_EINVAL
