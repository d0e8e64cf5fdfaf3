"""Shared helpers of the GPU parity tests: tolerances and error metrics."""
import numpy as np

TOL_FP64 = 1e-10      # per particle, relative (acceleration and potential)
TOL_FP32_RMS = 1e-5   # rms relative acceleration error of the FP32 form
TOL_FP32_MAX = 3e-5   # max per-particle relative acceleration error of the FP32 form (largest seen: 1.2e-5)
TOL_MOM_FP64 = 1e-14  # |sum m a| / sum |m a|
TOL_MOM_FP32 = 1e-6


def acc_rel(acc, ref):
    """|da| / max(|a|, 1e-3 rms |a|) per particle (the floor keeps particles
    with a ~ 0 near the centre of a symmetric system from dominating)."""
    an = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt((an**2).mean())
    return np.linalg.norm(acc - ref, axis=1) / np.maximum(an, floor)


def pot_rel(pot, ref):
    return np.abs(pot - ref) / np.abs(ref)


def momentum_residual(m, acc):
    ma = m[:, None] * acc
    return np.linalg.norm(ma.sum(0)) / np.abs(ma).sum()


# walk forms under test: 0 per-leaf replay (Algorithm 1), 1 per-node shared
# pairs with one launch per depth, 2 one-sided symmetric pairs, 3 per-node
# shared pairs taken from the readiness queue of nodes, 4 the same from the
# readiness queue of sibling pairs
WALKS = {0: {"walk": 0}, 1: {"walk": 1, "schedule": 1}, 2: {"walk": 2}, 3: {"walk": 1, "schedule": 2},
         4: {"walk": 1, "schedule": 3}}


def solver(prec, walk=None, **opts):
    """A solver of the given precision; `walk` picks one of WALKS (absent:
    the library's defaults)."""
    from paper_2602_05804_gb300 import sfmm

    if walk is not None:
        opts = {**WALKS[walk], **opts}
    return sfmm.Solver(0, prec, **opts)
