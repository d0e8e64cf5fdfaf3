"""Batched-ensemble autotuning, through the library's own autotuner.

The tuning itself runs in the CUDA library (``sfmm_autotune_batch``): timed
trials on the caller's own systems pick each system's leaf size in
{8, 16, 32, 64} per (size bucket, profile class, theta, order, form) and the
batch's launch knobs (walk schedule, near-field blocks per SM, list chunk);
``sfmm_autotune_cache`` keeps the table in a JSON file.  This module only
chooses the default cache location and wraps the two calls for torch users.
"""
from __future__ import annotations

import os

from . import sfmm

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def autotuned_solver(device, precision, offsets, pos, mass, h, theta=0.5, order=2, cache=DEFAULT_CACHE, **options):
    """A Solver whose batch is built with autotuned leaf sizes and launch
    knobs (cached in ``cache``; None keeps the table in memory only).
    Returns (solver, leaf sizes per system)."""
    s = sfmm.Solver(device, precision, **options)
    if cache:
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        sfmm.sfmm_autotune_cache(s.ctx, cache)
    leaf = s.autotune_batch(offsets, pos, mass, h, theta, order)
    return s, leaf
