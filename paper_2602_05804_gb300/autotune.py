"""Leaf-size autotuner for batched ensembles.

Picks, per (size bucket, density profile, theta, order, arithmetic form), the
leaf size in {8, 16, 32, 64} that gives the shortest build + gravity time on
this GPU, from timed trials on a synthetic system of the bucket's typical
size, and caches the choices in a JSON file.  Sizes are bucketed by
floor(log2 N); profiles are the caller's labels ("plummer", "uniform", ...),
used to generate the trial system.
"""
from __future__ import annotations

import json
import math
import os
import time

CANDIDATES = (8, 16, 32, 64)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(n, profile, theta, order, precision):
    return "%d|%s|%.3f|%d|%s" % (int(math.log2(max(n, 2))), profile, theta, order, precision)


def _trial_system(n, profile, seed):
    import workloads

    gen = workloads.plummer if profile == "plummer" else workloads.uniform_sphere
    return gen(int(n), seed)


def _time_leaf(torch, solver_cls, pos, m, h, leaf, theta, order, precision, trials):
    from . import sfmm

    s = solver_cls(torch.cuda.current_device(), precision)
    try:
        n = len(m)
        pd = torch.from_numpy(pos).cuda()
        md = torch.from_numpy(m).cuda()
        hd = torch.from_numpy(h).cuda()
        acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        sfmm.sfmm_build(s.ctx, n, pd, md, hd, leaf)
        sfmm.sfmm_gravity(s.ctx, theta, order, acc, pot)  # warm-up (capacities)
        best = float("inf")
        for _ in range(trials):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sfmm.sfmm_build(s.ctx, n, pd, md, hd, leaf)
            sfmm.sfmm_gravity(s.ctx, theta, order, acc, pot)
            best = min(best, time.perf_counter() - t0)
        return best
    finally:
        s.close()


class Autotuner:
    def __init__(self, cache_path: str = DEFAULT_CACHE, trials: int = 3):
        self.cache_path = cache_path
        self.trials = trials
        self.table = {}
        if os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    self.table = json.load(f)
            except (OSError, ValueError):
                self.table = {}

    def save(self):
        os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
        tmp = self.cache_path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def leaf_size(self, n, profile, theta, order, precision):
        """Best leaf size for one system (timed trials on first use)."""
        key = _key(n, profile, theta, order, precision)
        if key not in self.table:
            import torch

            from .sfmm import Solver

            bucket = int(math.log2(max(n, 2)))
            ntrial = int(2 ** (bucket + 0.5))
            pos, m, h = _trial_system(ntrial, profile, 7000 + bucket)
            times = {leaf: _time_leaf(torch, Solver, pos, m, h, leaf, theta, order, precision, self.trials)
                     for leaf in CANDIDATES}
            best = min(times, key=times.get)
            self.table[key] = {"leaf_size": best, "trial_n": ntrial,
                               "ms": {str(k): 1e3 * v for k, v in times.items()}}
            self.save()
        return int(self.table[key]["leaf_size"])

    def leaf_sizes(self, sizes, profiles, theta, order, precision):
        return [self.leaf_size(int(n), p, theta, order, precision) for n, p in zip(sizes, profiles)]
