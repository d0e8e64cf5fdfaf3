"""Benchmark of the SFMM gravity solver on one GB300 (or N, one rank each).

A step is one pass of the whole hot path over one particle set: the tree
build (bounding box, Morton keys, sort, radix tree, centres, sizes) and the
gravity (moments, per-leaf walk with M2L/L2L/L2P, softened P2P, reductions),
with inputs resident in HBM.  Default workload: Plummer sphere, N = 10^6,
theta = 0.5, expansion order p = 2, leaf size 16.  The headline value is the
FP32 form's particles/s; the FP64 form and theta = 0.3 / 0.7 are measured
too and reported beside it.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank solves its own particle set (seed + rank): weak
scaling with no data-path collective; the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/sec & interactions/sec of SFMM gravity, FP32 vs FP64 form on 1 GB300"
WORKLOAD = dict(name="plummer_1e6", gen_name="plummer_1e6", n=1_000_000, seed=1002, theta=0.5, order=2,
                leaf_size=16)
FLOPS_PER_PAIR = 20      # far-field pair: dx 3, r^2 5, rsqrt 1, m r^-3 3, acc 6, pot 2 (FMA = 2)
L2_FLUSH_BYTES = 512 << 20


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _kernel_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2602_05804_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel, src_hash):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("source_sha") == src_hash:
            return e["dram_bytes_per_launch"]
    except (OSError, ValueError):
        pass
    return None


def _cpu_baseline(pos, m, h, w, budget_s=20.0):
    """The FP64 oracle as it stands, on the host cores: full tree build, then
    the per-leaf walk on a seeded sample of leaves (per-leaf independence,
    Algorithm 1), scaled to the whole particle set."""
    import oracle

    threads = oracle.max_threads()
    t0 = time.perf_counter()
    t = oracle.Tree(pos, m, h, w["leaf_size"], p=w["order"])
    t_build = time.perf_counter() - t0
    order = np.random.default_rng(7).permutation(t.nleaves).astype(np.int32)
    nsel = 64
    t_walk, nl_done, np_done = 0.0, 0, 0
    while True:
        sel = order[nl_done:nl_done + nsel]
        t0 = time.perf_counter()
        t.sfmm(w["theta"], leaf_sample=sel)
        dt = time.perf_counter() - t0
        t_walk += dt
        nl_done += nsel
        np_done += int(t.count[t.leaves[sel]].sum())
        if t_walk > budget_s or nl_done >= t.nleaves:
            break
        nsel = int(min(t.nleaves - nl_done, max(nsel, nsel * min(8.0, (budget_s - t_walk) / max(dt, 1e-3)))))
    t_full = t_build + t_walk * (t.n / max(np_done, 1))
    return {"value": t.n / t_full, "unit": "particles/s", "cores": threads, "kind": "oracle",
            "sample": "full FP64 oracle tree build (%.1f s) + Algorithms 1-2 on %d of %d leaves (%d particles, "
                      "%.1f s), scaled by particles" % (t_build, nl_done, t.nleaves, np_done, t_walk)}


REF_SLICES = 8  # each reference step walks one eighth of the leaves


def run_reference(args):
    """The oracle as it stands, timed on the host cores, each step a bounded
    slice of the headline workload: the full oracle tree build, then
    Algorithms 1-2 for one eighth of the leaves (a seeded permutation cut in
    eight; step k takes slice k mod 8).  Every leaf's result depends on the
    read-only tree alone, so a slice is exact work of the same solve.  value =
    particles whose forces the timed steps computed / their measured time;
    ms_per_step = the measured mean step time."""
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import oracle
    import workloads

    w = WORKLOAD
    pos, m, h = workloads.make(w["gen_name"], n=w["n"], seed=w["seed"])
    threads = oracle.max_threads()
    times, parts, builds = [], [], []
    perm = None
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t = oracle.Tree(pos, m, h, w["leaf_size"], p=w["order"])
        t1 = time.perf_counter()
        if perm is None:
            perm = np.random.default_rng(7).permutation(t.nleaves).astype(np.int32)
        sel = np.sort(perm[it % REF_SLICES::REF_SLICES])
        t.sfmm(w["theta"], leaf_sample=sel)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            builds.append(t1 - t0)
            parts.append(int(t.count[t.leaves[sel]].sum()))
        del t
    value = sum(parts) / sum(times)
    ms = 1e3 * float(np.mean(times))
    base = {"value": value, "unit": "particles/s", "cores": threads, "kind": "oracle",
            "sample": "per step: full FP64 oracle tree build of all %d particles (mean %.2f s) + Algorithms 1-2 "
                      "on one eighth of the leaves (mean %d particles); value = particles computed / measured "
                      "time over %d timed steps" % (w["n"], float(np.mean(builds)), int(np.mean(parts)),
                                                     args.steps)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded %s)" % w["gen_name"],
            "config": {"workload": w["name"], "n": w["n"], "theta": w["theta"], "order": w["order"],
                       "leaf_size": w["leaf_size"], "form": "oracle FP64 (CPU)",
                       "step": "tree build + one eighth of the leaves"},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def rank_workload(w, rank):
    """The particle set of one rank: every rank solves its own seeded system
    (weak scaling; no data-path exchange between ranks)."""
    return dict(w, seed=w["seed"] + rank)


def reduce_timing(dist, step_ms, n_local, device=None):
    """Whole-job throughput: the slowest rank's step time and the particles of
    all ranks.  Returns (max step ms over ranks, total particles)."""
    if dist is None:
        return step_ms, n_local
    import torch

    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def _flush(buf):
    buf.add_(1)


def time_steps(torch, solver, pos_d, m_d, h_d, acc, pot, w, theta, steps, warmup, flush):
    """Per-step device time (CUDA events on the solver's stream), L2 flushed
    between steps outside the events."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    from paper_2602_05804_gb300 import sfmm

    n = m_d.shape[0]
    for _ in range(warmup):
        sfmm.sfmm_build(solver.ctx, n, pos_d, m_d, h_d, w["leaf_size"])
        sfmm.sfmm_gravity(solver.ctx, theta, w["order"], acc, pot)
    stage = {"ms_build": 0.0, "ms_moments": 0.0, "ms_walk": 0.0, "ms_p2p": 0.0, "ms_reduce": 0.0}
    launches0 = solver.stats()["kernel_launches"]
    for k in range(steps):
        _flush(flush)
        ev[k][0].record(solver.stream)
        sfmm.sfmm_build(solver.ctx, n, pos_d, m_d, h_d, w["leaf_size"])
        sfmm.sfmm_gravity(solver.ctx, theta, w["order"], acc, pot)
        ev[k][1].record(solver.stream)
        st = solver.stats()
        for key in stage:
            stage[key] += st[key]
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    st = solver.stats()
    st["kernel_launches_per_step"] = (st["kernel_launches"] - launches0) / steps
    for key in stage:
        st[key] = stage[key] / steps
    return ms, st


def graph_block(torch, local, pos_d, m_d, h_d, acc, pot, w, steps, flush, warmup=3):
    """The headline step (FP32 form) through sfmm_solve_graph: build and
    gravity replayed as one captured CUDA graph per shape class, one host
    synchronisation per step (after warm-up calls that run, size and
    capture it).  Results are bitwise those of the ordinary calls."""
    from paper_2602_05804_gb300 import sfmm

    n = m_d.shape[0]
    off = np.array([0, n], np.int64)
    leaf = np.array([w["leaf_size"]], np.int32)
    s = sfmm.Solver(local, "fp32")
    for _ in range(max(3, warmup)):  # the first call runs, sizes and captures
        sfmm.sfmm_solve_graph(s.ctx, off, pos_d, m_d, h_d, leaf, w["theta"], w["order"], acc, pot)
    st0 = s.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        _flush(flush)
        ev[k][0].record(s.stream)
        sfmm.sfmm_solve_graph(s.ctx, off, pos_d, m_d, h_d, leaf, w["theta"], w["order"], acc, pot)
        ev[k][1].record(s.stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    st = s.stats()
    s.close()
    return {"ms_per_step": ms, "particles_per_s": n / (ms * 1e-3), "steps": steps,
            "replays": st["graph_replays"] - st0["graph_replays"],
            "kernels_per_step": (st["kernel_launches"] - st0["kernel_launches"]) / steps,
            "how": "sfmm_solve_graph: build + gravity as one CUDA graph, replayed; one synchronisation per step"}


def ensemble_block(torch, local, flush, steps):
    """Batched ensemble: 256 independent systems (sizes log-uniform in
    [10^3, 10^5], alternating Plummer / uniform sphere), theta 0.5, p 2:
    the FP32 form over the whole batch in the same launches, with leaf sizes
    and launch knobs from the library's autotuner (timed trials on these
    systems; the timed steps pass NULL leaf sizes, which take the tuned
    table), replayed as one captured CUDA graph and through the ordinary
    calls, against the FP64 form run system by system."""
    import workloads
    from paper_2602_05804_gb300 import sfmm
    from paper_2602_05804_gb300.autotune import DEFAULT_CACHE, autotuned_solver

    pos, m, h, off = workloads.ensemble(1004)
    sizes = np.diff(off)
    nsys, ntot = len(sizes), int(off[-1])
    dev = torch.device("cuda", local)
    pd, md, hd = (torch.from_numpy(x).to(dev) for x in (pos, m, h))
    acc = torch.empty((ntot, 3), dtype=torch.float64, device=dev)
    pot = torch.empty(ntot, dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    sb, leaf = autotuned_solver(local, "fp32", off, pd, md, hd, 0.5, 2, cache=DEFAULT_CACHE)
    t_tune = time.perf_counter() - t0
    try:
        with open(DEFAULT_CACHE) as f:
            knobs = json.load(f).get("knobs")
    except (OSError, ValueError):
        knobs = None
    def timed(step, k_steps):
        for _ in range(3):
            step()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
        for k in range(k_steps):
            _flush(flush)
            ev[k][0].record(sb.stream)
            step()
            ev[k][1].record(sb.stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    # the ordinary calls, autotuned leaf sizes (NULL)
    def ordinary():
        sfmm.sfmm_build_batch(sb.ctx, off, pd, md, hd, None)
        sfmm.sfmm_gravity_batch(sb.ctx, 0.5, 2, acc, pot)

    ms_o = timed(ordinary, steps)
    # all 256 systems as one captured CUDA graph (first call captures)
    r0 = sb.stats()["graph_replays"]
    ms_b = timed(lambda: sfmm.sfmm_solve_graph(sb.ctx, off, pd, md, hd, None, 0.5, 2, acc, pot), steps)
    replays = sb.stats()["graph_replays"] - r0
    sums = sfmm.sfmm_batch_sums(sb.ctx, nsys)
    sb.close()
    # FP64 form, one system at a time
    s64 = sfmm.Solver(local, "fp64")
    sfmm.sfmm_build(s64.ctx, int(sizes[0]), pd[:sizes[0]], md[:sizes[0]], hd[:sizes[0]], 16)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(nsys):
        a, b = int(off[k]), int(off[k + 1])
        sfmm.sfmm_build(s64.ctx, b - a, pd[a:b], md[a:b], hd[a:b], 16)
        sfmm.sfmm_gravity(s64.ctx, 0.5, 2, acc[a:b], pot[a:b])
    torch.cuda.synchronize()
    ms_s = 1e3 * (time.perf_counter() - t0)
    s64.close()
    mom = np.linalg.norm(sums[:, :3], axis=1) / sums[:, 3]
    hist = {str(v): int((leaf == v).sum()) for v in sorted(set(leaf.tolist()))}
    return {"systems": nsys, "n_total": ntot, "n_min": int(sizes.min()), "n_max": int(sizes.max()),
            "batched_fp32": {"particles_per_s": ntot / (ms_b * 1e-3), "ms_per_step": ms_b, "steps": steps,
                             "path": "sfmm_solve_graph: all systems' build + gravity as one captured CUDA graph",
                             "graph_replays": replays, "leaf_sizes": hist,
                             "max_momentum_residual": float(mom.max())},
            "batched_fp32_ordinary_calls": {"particles_per_s": ntot / (ms_o * 1e-3), "ms_per_step": ms_o},
            "autotune": {"seconds": t_tune, "leaf_sizes": hist, "knobs": knobs,
                         "how": "sfmm_autotune_batch: leaf size per (log2 N, profile class, theta, p, form) and "
                                "walk schedule / near-field blocks per SM / list chunk per batch, from timed trials"},
            "sequential_fp64": {"particles_per_s": ntot / (ms_s * 1e-3), "ms_per_step": ms_s},
            "speedup": ms_s / ms_b}


def measured_peaks(local, stream):
    """FMA throughput of this GPU measured by the library's own FMA kernel
    (eight independent chains per thread, every SM full): FP64, FP32 and
    packed FP32, best of five 50 ms launches each, with the SM clock sampled
    while it runs.  The FP32 peak is the larger of the scalar and packed
    rates."""
    from paper_2602_05804_gb300 import sfmm

    out = {}
    with ClockSampler(local) as clk:
        for key, form in (("fp64_tflops", 0), ("fp32_scalar_tflops", 1), ("fp32_packed_tflops", 2)):
            out[key], _ = sfmm.sfmm_fma_peak(local, form, stream, target_ms=50.0, reps=5)
    out["fp32_tflops"] = max(out["fp32_scalar_tflops"], out["fp32_packed_tflops"])
    out["clocks"] = clk.summary()
    out["how"] = ("sfmm_fma_peak: 152 x 4 blocks of 256 threads, 8 independent FMA chains per thread, "
                  "best of 5 launches of ~50 ms, CUDA events")
    return out


def _acc_rel(acc, ref):
    """|da| / max(|a|, 1e-3 rms |a|) per particle (the parity tests' metric)."""
    an = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt((an**2).mean())
    return np.linalg.norm(acc - ref, axis=1) / np.maximum(an, floor)


def _err_stats(e):
    return {"rms": float(np.sqrt((e**2).mean())), "max": float(e.max()), "mean": float(e.mean())}


def oracle_error_block(pos, m, h, w, results, nleaf=96, ntarget=4096):
    """Error of each result against the FP64 oracle: accelerations and
    potentials on a seeded sample of leaves of the oracle's tree of the
    result's leaf size (the oracle runs Algorithms 1-2 for those leaves only:
    exact, since a leaf's result depends on the read-only tree alone), plus
    the momentum residual over all particles.  Also each result's, and the
    oracle's, force error against the softened direct sum on seeded targets:
    the truncation error, which is what "equal force accuracy" compares.
    results: name -> (acc, pot, stats, leaf size)."""
    import oracle

    t0 = time.perf_counter()
    rng = np.random.default_rng(11)
    tg = np.sort(rng.choice(len(m), min(ntarget, len(m)), replace=False))
    a_d, _ = oracle.direct(pos, m, h, targets=tg)
    an = np.linalg.norm(a_d, axis=1)
    out = {}
    trees = {}
    for name, (acc, pot, st, leaf) in results.items():
        if leaf not in trees:
            t = oracle.Tree(pos, m, h, leaf, p=w["order"])
            r = np.random.default_rng(11 + leaf)
            sel = np.unique(np.concatenate([r.choice(t.nleaves, min(nleaf, t.nleaves), replace=False),
                                            [0, t.nleaves - 1]])).astype(np.int32)
            a_o, p_o, _ = t.sfmm(w["theta"], leaf_sample=sel)
            idx = np.concatenate([t.perm[t.first[L]:t.first[L] + t.count[L]] for L in t.leaves[sel]])
            leaf_of = np.empty(len(m), np.int64)
            for q, L in enumerate(t.leaves):
                leaf_of[t.perm[t.first[L]:t.first[L] + t.count[L]]] = q
            a_ot, _, _ = t.sfmm(w["theta"], leaf_sample=np.unique(leaf_of[tg]).astype(np.int32))
            trees[leaf] = (a_o, p_o, idx)
            out["oracle_leaf%d_vs_direct" % leaf] = _err_stats(np.linalg.norm(a_ot[tg] - a_d, axis=1) / an)
            out["sample_leaf%d" % leaf] = ("%d leaves (%d particles) vs the oracle; %d seeded targets vs the direct "
                                          "sum" % (len(sel), len(idx), len(tg)))
        a_o, p_o, idx = trees[leaf]
        ep = np.abs(pot[idx] - p_o[idx]) / np.abs(p_o[idx])
        out[name] = {"leaf_size": leaf, "acc_rel_vs_oracle": _err_stats(_acc_rel(acc[idx], a_o[idx])),
                     "pot_rel_vs_oracle": _err_stats(ep),
                     "momentum_residual": float(np.linalg.norm(st["momentum"]) / st["abs_momentum"]),
                     "acc_rel_vs_direct": _err_stats(np.linalg.norm(acc[tg] - a_d, axis=1) / an)}
    out["seconds"] = time.perf_counter() - t0
    return out


def fp64_tuned_block(torch, local, pos_d, m_d, h_d, acc, pot, w, steps, flush):
    """The FP64 form at the leaf size the library's autotuner picks for this
    particle set (sfmm_autotune_batch over the one system: timed trials of
    leaf 8, 16, 32, 64), through the captured graph.  The FP64 near field
    costs 64x the FP32 one per pair, so smaller leaves (more M2L, fewer pairs)
    pay off in this form."""
    from paper_2602_05804_gb300 import sfmm

    n = m_d.shape[0]
    off = np.array([0, n], np.int64)
    s = sfmm.Solver(local, "fp64")
    t0 = time.perf_counter()
    leaf = int(sfmm.sfmm_autotune_batch(s.ctx, off, pos_d, m_d, h_d, w["theta"], w["order"])[0])
    t_tune = time.perf_counter() - t0
    ls = np.array([leaf], np.int32)
    for _ in range(2):
        sfmm.sfmm_solve_graph(s.ctx, off, pos_d, m_d, h_d, ls, w["theta"], w["order"], acc, pot)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        _flush(flush)
        ev[k][0].record(s.stream)
        sfmm.sfmm_solve_graph(s.ctx, off, pos_d, m_d, h_d, ls, w["theta"], w["order"], acc, pot)
        ev[k][1].record(s.stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    st = s.stats()
    s.close()
    return ({"leaf_size": leaf, "ms_per_step": ms, "particles_per_s": n / (ms * 1e-3), "steps": steps,
             "autotune_seconds": t_tune,
             "how": "sfmm_autotune_batch (one system), then sfmm_solve_graph at the chosen leaf size"},
            (acc.cpu().numpy(), pot.cpu().numpy(), st, leaf))


def uniform_1e4_block(torch, local, flush, steps):
    """The small configuration: uniform sphere, N = 10^4, theta 0.5, leaf 10,
    p 2.  Both forms on the GPU against the full FP64 oracle (every particle)
    and the full softened direct sum; the oracle and the direct sum timed on
    the host cores."""
    import oracle
    import workloads
    from paper_2602_05804_gb300 import sfmm

    name = "uniform_1e4"
    wk = dict(workloads.WORKLOADS[name], order=2)
    pos, m, h = workloads.make(name)
    n = len(m)
    t0 = time.perf_counter()
    a_o, p_o, st_o = oracle.sfmm(pos, m, h, theta=wk["theta"], p=2, leaf_size=wk["leaf_size"])
    t_oracle = time.perf_counter() - t0
    t0 = time.perf_counter()
    a_d, p_d = oracle.direct(pos, m, h)
    t_direct = time.perf_counter() - t0
    an = np.linalg.norm(a_d, axis=1)
    dev = torch.device("cuda", local)
    pd, md, hd = (torch.from_numpy(x).to(dev) for x in (pos, m, h))
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev)
    pot = torch.empty(n, dtype=torch.float64, device=dev)
    out = {"n": n, "theta": wk["theta"], "leaf_size": wk["leaf_size"], "order": 2,
           "oracle": {"seconds": t_oracle, "particles_per_s": n / t_oracle, "cores": oracle.max_threads(),
                      "m2l": st_o["m2l"], "p2p_pairs": st_o["p2p_pairs"],
                      "acc_rel_vs_direct": _err_stats(np.linalg.norm(a_o - a_d, axis=1) / an)},
           "direct_seconds": t_direct}
    for prec in ("fp64", "fp32"):
        s = sfmm.Solver(local, prec, profile=1)
        ms, st = time_steps(torch, s, pd, md, hd, acc, pot, wk, wk["theta"], steps, 3, flush)
        s.close()
        a, p = acc.cpu().numpy(), pot.cpu().numpy()
        out[prec] = {"ms_per_step": float(np.mean(ms)), "particles_per_s": n / (np.mean(ms) * 1e-3),
                     "counts_equal_oracle": bool(st["m2l"] == st_o["m2l"] and st["p2p_pairs"] == st_o["p2p_pairs"]),
                     "acc_rel_vs_oracle": _err_stats(_acc_rel(a, a_o)),
                     "pot_rel_vs_oracle": _err_stats(np.abs(p - p_o) / np.abs(p_o)),
                     "acc_rel_vs_direct": _err_stats(np.linalg.norm(a - a_d, axis=1) / an),
                     "momentum_residual": float(np.linalg.norm(st["momentum"]) / st["abs_momentum"])}
    return out


M2L_FLOPS_P2 = 136       # FP32 M2L at p = 2 without the dipole terms (counted from the kernel source)
NCOEF_P2 = 10


def stage_rooflines(st, n, fp32_peak, hbm_peak):
    """Achieved fraction of each stage's roofline from live CUDA-event stage
    times: the build (which also forms the moments of the order in use)
    against HBM (algorithmic bytes), the walk (M2L) and P2P against the FP32
    FMA units (algorithmic flops)."""
    nn = st["nnodes"]
    b_build = n * (40 + 40 + 16) + nn * (16 + NCOEF_P2) * 8 + n * 32 + nn * (NCOEF_P2 + 4) * 8
    out = {}
    for key, ms, work, unit, peak in (
            ("build_and_moments", st["ms_build"] + st["ms_moments"], b_build / 1e9, "GB/s", hbm_peak),
            ("walk_m2l", st["ms_walk"], st["m2l_unique"] * M2L_FLOPS_P2 / 1e12, "TFLOP/s", fp32_peak),
            ("p2p", st["ms_p2p"], st["p2p_pairs"] * FLOPS_PER_PAIR / 1e12, "TFLOP/s", fp32_peak)):
        ach = work / (ms * 1e-3) if ms > 0 else 0.0
        out[key] = {"ms": ms, "achieved": ach, "unit": unit, "peak": peak, "frac": ach / peak}
    return out


def config_block(torch, local, flush, name, steps, fp32_peak, hbm_peak):
    """One more of the paper's workloads at its full size, FP32 form,
    theta 0.5, p 2, leaf 16: build + gravity per step (full pipeline) and
    gravity alone, the stage split and each stage's roofline fraction."""
    import workloads
    from paper_2602_05804_gb300 import sfmm

    wk = dict(workloads.WORKLOADS[name], order=2)
    t0 = time.perf_counter()
    pos, m, h = workloads.make(name)
    t_gen = time.perf_counter() - t0
    n = len(m)
    dev = torch.device("cuda", local)
    pd, md, hd = (torch.from_numpy(x).to(dev) for x in (pos, m, h))
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev)
    pot = torch.empty(n, dtype=torch.float64, device=dev)
    s = sfmm.Solver(local, "fp32", profile=1, walk=1)
    ms, st = time_steps(torch, s, pd, md, hd, acc, pot, wk, wk["theta"], steps, 2, flush)
    s.close()
    step = float(np.mean(ms))
    grav = st["ms_moments"] + st["ms_walk"] + st["ms_p2p"] + st["ms_reduce"]
    del pd, md, hd, acc, pot
    torch.cuda.empty_cache()
    return {"n": n, "theta": wk["theta"], "leaf_size": wk["leaf_size"], "form": "FP32", "steps": steps,
            "full_pipeline_particles_per_s": n / (step * 1e-3), "ms_per_step": step,
            "gravity_particles_per_s": n / (grav * 1e-3),
            "interactions_per_s": (st["p2p_pairs"] + st["m2l_unique"]) / (step * 1e-3),
            "counts": {"m2l_unique": st["m2l_unique"], "m2l_replicated": st["m2l"], "p2p_pairs": st["p2p_pairs"],
                       "nleaves": st["nleaves"], "nnodes": st["nnodes"]},
            "momentum_residual": float(np.linalg.norm(st["momentum"]) / st["abs_momentum"]),
            "stage_rooflines": stage_rooflines(st, n, fp32_peak, hbm_peak), "generate_s": t_gen}


def leapfrog_block(torch, local, orbits=20, steps_per_orbit=400, n=13000):
    """Gravity-only leapfrog of the orbiting binary polytrope (the gravity
    part of the binary test of Sect. 4): ~1.3e4 particles, 20 orbits at
    400 steps per orbit, records every 1% of the period; linear momentum
    drift and angular momentum fluctuation in both forms."""
    import workloads
    from paper_2602_05804_gb300 import sfmm

    pos, vel, m, h = workloads.binary_orbit(n, 1006)
    period = workloads.orbital_period()
    dt = period / steps_per_orbit
    nsteps = orbits * steps_per_orbit
    out = {"n": n, "orbits": orbits, "steps": nsteps, "dt": dt, "theta": 0.5, "order": 2, "leaf_size": 16}
    for prec in ("fp64", "fp32"):
        s = sfmm.Solver(local, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, rec = s.leapfrog(pos, vel, m, h, 16, 0.5, 2, dt, nsteps, record_every=steps_per_orbit // 100)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        s.close()
        scale = rec[:, 7].max()
        lz = rec[:, 6]
        out[prec] = {"ms_per_step": 1e3 * wall / nsteps,
                     "max_abs_linear_momentum": float(np.abs(rec[:, 1:4]).max()),
                     "max_linear_momentum_drift_rel": float(np.abs(rec[:, 1:4] - rec[0, 1:4]).max() / scale),
                     "angular_momentum_rel_std": float(np.std(lz) / abs(lz[0])),
                     "angular_momentum_rel_drift": float((lz[-1] - lz[0]) / abs(lz[0]))}
    return out


def accuracy_sweep_block(torch, local, n=100_000, thetas=None, trees=("morton",)):
    """Force accuracy against the direct sum (the opening-angle study of
    Sect. 4.1): Plummer and uniform spheres of 10^5 particles, theta from 0.1
    to 0.6 in steps of 0.05, p = 2, leaf 16; mean, maximum and 10th
    percentile of |a - a_direct| / |a_direct| over all particles, for both
    forms (the direct sum is the oracle's, on the host cores)."""
    import oracle
    import workloads
    from paper_2602_05804_gb300 import sfmm

    thetas = thetas or [round(0.1 + 0.05 * k, 2) for k in range(11)]
    out = {"n": n, "order": 2, "leaf_size": 16, "thetas": thetas}
    for prof, gen in (("plummer", workloads.plummer), ("uniform", workloads.uniform_sphere)):
        pos, m, h = gen(n, 1100 + len(prof))
        t0 = time.perf_counter()
        a_d, _ = oracle.direct(pos, m, h)
        t_direct = time.perf_counter() - t0
        an = np.linalg.norm(a_d, axis=1)
        res = {"direct_s": t_direct}
        for tree in trees:
            for prec in ("fp64", "fp32"):
                s = sfmm.Solver(local, prec)
                if tree != "morton":
                    s.set_option("tree", 1.0)
                s.build(pos, m, h, 16)
                rows = []
                for th in thetas:
                    acc, _ = s.gravity(th, 2, want_pot=False)
                    e = np.linalg.norm(acc.cpu().numpy() - a_d, axis=1) / an
                    rows.append([float(e.mean()), float(e.max()), float(np.percentile(e, 10))])
                s.close()
                res["%s_%s" % (tree, prec)] = {"mean": [r[0] for r in rows], "max": [r[1] for r in rows],
                                               "p10": [r[2] for r in rows]}
        out[prof] = res
    return out


def run_gpu(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import workloads
    from paper_2602_05804_gb300 import sfmm

    w = WORKLOAD
    wr = rank_workload(w, rank)
    pos, m, h = workloads.make(w["gen_name"], n=wr["n"], seed=wr["seed"])
    dev = torch.device("cuda", local)
    pos_d = torch.from_numpy(pos).to(dev)
    m_d = torch.from_numpy(m).to(dev)
    h_d = torch.from_numpy(h).to(dev)
    acc = torch.empty((w["n"], 3), dtype=torch.float64, device=dev)
    pot = torch.empty(w["n"], dtype=torch.float64, device=dev)
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    s32 = sfmm.Solver(local, "fp32", profile=1, walk=args.walk, schedule=args.schedule)
    s64 = sfmm.Solver(local, "fp64", profile=1, walk=args.walk, schedule=args.schedule)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.only == "fp64":
        ms64, st64 = time_steps(torch, s64, pos_d, m_d, h_d, acc, pot, w, w["theta"], args.steps, args.warmup, flush)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": w["n"] / (np.mean(ms64) * 1e-3), "unit": "particles/s",
                              "n_gpus": ws, "ms_per_step": float(np.mean(ms64)),
                              "stage_ms": {k: st64[k] for k in ("ms_build", "ms_moments", "ms_walk", "ms_p2p")},
                              "partial": "FP64 form step only (for profiler launch lists)"}))
        s32.close()
        s64.close()
        return 0
    barrier()
    with ClockSampler(local) as clk:
        # the step through the ordinary calls (sfmm_build + sfmm_gravity),
        # profiled: stage times, counts and results
        ms32, st32 = time_steps(torch, s32, pos_d, m_d, h_d, acc, pot, w, w["theta"], args.steps, args.warmup,
                                flush)
        ordinary_ms = float(np.mean(ms32))
        res_fp32 = (acc.cpu().numpy(), pot.cpu().numpy(), st32)
        inter = st32["p2p_pairs"] + st32["m2l_unique"]
        # headline: FP32 form, theta = 0.5, the same step captured as one CUDA
        # graph (sfmm_solve_graph, bitwise the same results), max over ranks
        barrier()
        t_wall0 = time.perf_counter()
        graph = graph_block(torch, local, pos_d, m_d, h_d, acc, pot, w, args.steps, flush, args.warmup)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    step_ms, n_all = reduce_timing(dist, graph["ms_per_step"], w["n"], dev)
    value = n_all / (step_ms * 1e-3)
    if args.only == "fp32":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws,
                              "ms_per_step": step_ms, "stage_ms": {k: st32[k] for k in ("ms_build", "ms_moments",
                                                                                         "ms_walk", "ms_p2p")},
                              "partial": "headline FP32 step only"}))
        s32.close()
        s64.close()
        return 0
    # FP64 form (same workload, fewer steps: it is ~50x slower)
    k64 = max(1, min(args.steps, 3))
    ms64, st64 = time_steps(torch, s64, pos_d, m_d, h_d, acc, pot, w, w["theta"], k64, 1, flush)
    fp64_ms = float(np.mean(ms64))
    res_fp64 = (acc.cpu().numpy(), pot.cpu().numpy(), st64)
    peaks_meas = measured_peaks(local, s32.stream.cuda_stream)
    # theta sweep of the FP32 form
    sweep = {}
    for th in (0.3, 0.7):
        ms_t, st_t = time_steps(torch, s32, pos_d, m_d, h_d, acc, pot, w, th, max(1, min(args.steps, 3)), 1, flush)
        sweep[str(th)] = {"particles_per_s": w["n"] / (np.mean(ms_t) * 1e-3),
                          "interactions_per_s": (st_t["p2p_pairs"] + st_t["m2l_unique"]) / (np.mean(ms_t) * 1e-3),
                          "ms_per_step": float(np.mean(ms_t)), "m2l": st_t["m2l"], "p2p_pairs": st_t["p2p_pairs"],
                          "stage_ms": {k[3:]: st_t[k] for k in ("ms_build", "ms_moments", "ms_walk", "ms_p2p")}}

    # the other walk on the same workload (same interactions, same results up
    # to summation order): the per-leaf replay of Algorithm 1 as printed, or the
    # per-node shared pairs
    other_mode = 0 if args.walk != 0 else 1
    other = sfmm.Solver(local, "fp32", profile=1, walk=other_mode)
    ms_o, st_o = time_steps(torch, other, pos_d, m_d, h_d, acc, pot, w, w["theta"], max(1, min(args.steps, 3)), 1,
                            flush)
    other.close()
    other_walk = {"walk": "per-leaf replay (Algorithm 1)" if other_mode == 0 else "per-node shared pairs",
                  "particles_per_s": ws * w["n"] / (np.mean(ms_o) * 1e-3), "ms_per_step": float(np.mean(ms_o)),
                  "stage_ms": {"build": st_o["ms_build"], "moments": st_o["ms_moments"], "walk": st_o["ms_walk"],
                               "p2p": st_o["ms_p2p"]},
                  "m2l": st_o["m2l"], "m2l_unique": st_o["m2l_unique"], "p2p_pairs": st_o["p2p_pairs"]}

    # one-sided symmetric pairs (walk mode 2): one D per pair for both sides
    sym = sfmm.Solver(local, "fp32", profile=1, walk=2)
    ms_s, st_s = time_steps(torch, sym, pos_d, m_d, h_d, acc, pot, w, w["theta"], max(1, min(args.steps, 3)), 1,
                            flush)
    sym.close()
    sym_walk = {"walk": "one-sided symmetric pairs (D once per pair, FP64 atomics to the partner)",
                "particles_per_s": ws * w["n"] / (np.mean(ms_s) * 1e-3), "ms_per_step": float(np.mean(ms_s)),
                "stage_ms": {"build": st_s["ms_build"], "moments": st_s["ms_moments"], "walk": st_s["ms_walk"],
                             "p2p": st_s["ms_p2p"]}}

    # the shared walk under its three node orders (bitwise the same results):
    # one launch per depth, one launch over a queue of nodes whose parent is
    # done, and the same over a queue of sibling pairs; the automatic choice
    # takes the node queue while the walk's per-node records take at most
    # twice the L2, else the pair queue
    schedules = {}
    for sched, label in ((1, "one launch per depth"), (2, "readiness queue of nodes"),
                         (3, "readiness queue of sibling pairs")):
        sq = sfmm.Solver(local, "fp32", profile=1, walk=1, schedule=sched)
        ms_q, st_q = time_steps(torch, sq, pos_d, m_d, h_d, acc, pot, w, w["theta"], max(1, min(args.steps, 3)), 1,
                                flush)
        sq.close()
        schedules[label] = {"ms_per_step": float(np.mean(ms_q)), "walk_ms": st_q["ms_walk"]}

    ensemble = None
    if not args.no_ensemble:
        ensemble = ensemble_block(torch, local, flush, max(1, min(args.steps, 5)))

    peaks, peak_kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_unit_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s, unit counts x max clock
    fp32_peak = peaks_meas["fp32_tflops"]
    fp64_peak = peaks_meas["fp64_tflops"]
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    leapfrog = None if args.no_leapfrog else leapfrog_block(torch, local)
    accuracy = None if args.no_accuracy else accuracy_sweep_block(torch, local, trees=("morton", "kd"))
    configs = None
    if not args.no_configs:
        configs = {name: config_block(torch, local, flush, name, max(1, min(args.steps, 5)), fp32_peak, hbm_peak)
                   for name in ("binary_polytrope_2e6", "clustered_1.6e7")}

    # e2e through the C ABI with HOST buffers (pinned), copies inside the region
    pos_h = torch.from_numpy(pos).pin_memory()
    m_h = torch.from_numpy(m).pin_memory()
    h_h = torch.from_numpy(h).pin_memory()
    acc_h = torch.empty((w["n"], 3), dtype=torch.float64).pin_memory()
    pot_h = torch.empty(w["n"], dtype=torch.float64).pin_memory()
    for _ in range(2):
        s32.solve_host(pos_h, m_h, h_h, w["leaf_size"], w["theta"], w["order"], acc_h, pot_h)
    ke = max(1, min(args.steps, 5))
    barrier()
    e2e_s = 0.0
    for _ in range(ke):
        _flush(flush)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s32.solve_host(pos_h, m_h, h_h, w["leaf_size"], w["theta"], w["order"], acc_h, pot_h)  # syncs
        e2e_s += time.perf_counter() - t1
    e2e_ms = 1e3 * e2e_s / ke
    if dist is not None:
        tt = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())

    fp64_tuned, res_fp64t = fp64_tuned_block(torch, local, pos_d, m_d, h_d, acc, pot, w, max(1, min(args.steps, 3)),
                                             flush)
    oracle_err = None
    if not args.no_oracle_error:
        oracle_err = oracle_error_block(pos, m, h, w, {"fp32": res_fp32 + (w["leaf_size"],),
                                                       "fp64": res_fp64 + (w["leaf_size"],),
                                                       "fp64_tuned_leaf": res_fp64t})
    small = None if args.no_configs else uniform_1e4_block(torch, local, flush, max(3, min(args.steps, 10)))

    # roofline of the dominant kernel
    clocks = clk.summary()
    shares = {"walk": st32["ms_walk"], "p2p": st32["ms_p2p"], "build": st32["ms_build"],
              "moments": st32["ms_moments"]}
    if st32["ms_p2p"] >= st32["ms_walk"]:
        kname, kms = "k_p2p<FP32>", st32["ms_p2p"]
        achieved = st32["p2p_pairs"] * FLOPS_PER_PAIR / (kms * 1e-3) / 1e12
        src = _kernel_hash("p2p.cu")
    else:
        # the walk evaluates every unique pair once (shared) or once per leaf (replay)
        nm2l = st32["m2l_unique"] if args.walk >= 1 else st32["m2l"]
        kname = "k_walk_level<2,FP32>" if args.walk >= 1 else "k_walk<2,FP32>"
        kms = st32["ms_walk"]
        achieved = nm2l * 136 / (kms * 1e-3) / 1e12
        src = _kernel_hash("walk_shared.cu" if args.walk >= 1 else "walk.cu", "walk_common.cuh", "expansion_gen.cuh")
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": _traffic(kname, src),
            "peak_source": "measured: FP32 FMA throughput of sfmm_fma_peak in this run (max of scalar and packed)",
            "peak_unit_count": fp32_unit_peak, "frac_of_unit_count": achieved / fp32_unit_peak,
            "ms_per_launch": kms, "stage_ms": shares,
            "work": ({"p2p_pairs": st32["p2p_pairs"], "flops_per_pair": FLOPS_PER_PAIR}
                     if kname.startswith("k_p2p") else {"m2l": nm2l, "flops_per_m2l": M2L_FLOPS_P2})}
    p64_ach = st64["p2p_pairs"] * FLOPS_PER_PAIR / (st64["ms_p2p"] * 1e-3) / 1e12
    roof64 = {"kernel": "k_p2p<FP64>", "bound": "alu", "achieved": p64_ach, "peak": fp64_peak, "unit": "TFLOP/s",
              "frac": p64_ach / fp64_peak, "traffic": _traffic("k_p2p<FP64>", _kernel_hash("p2p.cu")),
              "peak_source": "measured: FP64 FMA throughput of sfmm_fma_peak in this run",
              "ms_per_launch": st64["ms_p2p"],
              "work": {"p2p_pairs": st64["p2p_pairs"], "flops_per_pair": FLOPS_PER_PAIR},
              "stage_ms": {"walk": st64["ms_walk"], "p2p": st64["ms_p2p"], "build": st64["ms_build"],
                           "moments": st64["ms_moments"]}}

    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded %s, one per rank)" % w["gen_name"],
        "config": {"workload": w["name"], "n": w["n"], "theta": w["theta"], "order": w["order"],
                   "leaf_size": w["leaf_size"], "form": "FP32 (FP64 centres, decisions, reductions)",
                   "walk": {0: "per-leaf replay (Algorithm 1)", 1: "per-node shared pairs",
                            2: "one-sided symmetric pairs"}[args.walk],
                   "schedule": {0: "automatic", 1: "one launch per depth", 2: "readiness queue of nodes",
                                3: "readiness queue of sibling pairs"}[args.schedule],
                   "l2": "flushed between timed steps (512 MB write outside the events)",
                   "path": "sfmm_solve_graph: build + gravity replayed as one captured CUDA graph"},
        "interactions_per_s": ws * inter / (step_ms * 1e-3),
        "counts": {"m2l_replicated": st32["m2l"], "m2l_unique": st32["m2l_unique"],
                   "p2p_pairs": st32["p2p_pairs"], "p2p_leaf_pairs": st32["p2p_leaves"],
                   "mac_fallbacks": st32["mac_fallbacks"], "nleaves": st32["nleaves"]},
        "fp64_form": {"particles_per_s": ws * w["n"] / (fp64_ms * 1e-3), "ms_per_step": fp64_ms,
                      "speedup_fp32_over_fp64": fp64_ms / step_ms,
                      "speedup_at": ("same theta, p and tree: equal force accuracy, since both forms share the "
                                     "truncation error against the direct sum (oracle_error.*.acc_rel_vs_direct)"),
                      "tuned_leaf": dict(fp64_tuned, speedup_fp32_over_fp64=fp64_tuned["ms_per_step"] / step_ms,
                                         acc_rel_vs_direct_mean=(None if oracle_err is None else
                                                                 oracle_err["fp64_tuned_leaf"]["acc_rel_vs_direct"][
                                                                     "mean"])),
                      "acc_rel_vs_direct_mean": (None if oracle_err is None else
                                                 {f: oracle_err[f]["acc_rel_vs_direct"]["mean"]
                                                  for f in ("fp32", "fp64")}),
                      "stage_ms": {"walk": st64["ms_walk"], "p2p": st64["ms_p2p"], "build": st64["ms_build"]}},
        "momentum_residual": {"fp32": float(np.linalg.norm(st32["momentum"]) / st32["abs_momentum"]),
                              "fp64": float(np.linalg.norm(st64["momentum"]) / st64["abs_momentum"])},
        "theta_sweep_fp32": sweep,
        "other_walk_fp32": other_walk,
        "symmetric_walk_fp32": sym_walk,
        "walk_schedules_fp32": schedules,
        "graph_step_fp32": graph,
        "ordinary_calls_fp32": {"ms_per_step": ordinary_ms, "particles_per_s": ws * w["n"] / (ordinary_ms * 1e-3),
                                "how": "sfmm_build + sfmm_gravity per step (two host synchronisations); the "
                                       "stage times, counts and rooflines come from this run"},
        "ensemble_256": ensemble,
        "stage_rooflines": stage_rooflines(st32, w["n"], fp32_peak, hbm_peak),
        "configs": configs,
        "leapfrog_binary": leapfrog,
        "accuracy_sweep": accuracy,
        "e2e": {"value": ws * w["n"] / (e2e_ms * 1e-3), "unit": "particles/s",
                "h2d_bytes_per_step": int(w["n"] * 40), "d2h_bytes_per_step": int(w["n"] * 32)},
        "gpu_launches": int(round(graph["kernels_per_step"] * args.steps)),
        "roofline": roof,
        "roofline_fp64": roof64,
        "measured_peaks": peaks_meas,
        "oracle_error": oracle_err,
        "uniform_1e4": small,
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(pos, m, h, w)
    if rank == 0:
        print(json.dumps(line))
    s32.close()
    s64.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble measurement")
    ap.add_argument("--no-leapfrog", action="store_true", help="skip the 20-orbit binary leapfrog")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the theta sweep against the direct sum")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the binary-polytrope (2e6) and clustered-cloud (1.6e7) measurements")
    ap.add_argument("--workload", default="plummer_1e6",
                    choices=["plummer_1e6", "uniform_1e4", "binary_polytrope_2e6", "clustered_1.6e7"],
                    help="headline workload (default: the 10^6 Plummer sphere; the others are for profiling)")
    ap.add_argument("--n", type=int, default=None, help="particle count (default: the workload's 10^6)")
    ap.add_argument("--leaf", type=int, default=None, help="leaf size (default: the workload's 16)")
    ap.add_argument("--walk", type=int, default=1, choices=[0, 1, 2],
                    help="headline walk: 1 per-node shared pairs (default), 0 per-leaf replay (Algorithm 1), "
                         "2 one-sided symmetric pairs")
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 1, 2, 3],
                    help="walk 1 node order: 0 automatic (default), 1 one launch per depth, 2 readiness queue of "
                         "nodes, 3 readiness queue of sibling pairs")
    ap.add_argument("--only", default="all", choices=["all", "fp32", "fp64"],
                    help="fp32 / fp64: time the headline step of that form only (for profiler launch lists)")
    ap.add_argument("--no-oracle-error", action="store_true",
                    help="skip the per-result error against the oracle and the direct sum")
    args = ap.parse_args()
    if args.workload != "plummer_1e6":
        import workloads

        wk = workloads.WORKLOADS[args.workload]
        WORKLOAD.update(name=args.workload, gen_name=args.workload, n=wk["n"], seed=wk["seed"],
                        theta=wk["theta"], leaf_size=wk["leaf_size"])
    if args.leaf:
        WORKLOAD["leaf_size"] = int(args.leaf)
    if args.n:
        WORKLOAD["n"] = int(args.n)
        WORKLOAD["name"] = "%s_n%d" % (WORKLOAD["gen_name"].split("_")[0], args.n)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
