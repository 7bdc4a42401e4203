"""Benchmark of the batched tuning workload: 10,000 kernel variants drawn from the
tuning space over eight templates, 4,096 log-uniform parameter points per
template, every (variant, point) pair evaluated (exact int64 counts), predicted
(FP64-accurate) and ranked (top-16 per point) in one persistent launch.

One step = one pass of that whole path over the batch.  Prints one JSON line.
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank ranks its own point batch of the same size (weak
scaling; rank r draws its points with seed 3 + 7919 r); no data-path collective, the
process group only brackets the timing (barrier, max over ranks).
Other workloads: --workload eval | predict | fit | serve | calibrate | coupled
(coupled: the same fused path over the coupled-domain templates, triangles and bands).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "model evals/s (variant x param points), fused evaluate+predict+top-16"
UNIT = "evals/s"
WORKLOAD = "batched tuning space: 10,000 variants x 4,096 points per template, 8 templates, top-16, FP64-accurate"
DTYPE = "int64 counts, exact fixed-point (128-bit) predict, fp64 out"
WORKLOAD_COUPLED = ("coupled-domain tuning space (triangular matvec, syrk, band matvec, pair interactions): "
                    "10,000 variants x 4,096 points per template, 4 templates, top-16, FP64-accurate")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        def run():
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                         timeout=5).stdout.strip()
                    if out:
                        self.rows.append([x.strip() for x in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": sorted(reasons)}


def _oracle_sample(bp, w, target_s: float):
    """Time the oracle (structural counts + compensated dot + insertion top-16), as it
    stands, on all host cores, on a bounded sample of the workload: the first v
    variants and the first n points of every template, grown from 8 variants x 2 points
    per core (variants first, then points) until a pass takes at least half of target_s.
    Returns (evals/s, cores, v, n, evals, seconds)."""
    import numpy as np

    import oracle
    from paper_1604_04997_gb300 import workloads as W
    cores = os.cpu_count() or 1
    kern = {}
    per_t = []
    for ti, t in enumerate(bp.templates):
        ks = []
        for v in bp.variants[bp.var_off[ti]:bp.var_off[ti + 1]]:
            if v.key not in kern:
                kern[v.key] = oracle.Kernel(W.variant_ir(v))
            ks.append(kern[v.key])
        per_t.append(ks)

    def run(nv, n):
        evals = 0
        t0 = time.perf_counter()
        for ti, t in enumerate(bp.templates):
            ks = per_t[ti][:nv]
            if not ks:
                continue
            P = len(W.TEMPLATE_PARAMS[t])
            p0 = int(bp.pt_off[ti])
            pts = np.ascontiguousarray(bp.points[p0:p0 + n, :P])
            oracle.eval_predict_topk(ks, pts, w, 16, n_threads=cores)
            evals += len(ks) * len(pts)
        return evals, time.perf_counter() - t0

    vmax = max(len(k) for k in per_t)
    nv, n = 8, min(4096, 2 * cores)   # enough points to occupy every core
    while True:
        ev, dt = run(nv, n)
        if dt >= 0.5 * target_s or (nv >= vmax and n >= 4096):
            break
        grow = target_s / max(dt, 1e-3) * 1.1
        if nv < vmax:
            nv = min(vmax, max(nv * 2, int(nv * grow)))
        else:
            n = min(4096, max(n * 2, int(n * grow)))
    return ev / dt, cores, nv, n, ev, dt


def _sample_text(bp, nv, n, ev, dt):
    vmax = max(bp.var_off[t + 1] - bp.var_off[t] for t in range(len(bp.templates)))
    which = f"all {len(bp.variants)} variants" if nv >= vmax else f"the first {nv} variants of each template"
    return f"{which} x first {n} points of each template ({ev} evals, {dt:.1f} s, OpenMP over points)"


def cpu_baseline(bp, w, target_s: float = 8.0):
    value, cores, nv, n, ev, dt = _oracle_sample(bp, w, target_s)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": _sample_text(bp, nv, n, ev, dt)}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1604_04997_gb300 import workloads as W
    # the oracle alone: the workload comes from the seeded generators, nothing of the
    # CUDA library is built or loaded on this path
    oracle.build()
    coupled = args.workload == "coupled"
    bp = W.batched_space(args.variants, args.points, variant_seed=12 if coupled else 2, coupled=coupled)
    w = W.draw_weights(32, 1, 4)[0]
    # each step: the bounded sample that the probe sizes to about ref_step_s
    _, cores, n_var, n_pts, ev0, dt0 = _oracle_sample(bp, w, args.ref_step_s)
    base = {"cores": cores, "sample": _sample_text(bp, n_var, n_pts, ev0, dt0)}
    kern, per_t = {}, []
    for ti, t in enumerate(bp.templates):
        ks = []
        for v in bp.variants[bp.var_off[ti]:bp.var_off[ti + 1]][:n_var]:
            if v.key not in kern:
                kern[v.key] = oracle.Kernel(W.variant_ir(v))
            ks.append(kern[v.key])
        per_t.append(ks)

    def step():
        ev = 0
        for ti, t in enumerate(bp.templates):
            if per_t[ti]:
                P = len(W.TEMPLATE_PARAMS[t])
                p0 = int(bp.pt_off[ti])
                pts = np.ascontiguousarray(bp.points[p0:p0 + n_pts, :P])
                oracle.eval_predict_topk(per_t[ti], pts, w, 16, n_threads=base["cores"])
                ev += len(per_t[ti]) * len(pts)
        return ev

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    ev = 0
    for _ in range(args.steps):
        ev += step()
    dt = time.perf_counter() - t0
    value = ev / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
            "config": {"workload": WORKLOAD_COUPLED if coupled else WORKLOAD,
                       "reference_note": "the CPU oracle, timed on a bounded sample of the workload per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _plain_form(ctx, bp, d_w, dev, stream, fused_idx, reps=2):
    """The plain per-call form of the same (variant, point) pairs: per template, one
    pm_eval_counts into int64 [variants][points][32], then one pm_predict_topk of the
    FP64-accurate times with the per-point row list (group p = the rows v * n + p).
    Returns timings (ms per pass over all templates) and the share of points whose
    top-16 variant list equals the fused launch's."""
    import numpy as np
    import torch
    from paper_1604_04997_gb300 import workloads as W
    calls = []
    for t in range(len(bp.templates)):
        ids = bp.tables[bp.var_off[t]:bp.var_off[t + 1]]
        nv, n = len(ids), int(bp.pt_off[t + 1] - bp.pt_off[t])
        if nv == 0 or n == 0:
            continue
        P = len(W.TEMPLATE_PARAMS[bp.templates[t]])
        pts = torch.from_numpy(np.ascontiguousarray(bp.points[bp.pt_off[t]:bp.pt_off[t + 1], :P])).to(dev)
        F = torch.empty((nv, n, 32), dtype=torch.int64, device=dev)
        rows = torch.from_numpy((np.arange(nv, dtype=np.int64)[None, :] * n +
                                 np.arange(n, dtype=np.int64)[:, None]).reshape(-1)).to(dev)
        seg = np.arange(n + 1, dtype=np.int64) * nv
        ti = torch.empty(n * 16, dtype=torch.int64, device=dev)
        tt = torch.empty(n * 16, dtype=torch.float64, device=dev)
        calls.append((t, ids, pts, F, rows, seg, ti, tt, n))
    W1 = d_w.view(1, 32)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in calls]

    def run(timed):
        for (t, ids, pts, F, rows, seg, ti, tt, n), e in zip(calls, ev):
            if timed:
                e[0].record(stream)
            ctx.eval_counts(ids, pts, F, stream=stream)
            if timed:
                e[1].record(stream)
            ctx.predict_topk(F.view(-1, 32), W1, seg, 16, ti, tt, rows=rows, stream=stream)
            if timed:
                e[2].record(stream)

    with torch.cuda.stream(stream):
        run(False)
    torch.cuda.synchronize()
    eval_ms = rank_ms = 0.0
    for _ in range(reps):
        with torch.cuda.stream(stream):
            run(True)
        torch.cuda.synchronize()
        eval_ms += sum(e[0].elapsed_time(e[1]) for e in ev) / reps
        rank_ms += sum(e[1].elapsed_time(e[2]) for e in ev) / reps
    ctx.sync_status(stream)
    same = total = 0
    fi = fused_idx.cpu().numpy()
    for t, ids, pts, F, rows, seg, ti, tt, n in calls:
        plain_v = (ti.cpu().numpy().reshape(n, 16) // n).astype(np.int64)
        fv = fi[bp.pt_off[t]:bp.pt_off[t + 1]].astype(np.int64)
        same += int((plain_v == fv).all(axis=1).sum())
        total += n
    del calls
    torch.cuda.empty_cache()
    return {"ms": eval_ms + rank_ms, "eval_counts_ms": eval_ms, "predict_topk_ms": rank_ms,
            "points_with_identical_top16": same / max(1, total),
            "note": "per template: pm_eval_counts (all 32 counts to HBM, 10.5 GB) then pm_predict_topk "
                    "(PM_PREC_FP64, one model, per-point row lists; one row per lane for M <= 8): "
                    "the same exact arithmetic and ranking as the fused launch"}


def _serve_summary(ctx, bp, n_points, n_q):
    """A short autotuner query stream on the batched workload's tables and points:
    Poisson arrivals at 2,000 queries/s (1-50,000 candidates each, log-uniform), one of
    64 resident models per query, top-16 per query, host buffers in and out; then the
    first 200 of the same queries served one at a time."""
    from paper_1604_04997_gb300 import tuning
    from paper_1604_04997_gb300 import workloads as W
    ctx.serve_set_weights(W.draw_weights(32, 64, 4))
    nv = [int(bp.var_off[t + 1] - bp.var_off[t]) for t in range(len(bp.templates))]
    qs = W.draw_queries(n_q, 2000.0, nv, n_points, 64, 9, 50000)
    arrays = [tuning.query_arrays(bp, q) for q in qs]
    wall, st = _serve_stream(ctx, bp, qs, arrays, 200)
    n1 = min(200, n_q)
    wall1, st1 = _serve_stream(ctx, bp, qs[:n1], arrays[:n1], 0, sync=True)
    cand = sum(len(q.variant) for q in qs)
    cand1 = sum(len(q.variant) for q in qs[:n1])
    return {"queries": n_q, "rate_per_s": 2000.0, "batch_interval_us": 200, "p50_us": round(st["p50_us"], 1),
            "p99_us": round(st["p99_us"], 1), "max_us": round(st["max_us"], 1),
            "served_evals_per_s": cand / wall, "offered_evals_per_s": cand / qs[-1].arrival_s,
            "queries_per_batch": round(st["n_queries"] / max(1, st["n_batches"]), 2),
            "one_at_a_time_evals_per_s": cand1 / wall1, "one_at_a_time_p50_us": round(st1["p50_us"], 1),
            "latency_note": "submit to results in the caller's host buffers, measured in the library"}


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1604_04997_gb300 import binding as B
    from paper_1604_04997_gb300 import sharding
    from paper_1604_04997_gb300 import tuning
    from paper_1604_04997_gb300 import workloads as W

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    __graft_entry__.build()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ctx = B.Context(local)
    ctx.tune(not args.no_tune, args.tune_cache)
    # weak scaling: every rank ranks its own point batch (independent units, no exchange)
    coupled = args.workload == "coupled"
    bp = tuning.build(ctx, args.variants, args.points, point_seed=sharding.rank_point_seed(3, rank),
                      variant_seed=12 if coupled else 2, coupled=coupled)
    w = W.draw_weights(32, 1, 4)[0]
    n = bp.points.shape[0]
    stream = torch.cuda.Stream(dev)
    d_pts = torch.from_numpy(bp.points).to(dev)
    d_w = torch.from_numpy(w).to(dev)
    idx = torch.empty((n, 16), dtype=torch.int32, device=dev)
    tt = torch.empty((n, 16), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)   # 256 MB > L2

    def step(s):
        ctx.eval_predict_topk(bp.tables, bp.var_off, d_pts, bp.pt_off, d_w, 16, idx, tt, stream=s)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step(stream)
    torch.cuda.synchronize()
    ctx.sync_status(stream)
    info = ctx.plan_info(bp.tables, bp.var_off, bp.pt_off)
    tuning = _tuning_summary(ctx, bp)

    clocks = Clocks(local)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()                                   # L2 flush between timed steps (not timed)
            ev0[i].record(stream)
            step(stream)
            ev1[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ck = clocks.stop()
    ctx.sync_status(stream)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    ms = sum(step_ms) / len(step_ms)
    ms = sharding.max_over_ranks(ms, dev)
    if ws > 1:
        torch.distributed.barrier()

    # end to end through the C ABI with host buffers: points H2D, ranking D2H, every step
    h_pts = torch.from_numpy(bp.points).pin_memory()
    h_idx = torch.empty((n, 16), dtype=torch.int32).pin_memory()
    h_t = torch.empty((n, 16), dtype=torch.float64).pin_memory()
    e_steps = max(3, args.steps)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for i in range(e_steps):
            d_pts.copy_(h_pts, non_blocking=True)
            step(stream)
            h_idx.copy_(idx, non_blocking=True)
            h_t.copy_(tt, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e_steps
    e2e_ms = sharding.max_over_ranks(e2e_ms, dev)

    evals = bp.total_evals
    value = evals * ws / (ms / 1e3)
    plain = serve = None
    if not args.no_plain:
        plain = _plain_form(ctx, bp, d_w, dev, stream, idx)
        plain["vs_plain"] = plain["ms"] / ms
    if not args.no_serve and rank == 0:
        serve = _serve_summary(ctx, bp, args.points, args.serve_queries)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sms * 128 * max_mhz * 1e6           # lane-instruction issue rate at the maximum clock
    achieved = evals * info["work_per_eval"] / (ms / 1e3)
    measured_ops = B.pmm_int_issue_rate()          # integer multiply-add / xor / add chains, every lane
    traffic = _profile_traffic("rank_coupled_10000x4096.md" if coupled else
                               "rank_batched_10000x4096.md",
                               ("rank.cu", "eval_common.cuh", "kernels.h", "plan.cpp"))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE,
            "data": "synthetic",
            "config": {"workload": WORKLOAD_COUPLED if coupled else WORKLOAD, "variants": len(bp.variants),
                       "distinct_variants": bp.n_distinct,
                       "points_per_template": args.points, "evals_per_step": evals, "topk": 16,
                       "l2": "flushed (256 MB write) before every timed step",
                       "launch": {"warps_per_cta": info["nw"], "ctas": info["grid"], "units": info["units"],
                                  "ranking_groups": info["groups"], "slice": info["slice"] or None,
                                  "tuned": info["tuned"], "tuning": tuning},
                       "timed_region_wall_ms": wall * 1e3,
                       "plain_form": plain, "vs_plain": plain["vs_plain"] if plain else None,
                       "serve": serve},
            "e2e": {"value": evals * ws / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(bp.points.nbytes),
                    "d2h_bytes_per_step": int(n * 16 * (4 + 8))},
            "gpu_launches": 2 * args.steps,   # per step: the weight prepass and the fused ranking kernel
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T lane-ops/s", "frac": achieved / peak_ops, "traffic": traffic,
                         "kernel": "k_rank",
                         "ops_per_eval": info["work_per_eval"],
                         "peak_note": f"{sms} SMs x 128 lanes x {max_mhz:.0f} MHz (issue bound, derived)",
                         "measured_peak": measured_ops / 1e12, "frac_of_measured": achieved / measured_ops,
                         "measured_peak_note": "integer issue-rate probe (pmm_int_issue_rate): independent "
                                               "32-bit multiply-add, xor and add chains in every lane"},
            "clocks": ck,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(bp, w, target_s=args.cpu_s)
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def _clocks_and_time(fn, steps, warmup, stream, flush=None):
    """Warm up, then time `steps` calls of fn with CUDA events on `stream`; returns
    (mean ms, clock summary).  With `flush` (a buffer larger than L2) each call is
    timed alone after the buffer is rewritten; without it (inputs larger than L2)
    the calls are queued back to back between two events, so host launch latency
    does not enter the device time."""
    import torch
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    ck = Clocks(torch.cuda.current_device())
    ck.start()
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, ck.stop()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.zero_()
            ev0[i].record(stream)
            fn()
            ev1[i].record(stream)
    torch.cuda.synchronize()
    c = ck.stop()
    return sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)) / steps, c


def _tuning_summary(ctx, bp):
    """The autotuner's candidates for this plan, the default launch shape's time and
    the chosen one's (None when the shape came from a tuning cache or tuning is off)."""
    try:
        log = ctx.plan_tune_log(bp.tables, bp.var_off, bp.pt_off)
        if not log:
            return None
        default = [r for r in log if r[0] >= 2 ** 30 and int(r[1]) == 8]
        best = min(log, key=lambda r: r[3])
        return {"candidates": len(log),
                "default_shape_ms": max(default, key=lambda r: r[2])[3] if default else None,
                "chosen_shape_ms": best[3],
                "chosen": {"variants_per_unit": None if best[0] >= 2 ** 30 else int(best[0]),
                           "warps_per_cta": int(best[1]), "ctas_per_sm": int(best[2])}}
    except Exception:
        return None


def _profile_traffic(md: str, sources) -> "int | None":
    """DRAM bytes per launch recorded in a committed ncu summary under profiles/, or
    None when the kernel's sources changed since the capture (fingerprint mismatch)."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", md)).read()
        t = int(re.search(r"^traffic_bytes_per_launch: (\d+)", text, re.M).group(1))
        want = re.search(r"^source_sha256_16: ([0-9a-f]{16})", text, re.M).group(1)
        csrc = os.path.join(ROOT, "paper_1604_04997_gb300", "csrc")
        h = hashlib.sha256(b"".join(open(os.path.join(csrc, f), "rb").read() for f in sources)).hexdigest()[:16]
        return t if h == want else None
    except Exception:
        return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_other(args):
    """Secondary workloads (one JSON line each): materialised counts, cross-model
    prediction, weight fit."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1604_04997_gb300 import binding as B
    from paper_1604_04997_gb300 import tuning
    from paper_1604_04997_gb300 import workloads as W
    __graft_entry__.build()
    dev = torch.device("cuda:0")
    ctx = B.Context(0)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    hbm = float(_peaks().get("hbm_gbs", 6790.0))
    base = {"n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "gpu_launches": None}
    if args.workload == "eval":
        bp = tuning.build(ctx, args.variants, args.points)
        outs, calls = [], []
        for t in range(len(bp.templates)):
            ids = bp.tables[bp.var_off[t]:bp.var_off[t + 1]]
            P = len(W.TEMPLATE_PARAMS[bp.templates[t]])
            pts = torch.from_numpy(np.ascontiguousarray(bp.points[bp.pt_off[t]:bp.pt_off[t + 1], :P])).to(dev)
            out = torch.empty((len(ids), pts.shape[0], 32), dtype=torch.int64, device=dev)
            calls.append((ids, pts, out))
        def fn():
            for ids, pts, out in calls:
                ctx.eval_counts(ids, pts, out, stream=stream)
        ms, ck = _clocks_and_time(fn, args.steps, args.warmup, stream, flush)
        ctx.sync_status(stream)
        evals = bp.total_evals
        nbytes = evals * 32 * 8 + sum(int(c[1].numel()) * 8 * len(c[0]) for c in calls)
        line = dict(base, metric="materialised count evaluations/s (pm_eval_counts, int64 [tables][points][32])",
                    value=evals / (ms / 1e3), unit="evals/s", ms_per_step=ms, higher_is_better=True, dtype="int64",
                    config={"workload": "10,000 variants x 4,096 points per template, all 32 counts written",
                            "bytes_per_step": nbytes, "l2": "flushed before every timed step"},
                    roofline={"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": nbytes / (ms / 1e3) / 1e9 / hbm, "traffic": None, "kernel": "k_eval_counts",
                              "algorithmic_bytes": "256 B of counts written per evaluation + 8 B per parameter read"},
                    clocks=ck, gpu_launches=len(calls) * args.steps)
    elif args.workload == "predict":
        R, M = 1_000_000, 64
        F = torch.from_numpy(W.fit_features(R, 32, 7)).to(dev)
        Wm = torch.from_numpy(W.draw_weights(32, M, 8)).to(dev)
        T = torch.empty((R, M), dtype=torch.float64, device=dev)
        arg = torch.empty(M, dtype=torch.int64, device=dev)
        mn = torch.empty(M, dtype=torch.float64, device=dev)
        n_groups = 4096
        idx16 = torch.empty(n_groups * M * 16, dtype=torch.int64, device=dev)
        t16 = torch.empty(n_groups * M * 16, dtype=torch.float64, device=dev)
        seg_one = np.array([0, R], dtype=np.int64)
        seg_many = np.linspace(0, R, n_groups + 1).astype(np.int64)
        times = {}
        for name, prec, fn in (
                ("bf16x3_T", B.PREC_BF16X3, lambda: ctx.predict(F, Wm, T, B.PREC_BF16X3, stream=stream)),
                ("bf16x3_argmin", B.PREC_BF16X3,
                 lambda: ctx.predict_argmin(F, Wm, arg, mn, B.PREC_BF16X3, stream=stream)),
                ("fp64_T", B.PREC_FP64, lambda: ctx.predict(F, Wm, T, B.PREC_FP64, stream=stream)),
                ("fp64_topk16_one_group", B.PREC_FP64,
                 lambda: ctx.predict_topk(F, Wm, seg_one, 16, idx16, t16, stream=stream)),
                ("fp64_topk16_4096_groups", B.PREC_FP64,
                 lambda: ctx.predict_topk(F, Wm, seg_many, 16, idx16, t16, stream=stream))):
            times[name] = _clocks_and_time(fn, args.steps, args.warmup, stream, None)   # F, T > L2
        ms, ck = times["bf16x3_T"]
        nbytes = R * 32 * 8 + R * M * 8
        nb_arg = R * 32 * 8
        ms_arg = times["bf16x3_argmin"][0]
        line = dict(base, metric="cross-model predictions/s (1e6 rows x 32 features x 64 models, tensor cores)",
                    value=R * M / (ms / 1e3), unit="predictions/s", ms_per_step=ms, higher_is_better=True,
                    dtype="bf16 x3-term split, fp32 accumulate (tcgen05), fp64 output",
                    config={"workload": "1,000,000 feature rows x 32 int64 features x 64 weight vectors",
                            "bytes_per_step": nbytes, "l2": "inputs (256 MB) and output (512 MB) larger than L2",
                            "argmin_only_ms": ms_arg, "argmin_only_gbs": nb_arg / (ms_arg / 1e3) / 1e9,
                            "fp64_accurate_ms": times["fp64_T"][0],
                            # the exact path's integer work: ten 32-bit multiply-adds per 64 x 64-bit product
                            "fp64_accurate_frac_of_lane_op_peak":
                                R * M * 32 * 10 / (times["fp64_T"][0] / 1e3) /
                                (torch.cuda.get_device_properties(dev).multi_processor_count * 128 *
                                 float(_peaks().get("sm_max_mhz", 2070.0)) * 1e6),
                            "fp64_accurate_top16_ms": {"one group of 1e6 rows": times["fp64_topk16_one_group"][0],
                                                       "4096 groups of ~244 rows":
                                                           times["fp64_topk16_4096_groups"][0]}},
                    roofline={"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": nbytes / (ms / 1e3) / 1e9 / hbm,
                              "traffic": _profile_traffic("predict_tc_1e6x32x64.md", ("predict_tc.cu", "mbar_wait.cuh")),
                              "kernel": "k_predict_tc",
                              "algorithmic_bytes": "256 B read + 8 B written per (row, model)"},
                    clocks=ck, gpu_launches=args.steps)
    elif args.workload == "fit":
        R, M = 200_000, 64
        Fh = W.fit_features(R, 32, 5)
        Th = W.synth_timings(Fh, W.draw_weights(32, M, 6), 6)
        F = torch.from_numpy(Fh).to(dev)
        T = torch.from_numpy(Th).to(dev)
        Wo = torch.empty((M, 32), dtype=torch.float64, device=dev)
        fn = lambda: ctx.fit_weights(F, T, Wo, B.FIT_RELATIVE, B.PREC_BF16X3, 3, stream=stream)
        ms, ck = _clocks_and_time(fn, args.steps, args.warmup, stream, None)
        fn_ff = lambda: ctx.fit_weights(F, T, Wo, B.FIT_RELATIVE, B.PREC_FP64, 3, stream=stream)
        ms_ff, _ = _clocks_and_time(fn_ff, max(2, args.steps // 2), args.warmup, stream, None)
        peak_tc = float(_peaks().get("bf16_tflops", 1979.0))
        gram_flops = 2.0 * 32 * 32 * R * M          # the 64 Gram matrices' useful flops
        line = dict(base, metric="weight fits/s (200,000 rows x 32 features, 64 models, 3 refinement steps)",
                    value=M / (ms / 1e3), unit="model fits/s", ms_per_step=ms, higher_is_better=True,
                    dtype="Gram on tcgen05 from three bf16 terms of A, fp32 accumulation per 4096-row chunk "
                          "(exact bf16-digit Gram if refinement stalls), FP64 Cholesky, exact residual products",
                    config={"workload": "200,000 x 32 int64 features, 64 device models, relative objective",
                            "float_float_gram_ms_per_step": ms_ff},
                    roofline={"bound": "tensor", "achieved": gram_flops / (ms / 1e3) / 1e12, "peak": peak_tc,
                              "unit": "TFLOP/s", "frac": gram_flops / (ms / 1e3) / 1e12 / peak_tc, "traffic": None,
                              "kernel": "pm_fit_weights (whole call; the Gram kernel is a third of it)",
                              "note": "useful Gram flops 2 k^2 R M over the whole fit; the three-term split "
                                      "executes 9 bf16 term-pair products (one 128 x 96 MMA tile) per useful product"},
                    clocks=ck, gpu_launches=None)
    print(json.dumps(line))
    ctx.close()


def _serve_stream(ctx, b, qs, arrays, interval_us, sync=False):
    """Submit qs at their arrival times (or one at a time, waiting for each, if sync)
    and wait for all; returns (wall seconds, library latency stats)."""
    import numpy as np
    from paper_1604_04997_gb300 import binding as B
    outs = [(np.empty(16, dtype=np.int32), np.empty(16)) for _ in qs]
    ctx.serve_start(batch_interval_us=interval_us, n_streams=2, max_batch_queries=256)
    try:
        for i in range(min(16, len(qs))):   # warm-up: first launches, pinned pages
            (tb, pt), (oi, ot) = arrays[i], outs[i]
            tk = ctx.serve_submit(B.make_query(qs[i].model, 16, tb, pt, oi, ot))
            while ctx.serve_poll(tk, 100000) == B.PM_PENDING:
                pass
        ctx.serve_stats(reset=True)
        deadline = time.perf_counter() + 120.0
        t0 = time.perf_counter()
        tickets = []
        for q, (tb, pt), (oi, ot) in zip(qs, arrays, outs):
            if sync:
                tk = ctx.serve_submit(B.make_query(q.model, 16, tb, pt, oi, ot))
                while ctx.serve_poll(tk, 100000) == B.PM_PENDING:
                    assert time.perf_counter() < deadline, "serve stream did not finish"
                continue
            while time.perf_counter() - t0 < q.arrival_s:
                pass
            tickets.append(ctx.serve_submit(B.make_query(q.model, 16, tb, pt, oi, ot)))
        for tk in tickets:
            while ctx.serve_poll(tk, 100000) == B.PM_PENDING:
                assert time.perf_counter() < deadline, "serve stream did not finish"
        wall = time.perf_counter() - t0
        return wall, ctx.serve_stats(reset=True)
    finally:
        ctx.serve_stop()


def run_serve(args):
    """Autotuner serving: Poisson query stream over the batched workload's tables and
    points, one of 64 resident models per query, top-16 per query, host buffers in
    and out (end to end through pm_serve_submit / pm_serve_poll)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1604_04997_gb300 import binding as B
    from paper_1604_04997_gb300 import tuning
    from paper_1604_04997_gb300 import workloads as W
    __graft_entry__.build()
    rate = 2000.0
    ctx = B.Context(0)
    b = tuning.build(ctx, args.variants, args.points)
    ctx.serve_set_weights(W.draw_weights(32, 64, 4))
    nv = [int(b.var_off[t + 1] - b.var_off[t]) for t in range(len(b.templates))]

    def draw(n, r, seed=9):
        qs = W.draw_queries(n, r, nv, args.points, 64, seed, 50000)
        return qs, [tuning.query_arrays(b, q) for q in qs]

    n_q = args.serve_queries
    qs, arrays = draw(n_q, rate)
    ck = Clocks(torch.cuda.current_device())
    ck.start()
    wall, st = _serve_stream(ctx, b, qs, arrays, 200)
    clocks = ck.stop()
    cand = sum(len(q.variant) for q in qs)
    qs10, arr10 = draw(n_q, 10 * rate, 10)
    wall10, st10 = _serve_stream(ctx, b, qs10, arr10, 200)
    plain_n = min(n_q, 200)
    wallp, stp = _serve_stream(ctx, b, qs[:plain_n], arrays[:plain_n], 0, sync=True)
    ctx.close()
    small = B.Context(0, 64 << 20)
    bs = tuning.build(small, args.variants, args.points)
    small.serve_set_weights(W.draw_weights(32, 64, 4))
    qs10s = [W.QueryDraw(q.arrival_s, q.template, q.model, q.variant, q.point) for q in qs10]
    wall64, st64 = _serve_stream(small, bs, qs10s, [tuning.query_arrays(bs, q) for q in qs10s], 200)
    small.close()
    in_b = sum(len(q.variant) * 36 for q in qs)

    def summ(st, wall, n):
        return {"p50_us": round(st["p50_us"], 1), "p99_us": round(st["p99_us"], 1), "max_us": round(st["max_us"], 1),
                "batches": st["n_batches"], "queries_per_batch": round(st["n_queries"] / max(1, st["n_batches"]), 2),
                "evals_per_s": st["n_candidates"] / wall, "queries": n, "rejected": st["n_rejected"],
                "h2d_mb": round(st["h2d_bytes"] / 1e6, 2), "d2h_mb": round(st["d2h_bytes"] / 1e6, 2)}

    line = {"metric": "served candidate evaluations/s (Poisson 2,000 queries/s, 1-50,000 candidates each, "
                      "FP64-accurate top-16 per query)",
            "value": cand / wall, "unit": "evals/s", "n_gpus": 1, "steps": n_q, "warmup": 16,
            "ms_per_step": wall / n_q * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64 counts, exact fixed-point products, fp64 out", "data": "synthetic",
            "config": {"workload": f"{n_q} queries over 10,000 variants x 4,096 points per template, 64 models",
                       "latency_note": "submit to results in the caller's host buffers, measured in the library",
                       "offered_evals_per_s": cand / qs[-1].arrival_s,
                       "rate_2000": summ(st, wall, n_q), "rate_20000": summ(st10, wall10, n_q),
                       "rate_20000_budget_64MiB": summ(st64, wall64, n_q),
                       "plain_one_at_a_time": summ(stp, wallp, plain_n)},
            "e2e": {"value": cand / wall, "unit": "evals/s", "h2d_bytes_per_step": in_b / n_q,
                    "d2h_bytes_per_step": 16 * 12 + 4},
            "roofline": None, "clocks": clocks, "gpu_launches": 2 * st["n_batches"]}
    print(json.dumps(line))


def run_calibrate(args):
    """Fit the model to this GPU from timed measurement kernels and predict held-out
    test kernels (Sec. 4-5): the model's own accuracy on GB300."""
    import __graft_entry__
    from paper_1604_04997_gb300 import binding as B
    from paper_1604_04997_gb300 import calibrate as C
    __graft_entry__.build()
    ctx = B.Context(0)
    t0 = time.perf_counter()
    r = C.calibrate(ctx, quick=args.steps < 5)
    wall = time.perf_counter() - t0
    ctx.close()
    groups = {k: round(v["geomean_rel_err"], 4) for k, v in r["test"]["groups"].items()}
    mgroups = {k: round(v["geomean_rel_err"], 4) for k, v in r["measurement"]["groups"].items()}
    line = {"metric": "geomean relative prediction error on held-out test kernels (weights fitted on this GPU)",
            "value": r["test"]["geomean_rel_err"], "unit": "fraction", "n_gpus": 1, "steps": 1, "warmup": 4,
            "ms_per_step": wall * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32/fp64 kernels; exact counts; FP64 fit", "data": "synthetic",
            "config": {"workload": f"{r['measurement']['n']} measurement + {r['test']['n']} test kernel runs, "
                                   "30 timed runs each, first 4 dropped, minimum kept",
                       "measurement_geomean_rel_err": r["measurement"]["geomean_rel_err"],
                       "test_groups": groups, "measurement_groups": mgroups,
                       "fit": {k: r["fit_report"][k] for k in ("rank", "cond_est", "rel_resid", "status")},
                       "selection": {k: r["selection"][k] for k in ("top1_hit_rate", "mean_top1_slowdown",
                                                                     "mean_top2_slowdown")},
                       "weights": r["weights"]},
            "roofline": None, "gpu_launches": None}
    print(json.dumps(line))
    if args.calib_out:
        json.dump(r, open(args.calib_out, "w"), indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variants", type=int, default=10000)
    ap.add_argument("--points", type=int, default=4096)
    ap.add_argument("--cpu-s", type=float, default=8.0)
    ap.add_argument("--ref-step-s", type=float, default=4.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="use the default launch shape")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of tuned schedules: read if it holds this workload, else written")
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "eval", "predict", "fit", "serve", "calibrate", "coupled"])
    ap.add_argument("--calib-out", default=None, help="write the full calibration result (JSON) here")
    ap.add_argument("--serve-queries", type=int, default=1000)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-call form")
    ap.add_argument("--no-serve", action="store_true", help="skip the short serving stream")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "calibrate":
        run_calibrate(args)
    elif args.workload not in ("batched", "coupled"):
        run_other(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
