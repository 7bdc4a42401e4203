"""Fit the run-time model to this GPU and evaluate it on held-out kernels (Sec. 4, Sec. 5).

Measurement kernels (Sec. 4.1) exercise the counted properties: streaming copies and
sums, strided and filled-stride accesses, transposes, tiled and naive matrix
products, arithmetic of each kind, and an empty kernel for the per-group overhead.
Each is timed with the protocol of Sec. 4.2 (30 runs, the first 4 dropped, the
minimum kept); its properties come from its IR through pm_compile_counts and
pm_eval_counts; the weights are the relative-error least-squares fit of Sec. 4.3
(pm_fit_weights).  Test kernels (a 5-point stencil, a skinny matrix product, batched
matrix-vector products, a reduction, axpy, vector add, all-pairs n-body, a 5 x 5
convolution) are timed the same way and predicted with the fitted weights
(pm_predict).  Everything that computes runs in
the library's CUDA kernels; this module only lists configurations and marshals
arrays.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import binding as B
from . import workloads as W

COLUMN_NAMES = (
    "const", "work-groups", "barriers",
    "f32 add", "f32 mul", "f32 div", "f32 pow/exp", "f32 special",
    "f64 add", "f64 mul", "f64 div", "f64 pow/exp", "f64 special",
    "local ld f32", "local ld f64", "local st",
    "gld32 s0", "gld32 s1", "gld32 filled", "gld32 partial", "gld32 >4",
    "gld64 s0", "gld64 s1", "gld64 >=2",
    "gst32 s1", "gst32 filled", "gst32 partial/>4",
    "gst64 s1", "gst64 >=2",
    "min(gld32,gst32) s1", "min(gld64,gst64) s1", "128-bit")


@dataclasses.dataclass(frozen=True)
class Case:
    probe: W.Probe
    params: Tuple[int, ...]     # (n,) or (n, m, l)
    group: str                  # kernel class, for reporting

    @property
    def label(self) -> str:
        return f"{self.probe.name}@{'x'.join(str(x) for x in self.params)}"


def measurement_set(quick: bool = False) -> List[Case]:
    """Measurement kernels and sizes (Sec. 4.1's classes at GB300-sized problems)."""
    P = W.Probe
    out: List[Case] = []
    pw = lambda lo, hi, step=1: [1 << e for e in range(lo, hi + 1, step)]
    if quick:
        pw = lambda lo, hi, step=1: [1 << lo, 1 << hi]
    g1 = (256, 512)
    g2 = ((16, 16), (32, 16), (32, 32))
    for i, n in enumerate(pw(10, 15)):
        gx, gy = g2[i % 3]
        out.append(Case(P("empty", gx=gx, gy=gy), (n,), "empty"))
    for kind in ("copy", "sum4", "index"):
        for i, n in enumerate(pw(24, 28)):
            out.append(Case(P(kind, gx=g1[i % 2]), (n,), "stride-1 " + kind))
    for s in (1, 2, 3):
        for i, n in enumerate(pw(22, 26, 2) if not quick else pw(22, 26)):
            out.append(Case(P("vsa", s, gx=g1[i % 2]), (n,), f"scale-add stride {s}"))
    for s in (2, 3):
        for i, n in enumerate(pw(15, 21, 3) if not quick else pw(15, 21)):
            out.append(Case(P("filled", s, 256, gx=g1[i % 2]), (n,), f"stride-{s} filled"))
    for kind in ("transpose_p", "transpose_r", "transpose_w"):
        for i, n in enumerate(pw(11, 14)):
            T = 16 if kind != "transpose_p" or i % 2 == 0 else 32
            out.append(Case(P(kind, gx=T, gy=T), (n,), kind))
    for shape in range(4):
        for i, n in enumerate(pw(8, 11)):
            n_, m_, l_ = [(n, n, n), (n, n, n // 2), (n, n // 2, n), (n // 2, n, n)][shape]
            T = 16 if i % 2 == 0 else 32
            out.append(Case(P("matmul", gx=T, gy=T), (n_, m_, l_), "tiled matmul"))
    for n in pw(8, 11):
        out.append(Case(P("matmul_naive", gx=16, gy=16), (n, n, n), "naive matmul"))
    for t in range(5):
        for k in ((256, 512, 768) if not quick else (256,)):
            for i, n in enumerate(pw(9, 11) if not quick else pw(9, 10)):
                gx, gy = g2[i % 3]
                out.append(Case(P("arith", t, k, gx, gy), (n,), "arith " + W.ARITH_TYPES[t]))
    # fp64 data and arithmetic
    for kind in ("copy", "sum4", "index"):
        for i, n in enumerate(pw(23, 27)):
            out.append(Case(P(kind, gx=g1[i % 2], f64=True), (n,), f"stride-1 {kind} f64"))
    for s in (1, 2):
        for i, n in enumerate(pw(22, 26, 2) if not quick else pw(22, 26)):
            out.append(Case(P("vsa", s, gx=g1[i % 2], f64=True), (n,), f"scale-add stride {s} f64"))
    for t in range(3):
        for k in ((128, 256) if not quick else (128,)):
            for i, n in enumerate(pw(8, 10) if not quick else pw(8, 9)):
                gx, gy = g2[i % 3]
                out.append(Case(P("arith", t, k, gx, gy, f64=True), (n,), "arith f64 " + W.ARITH_TYPES[t]))
    # local-memory trees with barriers (other tile and group sizes than the test reductions)
    for E, gx in ((16, 128), (64, 512)):
        for n in pw(22, 28, 2) if not quick else pw(22, 28):
            out.append(Case(P("reduction", E, gx=gx), (n,), "local reduction"))
    return out


def test_set(quick: bool = False) -> List[Case]:
    """Held-out test kernels (Sec. 5's families where the IR covers them)."""
    P = W.Probe
    pw = lambda lo, hi: [1 << e for e in range(lo, hi + 1)] if not quick else [1 << lo, 1 << hi]
    out: List[Case] = []
    for n in pw(10, 14):
        out.append(Case(P("stencil", gx=16, gy=16), (n,), "5-point stencil"))
    for n in pw(7, 10):   # skinny: n = l, m = 8 n
        out.append(Case(P("matmul", gx=16, gy=16), (n, 8 * n, n), "skinny matmul"))
    for b in pw(12, 18):
        out.append(Case(P("matvec"), (b,), "batched matvec f64"))
    for n in pw(22, 28):
        out.append(Case(P("reduction", 32, gx=256), (n,), "reduction"))
    for n in pw(21, 27):
        out.append(Case(P("axpy", 32, gx=256), (n,), "axpy f64"))
    for n in pw(22, 28):
        out.append(Case(P("vecadd", 16, gx=256), (n,), "vector add"))
    for n in pw(12, 16):
        out.append(Case(P("nbody", gx=256), (n,), "n-body"))
    for n in pw(10, 14):
        out.append(Case(P("conv5", gx=32, gy=8), (n,), "5x5 convolution"))
    return out


def features(ctx: B.Context, cases: Sequence[Case]):
    """Exact property rows (int64 [R][32]) of the cases, on the device."""
    import torch
    dev = torch.device(f"cuda:{ctx.device}")
    rows = np.zeros((len(cases), 32), dtype=np.int64)
    by_probe: Dict[W.Probe, List[int]] = {}
    for i, c in enumerate(cases):
        by_probe.setdefault(c.probe, []).append(i)
    for probe, idx in by_probe.items():
        P = probe.n_params
        hi = [max(cases[i].params[j] for i in idx) for j in range(P)]
        tid, _ = ctx.compile_counts(W.probe_ir(probe), 32, [1] * P, hi)
        pts = torch.tensor([list(cases[i].params) for i in idx], dtype=torch.int64, device=dev)
        out = torch.empty((1, len(idx), 32), dtype=torch.int64, device=dev)
        ctx.eval_counts([tid], pts, out)
        ctx.sync_status()
        rows[idx] = out[0].cpu().numpy()
    return rows


def time_cases(cases: Sequence[Case], runs: int = 30, skip: int = 4) -> np.ndarray:
    """Minimum of runs - skip timed runs per case (Sec. 4.2), in seconds."""
    t = np.zeros(len(cases))
    for i, c in enumerate(cases):
        p = c.probe
        n = c.params[0]
        m, l = (c.params[1], c.params[2]) if len(c.params) == 3 else (0, 0)
        t[i] = B.pmm_time(p.kind, p.variant, p.k, p.gx, p.gy, n, m, l, runs, skip, f64=p.f64)[0] * 1e-3
    return t


def _geomean(x) -> float:
    x = np.asarray(x, dtype=np.float64)
    return float(np.exp(np.mean(np.log(np.maximum(x, 1e-12))))) if len(x) else float("nan")


def selection_families(quick: bool = False) -> Dict[str, Tuple[List[W.Probe], List[Tuple[int, ...]]]]:
    """Configuration choices for one computation each (tile, group size, local
    prefetch or not) and the problem sizes to choose them for."""
    P = W.Probe
    two = lambda a, b: [a, b]
    fams = {
        "transpose": ([P(k, gx=T, gy=T) for k in ("transpose_p", "transpose_r", "transpose_w") for T in (16, 32)],
                      [(1 << 11,), (1 << 13,)] if not quick else [(1 << 11,)]),
        "matmul": ([P(k, gx=T, gy=T) for k in ("matmul", "matmul_naive") for T in (16, 32)],
                   [(512, 512, 512), (2048, 2048, 2048)] if not quick else [(512, 512, 512)]),
        "reduction": ([P("reduction", E, gx=Wg) for E, Wg in ((16, 128), (16, 256), (32, 256), (32, 512), (64, 256),
                                                              (64, 512))],
                      [(1 << 22,), (1 << 26,)] if not quick else [(1 << 22,)]),
        "vector add": ([P("vecadd", E, gx=Wg) for E, Wg in ((16, 256), (32, 256), (32, 512), (64, 512))],
                       [(1 << 22,), (1 << 26,)] if not quick else [(1 << 22,)]),
    }
    return fams


def select(ctx: B.Context, weights: np.ndarray, quick: bool = False, runs: int = 30, skip: int = 4) -> dict:
    """Model-guided configuration selection (the extension the paper proposes in
    Sec. 6.2): rank every candidate configuration of a computation with the fitted
    model through the serve API, then time all of them.  Reports whether the
    predicted best is the measured best, and the slowdown of the predicted best and
    of the best of the predicted top two (an autotuner that times only two) against
    the measured best."""
    fams = selection_families(quick)
    ctx.serve_set_weights(np.ascontiguousarray(weights, dtype=np.float64).reshape(1, 32))
    ctx.serve_start(batch_interval_us=0, n_streams=1, max_batch_queries=16)
    out = {}
    try:
        for fam, (probes, sizes) in fams.items():
            P = probes[0].n_params
            hi = [max(sz[j] for sz in sizes) for j in range(P)]
            tids = [ctx.compile_counts(W.probe_ir(p), 32, [1] * P, hi)[0] for p in probes]
            rows = []
            for sz in sizes:
                tables = np.array(tids, dtype=np.int32)
                pts = np.zeros((len(probes), 4), dtype=np.int64)
                pts[:, :P] = sz
                idx, tt = np.zeros(16, dtype=np.int32), np.zeros(16)
                tk = ctx.serve_submit(B.make_query(0, len(probes), tables, pts, idx, tt))
                while ctx.serve_poll(tk, 100000) == B.PM_PENDING:
                    pass
                order = [int(i) for i in idx[:len(probes)]]
                meas = time_cases([Case(p, sz, fam) for p in probes], runs, skip)
                best = float(meas.min())
                rows.append({"size": list(sz), "candidates": [p.name for p in probes],
                             "predicted_order": order, "predicted_s": [float(x) for x in tt[:len(probes)]],
                             "measured_s": [float(x) for x in meas],
                             "top1_hit": bool(meas[order[0]] == best),
                             "top1_slowdown": float(meas[order[0]] / best - 1.0),
                             "top2_slowdown": float(min(meas[order[0]], meas[order[1]]) / best - 1.0)})
            out[fam] = rows
    finally:
        ctx.serve_stop()
    flat = [r for rows in out.values() for r in rows]
    return {"families": out, "top1_hit_rate": float(np.mean([r["top1_hit"] for r in flat])),
            "mean_top1_slowdown": float(np.mean([r["top1_slowdown"] for r in flat])),
            "mean_top2_slowdown": float(np.mean([r["top2_slowdown"] for r in flat]))}


def calibrate(ctx: B.Context, quick: bool = False, runs: int = 30, skip: int = 4) -> dict:
    """Time the measurement set, fit the weights, predict the test set."""
    import torch
    dev = torch.device(f"cuda:{ctx.device}")
    meas, test = measurement_set(quick), test_set(quick)
    Fm, Ft = features(ctx, meas), features(ctx, test)
    tm, tt = time_cases(meas, runs, skip), time_cases(test, runs, skip)
    w = torch.zeros((1, 32), dtype=torch.float64, device=dev)
    rc, rep = ctx.fit_weights(torch.from_numpy(Fm).to(dev), torch.from_numpy(tm[:, None].copy()).to(dev), w,
                              B.FIT_RELATIVE, B.PREC_BF16X3, 3)
    pm = torch.empty((len(meas), 1), dtype=torch.float64, device=dev)
    pt = torch.empty((len(test), 1), dtype=torch.float64, device=dev)
    ctx.predict(torch.from_numpy(Fm).to(dev), w, pm, B.PREC_FP64)
    ctx.predict(torch.from_numpy(Ft).to(dev), w, pt, B.PREC_FP64)
    ctx.sync_status()
    pm, pt, wv = pm.cpu().numpy()[:, 0], pt.cpu().numpy()[:, 0], w.cpu().numpy()[0]
    em, et = np.abs(pm - tm) / tm, np.abs(pt - tt) / tt

    def per_group(cases, err, meas_t, pred_t):
        g: Dict[str, List[int]] = {}
        for i, c in enumerate(cases):
            g.setdefault(c.group, []).append(i)
        return {k: {"geomean_rel_err": _geomean(err[v]), "max_rel_err": float(np.max(err[v])),
                    "cases": [(cases[i].label, float(meas_t[i]), float(pred_t[i])) for i in v]} for k, v in g.items()}

    return {
        "selection": select(ctx, wv, quick, runs, skip),
        "fit_status": rc, "fit_report": rep[0],
        "weights": {COLUMN_NAMES[i]: float(wv[i]) for i in range(32) if wv[i] != 0.0},
        "measurement": {"n": len(meas), "geomean_rel_err": _geomean(em), "groups": per_group(meas, em, tm, pm)},
        "test": {"n": len(test), "geomean_rel_err": _geomean(et), "groups": per_group(test, et, tt, pt)},
    }
