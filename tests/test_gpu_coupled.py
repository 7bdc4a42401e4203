"""GPU parity on coupled-domain kernels (triangles, bands: counts with a table
denominator): exact counts, the fused evaluate -> predict -> top-k launch and the
serve loop, all through the C ABI, against the oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import tuning
from paper_1604_04997_gb300 import workloads as W
from test_gpu_eval import _check_topk, _eval, _run_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    ctx = B.Context(0, 64 << 20)
    yield ctx, torch.device("cuda:0")
    ctx.close()


@pytest.mark.parametrize("t", W.COUPLED_TEMPLATES)
def test_coupled_counts_exact(env, t):
    """Every variant of the template, one launch: small sizes (empty and partial tiles,
    w = 0 and w >= n) against brute force, log-uniform points to 65536 per axis."""
    ctx, dev = env
    vs = [v for v in W.coupled_variants() if v.template == t]
    P = len(W.TEMPLATE_PARAMS[t])
    ids = tuning.compile_variants(ctx, vs, 0 if t == "band" else 1, 65536)   # band: w = 0 is in the box
    if P == 1:
        small = np.arange(1, 40).reshape(-1, 1)
    else:
        small = np.array([(a, b) for a in (1, 2, 5, 31, 33, 64) for b in (1, 2, 9, 40, 70)])
        if t == "band":
            small = np.concatenate([small, [[5, 0], [64, 0], [7, 100]]])
        if t == "syrk":
            small = small[::4]
    pts = np.concatenate([small, W.draw_points(P, 200, 41, 1, 65536)])
    got = _eval(ctx, dev, ids, pts)
    for i, v in enumerate(vs):
        k = oracle.Kernel(W.variant_ir(v))
        assert np.array_equal(got[i][len(small):], k.features(pts[len(small):], 32, "struct")), v.name
        if i % 3 == 0:
            assert np.array_equal(got[i][:len(small)], k.features(small, 32, "brute")), v.name


def test_coupled_topk_reduced(env):
    """All four coupled templates, 300 drawn variants, 100 points each: every point's
    top-16 against the oracle's ranking."""
    ctx, dev = env
    bp = tuning.build(ctx, n_variants=300, n_points=100, variant_seed=51, point_seed=52, coupled=True)
    w = W.draw_weights(32, 1, 53)[0]
    idx, tt = _run_topk(ctx, dev, bp, w, 16)
    _check_topk(bp, idx, tt, w, 16, range(bp.points.shape[0]))


def test_coupled_topk_full_size_sampled(env):
    """The coupled workload at the bench's size (10,000 variants, 4,096 points per
    template) in its launch configuration; sampled points checked against the oracle."""
    ctx, dev = env
    bp = tuning.build(ctx, variant_seed=12, coupled=True)
    w = W.draw_weights(32, 1, 4)[0]
    idx, tt = _run_topk(ctx, dev, bp, w, 16)
    rng = np.random.default_rng(1)
    rows = sorted(set(rng.choice(bp.points.shape[0], 24, replace=False).tolist()) |
                  {0, 4095, 4096, bp.points.shape[0] - 1})
    _check_topk(bp, idx, tt, w, 16, rows)


def test_coupled_serve(env):
    """Serve queries over coupled-domain candidates: each query's top-k against the
    oracle's times of the same candidates."""
    ctx, dev = env
    b = tuning.build(ctx, n_variants=120, n_points=256, variant_seed=61, point_seed=62, coupled=True)
    Wm = W.draw_weights(32, 4, 63)
    ctx.serve_set_weights(Wm)
    ctx.serve_start(batch_interval_us=200, n_streams=2, max_batch_queries=64)
    try:
        nv = [int(b.var_off[t + 1] - b.var_off[t]) for t in range(len(b.templates))]
        qs = W.draw_queries(12, 2000.0, nv, 256, 4, 64, 2000)
        keep, tickets = [], []
        for q in qs:
            tables, points = tuning.query_arrays(b, q)
            idx = np.full(16, -7, dtype=np.int32)
            tt = np.zeros(16)
            keep.append((q, idx, tt, tables, points))   # read when the batch forms: keep alive
            tickets.append(ctx.serve_submit(B.make_query(q.model, 16, tables, points, idx, tt)))
        t0 = time.time()
        for tk in tickets:
            while ctx.serve_poll(tk, 100000) == B.PM_PENDING:
                assert time.time() - t0 < 30
        for q, idx, tt, _, _ in keep:
            t = q.template
            P = len(W.TEMPLATE_PARAMS[b.templates[t]])
            pts = b.points[b.pt_off[t] + q.point][:, :P]
            times = np.empty(len(q.variant))
            for vi in np.unique(q.variant):
                sel = np.nonzero(q.variant == vi)[0]
                F = oracle.Kernel(W.variant_ir(b.variants[b.var_off[t] + vi])).features(pts[sel], 32, "struct")
                times[sel] = oracle.predict(F, Wm[q.model:q.model + 1])[:, 0]
            m = min(16, len(times))
            order = np.lexsort((np.arange(len(times)), times))[:m]
            got = idx[:m]
            assert len(set(got.tolist())) == m and (got >= 0).all()
            assert np.allclose(np.sort(times[got]), times[order], rtol=1e-12, atol=0)
            assert np.allclose(tt[:m], times[got], rtol=1e-12, atol=0)
    finally:
        ctx.serve_stop()


def test_coupled_counts_layout12(env):
    """Materialised 12-column counts of coupled-domain tables (exact division by the
    table denominator in the 12-column kernel) against the oracle."""
    import torch
    ctx, dev = env
    for t in W.COUPLED_TEMPLATES:
        vs = [v for v in W.coupled_variants() if v.template == t][::7]
        P = len(W.TEMPLATE_PARAMS[t])
        ids = [ctx.compile_counts(W.variant_ir(v), 12, [1] * P, [65536] * P)[0] for v in vs]
        pts = W.draw_points(P, 130, 78, 1, 65536)
        out = torch.full((len(ids), len(pts), 12), -7, dtype=torch.int64, device=dev)
        ctx.eval_counts(ids, torch.from_numpy(pts).to(dev), out)
        ctx.sync_status()
        got = out.cpu().numpy()
        for i, v in enumerate(vs):
            assert np.array_equal(got[i], oracle.Kernel(W.variant_ir(v)).features(pts, 12, "struct")), v.name
