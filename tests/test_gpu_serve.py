"""Serve loop (pm_serve_*) against the oracle: each query's topk (candidate index,
time) must be the oracle's ranking of the same candidates, ordered by (time,
candidate index).  Reading of ties: the returned candidates' oracle times, sorted,
equal the oracle's topk times, and each returned time matches its candidate's oracle
time to FP64 accuracy."""
import time

import numpy as np
import pytest

import oracle
from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import tuning
from paper_1604_04997_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_MODELS = 8


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    ctx = B.Context(0, 64 << 20)
    b = tuning.build(ctx, n_variants=240, n_points=512, variant_seed=31, point_seed=32)
    Wm = W.draw_weights(32, N_MODELS, 33)
    ctx.serve_set_weights(Wm)
    ctx.serve_start(batch_interval_us=200, n_streams=2, max_batch_queries=256)
    yield ctx, b, Wm
    ctx.serve_stop()
    ctx.close()


def _oracle_times(b, q, Wm):
    """Oracle prediction of every candidate of query q (features by the oracle's own
    counting of each variant's IR)."""
    t = q.template
    n = len(q.variant)
    times = np.empty(n)
    P = len(W.TEMPLATE_PARAMS[W.TEMPLATES[t]])
    pts = b.points[b.pt_off[t] + q.point][:, :P]
    for vi in np.unique(q.variant):
        sel = np.nonzero(q.variant == vi)[0]
        k = oracle.Kernel(W.variant_ir(b.variants[b.var_off[t] + vi]))
        F = k.features(pts[sel], 32, "struct")
        times[sel] = oracle.predict(F, Wm[q.model:q.model + 1])[:, 0]
    return times


def _check(times, topk, idx, tt):
    n = len(times)
    order = np.lexsort((np.arange(n), times))[:topk]
    m = min(n, topk)
    assert (idx[m:topk] == -1).all() and np.isinf(tt[m:topk]).all()
    got = idx[:m]
    assert len(set(got.tolist())) == m and (got >= 0).all() and (got < n).all()
    assert np.allclose(np.sort(times[got]), times[order[:m]], rtol=1e-12, atol=0)
    assert np.allclose(tt[:m], times[got], rtol=1e-12, atol=0)
    assert (np.diff(tt[:m]) >= 0).all()


def _run(ctx, b, qs, topk=16, timeout_s=30.0):
    keep, tickets = [], []
    for q in qs:
        tables, points = tuning.query_arrays(b, q)
        idx = np.full(16, -7, dtype=np.int32)
        tt = np.zeros(16)
        keep.append((tables, points, idx, tt))
        tickets.append(ctx.serve_submit(B.make_query(q.model, topk, tables, points, idx, tt)))
    t0 = time.time()
    for tk in tickets:
        while ctx.serve_poll(tk, 100000) == B.PM_PENDING:
            assert time.time() - t0 < timeout_s
    return [(k[2], k[3]) for k in keep]


def _draw(b, n, seed, max_cand=3000):
    nv = [int(b.var_off[t + 1] - b.var_off[t]) for t in range(len(b.templates))]
    return W.draw_queries(n, 2000.0, nv, 512, N_MODELS, seed, max_cand)


def test_serve_matches_oracle(env):
    ctx, b, Wm = env
    qs = _draw(b, 24, 40)
    res = _run(ctx, b, qs)
    for q, (idx, tt) in zip(qs, res):
        _check(_oracle_times(b, q, Wm), 16, idx, tt)


def test_serve_topk_below_16_and_tiny_queries(env):
    ctx, b, Wm = env
    qs = _draw(b, 12, 41, max_cand=20)
    for topk in (1, 5):
        res = _run(ctx, b, qs, topk)
        for q, (idx, tt) in zip(qs, res):
            times = _oracle_times(b, q, Wm)
            order = np.lexsort((np.arange(len(times)), times))[:topk]
            m = min(len(times), topk)
            assert np.allclose(np.sort(times[idx[:m]]), times[order[:m]], rtol=1e-12, atol=0)
            assert (idx[topk:] == -7).all()   # entries past topk are not written


def test_serve_alone_and_in_mix_identical(env):
    ctx, b, Wm = env
    (qa,) = _draw(b, 1, 42, max_cand=5000)
    (ia, ta), = _run(ctx, b, [qa])
    mix = _draw(b, 40, 43)
    res = _run(ctx, b, mix[:20] + [qa] + mix[20:])
    ib, tb = res[20]
    assert (ia == ib).all() and (ta.view(np.int64) == tb.view(np.int64)).all()


def test_serve_empty_query_and_errors(env):
    ctx, b, Wm = env
    idx = np.zeros(32, dtype=np.int32)
    tt = np.zeros(32)
    e32, e64 = np.zeros(0, dtype=np.int32), np.zeros((0, 4), dtype=np.int64)
    tk = ctx.serve_submit(B.make_query(0, 4, e32, e64, idx, tt))
    assert ctx.serve_poll(tk, 0) == B.PM_OK
    assert (idx[:4] == -1).all() and np.isinf(tt[:4]).all()
    with pytest.raises(B.PMError) as e:
        ctx.serve_poll(tk, 0)          # a finished ticket is forgotten
    assert e.value.code == -10
    tables = np.array([int(b.tables[0])], dtype=np.int32)
    pts = np.zeros((1, 4), dtype=np.int64)
    with pytest.raises(B.PMError) as e:
        ctx.serve_submit(B.make_query(N_MODELS, 4, tables, pts, idx, tt))     # no such model
    assert e.value.code == -1
    with pytest.raises(B.PMError) as e:
        ctx.serve_submit(B.make_query(0, 17, tables, pts, idx, tt))           # topk > 16
    assert e.value.code == -1
    with pytest.raises(B.PMError) as e:
        ctx.serve_submit(B.make_query(0, 4, np.array([1 << 30], dtype=np.int32), pts, idx, tt))
    assert e.value.code == -1
    # a point outside the table's box: the query completes with PM_ERR_OUT_OF_BOX
    P = len(W.TEMPLATE_PARAMS[b.templates[0]])
    bad = np.full((2, 4), 100, dtype=np.int64)
    bad[1, :P] = W.BOX_HI + 1
    tables2 = np.array([int(b.tables[0])] * 2, dtype=np.int32)
    tk = ctx.serve_submit(B.make_query(0, 2, tables2, bad, idx, tt))
    t0 = time.time()
    with pytest.raises(B.PMError) as e:
        while ctx.serve_poll(tk, 100000) == B.PM_PENDING:
            assert time.time() - t0 < 30
    assert e.value.code == -9
    assert idx[0] == 0 and idx[1] == -1    # the in-box candidate is still ranked
    # more candidates than the 64 MiB budget can ever hold
    n = 2_000_000
    big_t = np.full(n, int(b.tables[0]), dtype=np.int32)
    big_p = np.full((n, 4), 100, dtype=np.int64)
    rejected = ctx.serve_stats()["n_rejected"]
    with pytest.raises(B.PMError) as e:
        ctx.serve_submit(B.make_query(0, 4, big_t, big_p, idx, tt))
    assert e.value.code == -6
    assert ctx.serve_stats()["n_rejected"] == rejected + 1


def test_serve_small_budget_queues_and_stats(env):
    _, b0, Wm = env
    ctx = B.Context(0, 1 << 20)   # 1 MiB: two 10,000-candidate queries at most in flight
    try:
        b = tuning.build(ctx, n_variants=240, n_points=512, variant_seed=31, point_seed=32)
        ctx.serve_set_weights(Wm)
        ctx.serve_start(batch_interval_us=0, n_streams=3, max_batch_queries=8)
        nv = [int(b.var_off[t + 1] - b.var_off[t]) for t in range(len(b.templates))]
        qs = [q for q in W.draw_queries(60, 2000.0, nv, 512, N_MODELS, 44, 10000) if len(q.variant) > 3000][:10]
        res = _run(ctx, b, qs)
        for q, (idx, tt) in zip(qs, res):
            _check(_oracle_times(b, q, Wm), 16, idx, tt)
        st = ctx.serve_stats(reset=True)
        n_cand = sum(len(q.variant) for q in qs)
        assert st["n_queries"] == len(qs) and st["n_candidates"] == n_cand
        assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
        assert 0 < st["mean_us"] <= st["max_us"]
        # every candidate's point (32 B) went up, every query's results came back
        assert st["h2d_bytes"] >= 32 * n_cand and st["d2h_bytes"] > 0 and st["n_rejected"] == 0
        st2 = ctx.serve_stats()
        assert st2["n_queries"] == 0 and st2["h2d_bytes"] == 0 and st2["d2h_bytes"] == 0
        assert st2["n_rejected"] == 0 and st2["max_us"] == 0
        with pytest.raises(B.PMError) as e:
            ctx.serve_set_weights(Wm)      # weights are fixed while serving
        assert e.value.code == -6
    finally:
        ctx.serve_stop()
        ctx.close()
