"""GPU parity: counts (bit-exact), predictions (FP64-accurate) and the fused
evaluate -> predict -> top-k launch, all through the C ABI, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import tuning
from paper_1604_04997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    ctx = B.Context(0)
    yield ctx, torch.device("cuda:0")
    ctx.close()


def _eval(ctx, dev, ids, pts):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.int64)).to(dev)
    out = torch.full((len(ids), len(pts), 32), -7, dtype=torch.int64, device=dev)
    ctx.eval_counts(ids, d, out)
    ctx.sync_status()
    return out.cpu().numpy()


def test_small_workload_counts_exact(env):
    """Eight templates x 32 points, powers of two 64..256 and 64..8192."""
    ctx, dev = env
    for v in W.tiny_variants():
        ir = W.variant_ir(v)
        P = len(W.TEMPLATE_PARAMS[v.template])
        tid, _ = ctx.compile_counts(ir, 32, [64] * P, [8192] * P)
        k = oracle.Kernel(ir)
        for sizes in (W.POW2_SMALL, (64, 128, 256, 512, 1024, 2048, 4096, 8192)):
            pts = W.tiny_points(v.template, 32, sizes)
            got = _eval(ctx, dev, [tid], pts)[0]
            assert np.array_equal(got, k.features(pts, 32, "struct")), v.name
        pts = W.tiny_points(v.template, 32, (64, 128) if P == 3 else W.POW2_SMALL)
        assert np.array_equal(_eval(ctx, dev, [tid], pts)[0], k.features(pts, 32, "brute")), v.name


def test_small_n_pieces_exact(env):
    ctx, dev = env
    for t in W.TEMPLATES:
        vs = [W.canonical(t, 2 if t == "copy" else 1)] + \
             [x for i, x in enumerate(v for v in W.all_variants() if v.template == t) if i % 41 == 5][:3]
        P = len(W.TEMPLATE_PARAMS[t])
        pts = np.arange(1, 97).reshape(-1, 1) if P == 1 else \
            np.array([(a, b, c) for a in (1, 16, 17, 70) for b in (1, 3, 64) for c in (2, 33, 96)])
        for v in vs:
            ir = W.variant_ir(v)
            tid, _ = ctx.compile_counts(ir, 32, [1] * P, [65536] * P)
            assert np.array_equal(_eval(ctx, dev, [tid], pts)[0], oracle.Kernel(ir).features(pts, 32, "struct")), v.name


@pytest.mark.parametrize("n_points", [1, 127, 128, 129, 1000])
def test_many_tables_ragged(env, n_points):
    ctx, dev = env
    vs = [v for v in W.all_variants() if v.template == "stencil"][::17][:40]
    ids = tuning.compile_variants(ctx, vs, 64, 65536)
    pts = W.draw_points(1, n_points, 100 + n_points)
    got = _eval(ctx, dev, ids, pts)
    for i, v in enumerate(vs):
        assert np.array_equal(got[i], oracle.Kernel(W.variant_ir(v)).features(pts, 32, "struct")), v.name


def test_more_tables_than_one_launch_holds(env):
    """pm_eval_counts launches at most 65,535 tables at a time (the grid's y limit):
    70,000 entries (two distinct tables, alternating in runs) on 3 points cross that
    boundary, and every table's row block equals the oracle's counts."""
    ctx, dev = env
    vs = [W.canonical("stencil"), [v for v in W.all_variants() if v.template == "stencil"][7]]
    ids = tuning.compile_variants(ctx, vs, 64, 65536)
    pts = np.array([[64], [1000], [65536]], dtype=np.int64)
    ref = [oracle.Kernel(W.variant_ir(v)).features(pts, 32, "struct") for v in vs]
    which = (np.arange(70000) // 7) % 2          # runs of 7, so both sides of 65,535 differ
    got = _eval(ctx, dev, [ids[i] for i in which], pts)
    assert got.shape == (70000, 3, 32)
    for i in (0, 1):
        assert (got[which == i] == ref[i][None]).all()


def test_layout12(env):
    ctx, dev = env
    import torch
    for v in W.tiny_variants():
        ir = W.variant_ir(v)
        P = len(W.TEMPLATE_PARAMS[v.template])
        tid, _ = ctx.compile_counts(ir, 12, [64] * P, [8192] * P)
        pts = W.tiny_points(v.template, 32)
        d = torch.from_numpy(pts).to(dev)
        out = torch.empty((1, 32, 12), dtype=torch.int64, device=dev)
        ctx.eval_counts([tid], d, out)
        ctx.sync_status()
        assert np.array_equal(out.cpu().numpy()[0], oracle.Kernel(ir).features(pts, 12, "struct"))


def test_out_of_box_and_empty(env):
    import torch
    ctx, dev = env
    tid, _ = ctx.compile_counts(W.variant_ir(W.canonical("vecadd")), 32, [64], [1024])
    pts = np.array([[64], [1025], [100]], dtype=np.int64)
    d = torch.from_numpy(pts).to(dev)
    out = torch.full((1, 3, 32), -7, dtype=torch.int64, device=dev)
    ctx.eval_counts([tid], d, out)
    with pytest.raises(B.PMError) as e:
        ctx.sync_status()
    assert e.value.code == -9
    o = out.cpu().numpy()[0]
    assert (o[1] == 0).all() and o[0][3] == 64 and o[2][3] == 100
    ctx.sync_status()  # cleared
    ctx.eval_counts([tid], d[:0], out)  # no points: nothing to do
    ctx.sync_status()


# ----------------------------------------------------------------------------- prediction

def _rand_features(R, k, seed):
    rng = np.random.default_rng(seed)
    F = W.fit_features(R, k, seed)
    F[:, rng.integers(0, k)] += rng.integers(0, 2 ** 48, size=R)
    return F


@pytest.mark.parametrize("R,M", [(1, 1), (31, 3), (1000, 64), (4099, 17)])
def test_predict_fp64_accurate(env, R, M):
    import torch
    ctx, dev = env
    F = _rand_features(R, 32, R)
    Wm = W.draw_weights(32, M, M)
    T = torch.empty((R, M), dtype=torch.float64, device=dev)
    ctx.predict(torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev), T)
    ref = oracle.predict(F, Wm)
    mag = oracle.predict_abs(F, Wm)
    err = np.abs(T.cpu().numpy() - ref)
    assert (err <= 1e-12 * mag).all()          # stated bound ~ k 2^-44 = 1.8e-12 of sum |terms|
    assert (err <= 1e-9 * np.abs(ref)).all()   # the FP64-path tolerance


def test_predict_cancellation_and_native(env):
    import torch
    ctx, dev = env
    rng = np.random.default_rng(3)
    F = rng.integers(-2 ** 40, 2 ** 40, size=(777, 12), dtype=np.int64)
    Wm = rng.uniform(-1e-6, 1e-6, size=(5, 12))
    ref, mag = oracle.predict(F, Wm), oracle.predict_abs(F, Wm)
    for prec, tol in ((B.PREC_FP64, 1e-12), (B.PREC_NATIVE_FP64, 1e-14)):
        T = torch.empty((777, 5), dtype=torch.float64, device=dev)
        ctx.predict(torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev), T, prec)
        assert (np.abs(T.cpu().numpy() - ref) <= tol * mag).all()


def test_predict_argmin(env):
    import torch
    ctx, dev = env
    F = _rand_features(5000, 32, 9)
    F[4000] = F[17]                        # exact tie: the smaller row wins
    Wm = W.draw_weights(32, 64, 10)
    ref = oracle.predict(F, Wm)
    arg = torch.empty(64, dtype=torch.int64, device=dev)
    mn = torch.empty(64, dtype=torch.float64, device=dev)
    ctx.predict_argmin(torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev), arg, mn)
    a, m = arg.cpu().numpy(), mn.cpu().numpy()
    for j in range(64):
        assert abs(m[j] - ref[:, j].min()) <= 1e-12 * ref[:, j].min()
        assert abs(ref[a[j], j] - ref[:, j].min()) <= 1e-11 * ref[:, j].min()
        assert a[j] != 4000


# ----------------------------------------------------------------------------- fused top-k

def _check_topk(bp, idx, tt, w, topk, sample_rows):
    """Per sampled point: the returned ids are a valid top-k under the oracle's
    times (unique up to near-ties), and the returned times match the oracle."""
    for t_i, t in enumerate(bp.templates):
        v0, v1 = bp.var_off[t_i], bp.var_off[t_i + 1]
        rows = [r for r in sample_rows if bp.pt_off[t_i] <= r < bp.pt_off[t_i + 1]]
        if not rows or v1 == v0:
            continue
        P = len(W.TEMPLATE_PARAMS[t])
        kern = {}
        Tref = np.zeros((v1 - v0, len(rows)))
        for j, v in enumerate(bp.variants[v0:v1]):
            if v.key not in kern:
                F = oracle.Kernel(W.variant_ir(v)).features(bp.points[rows][:, :P], 32, "struct")
                kern[v.key] = oracle.predict(F, w[None])[:, 0]
            Tref[j] = kern[v.key]
        for c, r in enumerate(rows):
            col = Tref[:, c]
            order = sorted(range(len(col)), key=lambda i: (col[i], i))
            n_real = min(topk, v1 - v0)
            got_i, got_t = idx[r][:n_real], tt[r][:n_real]
            assert len(set(got_i.tolist())) == n_real and (got_i >= 0).all()
            assert np.allclose(got_t, col[order[:n_real]], rtol=1e-9, atol=0)
            assert np.allclose(col[got_i], got_t, rtol=1e-9, atol=0)
            # identical ids wherever the oracle's ranking has no near-tie
            for q in range(n_real):
                nxt = col[order[q + 1]] if q + 1 < len(order) else np.inf
                prv = col[order[q - 1]] if q > 0 else -np.inf
                if nxt - col[order[q]] > 1e-9 * col[order[q]] and col[order[q]] - prv > 1e-9 * col[order[q]]:
                    assert got_i[q] == order[q]
            if n_real < topk:
                assert (idx[r][n_real:] == -1).all()


def _run_topk(ctx, dev, bp, w, topk):
    import torch
    d_pts = torch.from_numpy(bp.points).to(dev)
    n = bp.points.shape[0]
    idx = torch.full((n, topk), -5, dtype=torch.int32, device=dev)
    tt = torch.empty((n, topk), dtype=torch.float64, device=dev)
    ctx.eval_predict_topk(bp.tables, bp.var_off, d_pts, bp.pt_off, torch.from_numpy(w).to(dev), topk, idx, tt)
    ctx.sync_status()
    return idx.cpu().numpy(), tt.cpu().numpy()


@pytest.mark.parametrize("topk", [1, 16])
def test_fused_topk_reduced(env, topk):
    ctx, dev = env
    bp = tuning.build(ctx, n_variants=400, n_points=100, variant_seed=21, point_seed=22)
    w = W.draw_weights(32, 1, 4)[0]
    idx, tt = _run_topk(ctx, dev, bp, w, topk)
    _check_topk(bp, idx, tt, w, topk, range(bp.points.shape[0]))


def test_fused_topk_few_variants_and_ragged(env):
    """Templates with fewer variants than k, and point counts off the 32-point units."""
    ctx, dev = env
    bp = tuning.build(ctx, n_variants=40, n_points=45, variant_seed=5, point_seed=6)
    w = W.draw_weights(32, 1, 7)[0]
    idx, tt = _run_topk(ctx, dev, bp, w, 16)
    _check_topk(bp, idx, tt, w, 16, range(bp.points.shape[0]))


def test_fused_topk_full_size_sampled(env):
    """The batched workload at full size (10,000 variants, 4,096 points per template)
    in the bench's launch configuration; sampled points checked against the oracle."""
    ctx, dev = env
    bp = tuning.build(ctx)
    w = W.draw_weights(32, 1, 4)[0]
    idx, tt = _run_topk(ctx, dev, bp, w, 16)
    rng = np.random.default_rng(0)
    rows = sorted(set(rng.choice(bp.points.shape[0], 48, replace=False).tolist()) |
                  {0, 4095, 4096, bp.points.shape[0] - 1})
    _check_topk(bp, idx, tt, w, 16, rows)
