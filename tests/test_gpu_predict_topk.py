"""GPU parity of pm_predict_topk (top-k rows per (group, model) over materialised
features, configuration selection of Sec. 6.1): bit for bit against the (time, row)
order of pm_predict's own output, and against the oracle's times (Dot2) within the
FP64 path's tolerance, with ids unique up to near-ties.  Ragged groups (empty, one
row, around the 32-row tile and the 1,024-position unit), row lists in the
[tables][points] layout, a group of a million rows, and bad inputs."""
import numpy as np
import pytest

import oracle
from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import workloads as W
from test_gpu_eval import _rand_features

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    ctx = B.Context(0, 64 << 20)
    yield ctx, torch.device("cuda:0")
    ctx.close()


def _run(ctx, dev, F, Wm, seg_off, topk, rows=None):
    import torch
    G, M = len(seg_off) - 1, Wm.shape[0]
    dF, dW = torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev)
    idx = torch.full((G, M, topk), -5, dtype=torch.int64, device=dev)
    tt = torch.full((G, M, topk), np.nan, dtype=torch.float64, device=dev)
    ctx.predict_topk(dF, dW, seg_off, topk, idx, tt, rows=None if rows is None else torch.from_numpy(rows).to(dev))
    ctx.sync_status()
    T = torch.empty((F.shape[0], M), dtype=torch.float64, device=dev)
    ctx.predict(dF, dW, T)
    ctx.sync_status()
    return idx.cpu().numpy(), tt.cpu().numpy(), T.cpu().numpy()


def _check(idx, tt, Tgpu, Tref, seg_off, topk, rows=None, groups=None, models=None):
    """Tref: the oracle's times [R][len(models)] for the checked models."""
    G = len(seg_off) - 1
    models = list(range(Tgpu.shape[1])) if models is None else models
    for g in (range(G) if groups is None else groups):
        pos = np.arange(seg_off[g], seg_off[g + 1])
        mem = pos if rows is None else rows[pos]
        n_real = min(topk, len(mem))
        for mi, m in enumerate(models):
            got_i, got_t = idx[g, m], tt[g, m]
            # bit for bit: the first rows of pm_predict's times in (time, row) order
            col = Tgpu[mem, m]
            order = np.lexsort((mem, col))[:n_real]
            assert np.array_equal(got_i[:n_real], mem[order]), (g, m)
            assert np.array_equal(got_t[:n_real].view(np.int64), col[order].view(np.int64)), (g, m)
            assert (got_i[n_real:] == -1).all() and np.isinf(got_t[n_real:]).all()
            # the oracle: the k smallest times, and each returned row's own time
            ref = Tref[mem, mi]
            assert np.allclose(got_t[:n_real], np.sort(ref)[:n_real], rtol=1e-9, atol=0), (g, m)
            assert np.allclose(Tref[got_i[:n_real], mi], got_t[:n_real], rtol=1e-9, atol=0), (g, m)
            so = np.lexsort((mem, ref))
            for q in range(n_real):   # identical ids wherever the oracle's order has no near-tie
                v = ref[so[q]]
                nxt = ref[so[q + 1]] if q + 1 < len(so) else np.inf
                prv = ref[so[q - 1]] if q > 0 else -np.inf
                if nxt - v > 1e-9 * abs(v) and v - prv > 1e-9 * abs(v):
                    assert got_i[q] == mem[so[q]], (g, m, q)


SIZES = [0, 1, 15, 16, 17, 31, 33, 0, 1023, 1024, 1025, 2100]


@pytest.mark.parametrize("M,topk", [(1, 1), (3, 5), (64, 16), (17, 16)])
def test_topk_contiguous_ragged_groups(env, M, topk):
    ctx, dev = env
    seg_off = np.concatenate([[0], np.cumsum(SIZES)]).astype(np.int64)
    R = int(seg_off[-1])
    F = _rand_features(R, 32, 31 + M)
    F[seg_off[3] + 9] = F[seg_off[3] + 2]           # exact tie inside a group: the smaller row first
    F[seg_off[11] + 1500] = F[seg_off[11] + 7]      # ... and across two units of one group
    Wm = W.draw_weights(32, M, 40 + topk)
    idx, tt, Tg = _run(ctx, dev, F, Wm, seg_off, topk)
    _check(idx, tt, Tg, oracle.predict(F, Wm), seg_off, topk)


@pytest.mark.parametrize("n_tables,n_points", [(300, 40), (1500, 12)])
def test_topk_row_list_per_point(env, n_tables, n_points):
    """Counts laid out [tables][points][k] (pm_eval_counts' output): one group per
    point, its rows t * n_points + p listed through d_rows; layout 12."""
    ctx, dev = env
    R = n_tables * n_points
    F = np.random.default_rng(n_tables).integers(0, 2 ** 40, size=(R, 12), dtype=np.int64)
    Wm = W.draw_weights(12, 8, 5)
    rows = (np.arange(n_tables)[None, :] * n_points + np.arange(n_points)[:, None]).ravel().astype(np.int64)
    seg_off = np.arange(0, R + 1, n_tables, dtype=np.int64)
    idx, tt, Tg = _run(ctx, dev, F, Wm, seg_off, 16, rows)
    _check(idx, tt, Tg, oracle.predict(F, Wm), seg_off, 16, rows)


@pytest.mark.parametrize("M", [1, 2, 5])
def test_topk_row_list_few_models(env, M):
    """The plain per-call form of a tuning-space ranking: [tables][points][32] counts,
    one group per point over 1,250 tables (two units and a merge per group), few
    models (one row per lane), ties from duplicated tables."""
    ctx, dev = env
    n_tables, n_points = 1250, 9
    R = n_tables * n_points
    F = np.random.default_rng(M).integers(0, 2 ** 36, size=(R, 32), dtype=np.int64)
    F[7 * n_points:8 * n_points] = F[3 * n_points:4 * n_points]     # table 7 duplicates table 3
    Wm = W.draw_weights(32, M, 6 + M)
    rows = (np.arange(n_tables)[None, :] * n_points + np.arange(n_points)[:, None]).ravel().astype(np.int64)
    seg_off = np.arange(0, R + 1, n_tables, dtype=np.int64)
    idx, tt, Tg = _run(ctx, dev, F, Wm, seg_off, 16, rows)
    _check(idx, tt, Tg, oracle.predict(F, Wm), seg_off, 16, rows)


def test_topk_one_group_of_a_million_rows(env):
    """1,000,000 rows x 32 features x 64 models, one group: the per-model top-16
    (977 units merged per model); sampled models against the oracle."""
    ctx, dev = env
    R = 1_000_000
    F = W.fit_features(R, 32, 77)
    Wm = W.draw_weights(32, 64, 78)
    seg_off = np.array([0, R], dtype=np.int64)
    idx, tt, Tg = _run(ctx, dev, F, Wm, seg_off, 16)
    models = [0, 13, 40, 63]
    _check(idx, tt, Tg, oracle.predict(F, Wm[models]), seg_off, 16, models=models)


def test_topk_empty_and_degenerate(env):
    import torch
    ctx, dev = env
    F = _rand_features(40, 32, 3)
    Wm = W.draw_weights(32, 2, 3)
    idx, tt, Tg = _run(ctx, dev, F, Wm, np.array([0, 0, 0], dtype=np.int64), 4)   # two empty groups
    assert (idx == -1).all() and np.isinf(tt).all()
    idx, tt, Tg = _run(ctx, dev, F, Wm, np.array([5, 40], dtype=np.int64), 16)   # offsets not from 0
    _check(idx, tt, Tg, oracle.predict(F, Wm), np.array([5, 40]), 16)
    # G == 0 writes nothing
    out = torch.full((1,), -5, dtype=torch.int64, device=dev)
    ctx.predict_topk(torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev), np.array([0], dtype=np.int64), 4,
                     out, out)
    ctx.sync_status()
    assert out.item() == -5


def test_topk_bad_arguments(env):
    import torch
    ctx, dev = env
    F = torch.from_numpy(_rand_features(64, 32, 4)).to(dev)
    Wm = torch.from_numpy(W.draw_weights(32, 2, 4)).to(dev)
    idx = torch.empty((1, 2, 16), dtype=torch.int64, device=dev)
    tt = torch.empty((1, 2, 16), dtype=torch.float64, device=dev)
    ok = np.array([0, 64], dtype=np.int64)
    for so, k, prec in ((ok, 0, B.PREC_FP64), (ok, 17, B.PREC_FP64), (np.array([0, 65]), 4, B.PREC_FP64),
                        (np.array([-1, 3]), 4, B.PREC_FP64), (ok, 4, B.PREC_BF16X3)):
        with pytest.raises(B.PMError) as e:
            ctx.predict_topk(F, Wm, so, k, idx, tt, precision=prec)
        assert e.value.code == -1
    with pytest.raises(B.PMError):
        ctx.predict_topk(F, Wm, np.array([0, 5, 3], dtype=np.int64), 4,
                         torch.empty((2, 2, 4), dtype=torch.int64, device=dev),
                         torch.empty((2, 2, 4), dtype=torch.float64, device=dev))
    # a listed row outside [0, R): skipped, reported by pm_sync_status
    rows = torch.tensor([3, 64, 5, -2], dtype=torch.int64, device=dev)
    ctx.predict_topk(F, Wm, np.array([0, 4], dtype=np.int64), 4, idx, tt, rows=rows)
    with pytest.raises(B.PMError) as e:
        ctx.sync_status()
    assert e.value.code == -1
    got = idx.view(-1)[:8].reshape(2, 4).cpu().numpy()   # [G=1][M=2][topk=4]
    assert set(got[:, :2].ravel().tolist()) == {3, 5} and (got[:, 2:] == -1).all()
    ctx.sync_status()
