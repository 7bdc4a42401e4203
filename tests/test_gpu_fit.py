"""GPU weight fit (Sec. 4.3) against the oracle's Householder QR."""
import numpy as np
import pytest

import oracle
from paper_1604_04997_gb300 import binding as B
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


def _fit(ctx, dev, F, T, objective=B.FIT_RELATIVE, steps=3, precision=None):
    """precision PREC_BF16X3 (default): Gram matrices on the tensor cores from exact
    digits; PREC_FP64: float-float Gram on the FP32 pipes."""
    import torch
    M = T.shape[1]
    Wd = torch.empty((M, F.shape[1]), dtype=torch.float64, device=dev)
    rc, rep = ctx.fit_weights(torch.from_numpy(F).to(dev), torch.from_numpy(np.ascontiguousarray(T)).to(dev), Wd,
                              objective, B.PREC_BF16X3 if precision is None else precision, steps)
    return rc, rep, Wd.cpu().numpy()


def _scaled_err(F, T, m, w, wref, objective):
    """Norm-wise relative weight error in the coordinates of the scaled problem:
    each weight times the largest entry of its column of the least-squares matrix."""
    A = F.astype(float) / (T[:, m:m + 1] if objective == "relative" else 1.0)
    sc = np.abs(A).max(axis=0)
    return np.linalg.norm((w - wref) * sc) / np.linalg.norm(wref * sc)


@pytest.mark.parametrize("precision", ["bf16x3", "fp64"])
@pytest.mark.parametrize("objective", ["relative", "absolute"])
def test_fit_matches_qr(env, objective, precision):
    ctx, dev = env
    F = W.fit_features(20000, 32, 5)
    wt = W.draw_weights(32, 6, 6)
    T = W.synth_timings(F, wt, 6)
    rc, rep, Wg = _fit(ctx, dev, F, T, B.FIT_RELATIVE if objective == "relative" else B.FIT_ABSOLUTE,
                       precision=B.PREC_BF16X3 if precision == "bf16x3" else B.PREC_FP64)
    assert rc == 0
    for m in range(6):
        wref, rank, cond, res = oracle.fit(F, T[:, m], objective)
        assert rank == 32 and cond <= 1e6
        assert _scaled_err(F, T, m, Wg[m], wref, objective) <= 1e-8
        assert rep[m]["rank"] == 32 and rep[m]["status"] == 0
        assert abs(rep[m]["rel_resid"] - res) <= 1e-6 * res


def test_fit_noise_free_recovers_truth(env):
    ctx, dev = env
    F = W.fit_features(5000, 32, 7)
    wt = W.draw_weights(32, 3, 8)
    T = W.synth_timings(F, wt, 9, sigma=0.0)
    rc, rep, Wg = _fit(ctx, dev, F, T)
    for m in range(3):
        assert _scaled_err(F, T, m, Wg[m], wt[m], "relative") <= 1e-10
        assert rep[m]["rel_resid"] < 1e-12


def test_fit_zero_column_and_rank_deficiency(env):
    ctx, dev = env
    F = W.fit_features(3000, 32, 10)
    F[:, 5] = 0                      # a property no measurement kernel exercises: weight 0
    F[:, 9] = 2 * F[:, 8]            # exactly dependent columns: rank deficient
    wt = W.draw_weights(32, 2, 11)
    T = W.synth_timings(F, wt, 12)
    rc, rep, Wg = _fit(ctx, dev, F, T)
    assert rc == B.PM_WARN_RANK_DEFICIENT
    assert (Wg[:, 5] == 0).all()
    for m in range(2):
        assert rep[m]["rank"] == 30 and rep[m]["n_dropped"] == 1 and rep[m]["status"] == 1
        # the fitted times (unique even when the weights are not) match the QR fit
        wref, rank, *_ = oracle.fit(F, T[:, m], "relative")
        assert rank == 30
        p, pref = oracle.predict(F, Wg[m][None])[:, 0], oracle.predict(F, wref[None])[:, 0]
        assert np.allclose(p, pref, rtol=1e-7, atol=0)


def test_fit_small_workload_from_gpu_counts(env):
    """The small workload: counts of the eight templates (12 columns) evaluated on the
    GPU, synthetic timings, one device model."""
    import torch
    ctx, dev = env
    rows = []
    for v in W.tiny_variants():
        P = len(W.TEMPLATE_PARAMS[v.template])
        tid, _ = ctx.compile_counts(W.variant_ir(v), 12, [64] * P, [8192] * P)
        pts = W.tiny_points(v.template, 32, (64, 128, 256, 512, 1024, 2048, 4096, 8192))
        out = torch.empty((1, 32, 12), dtype=torch.int64, device=dev)
        ctx.eval_counts([tid], torch.from_numpy(pts).to(dev), out)
        rows.append(out.cpu().numpy()[0])
    ctx.sync_status()
    F = np.concatenate(rows)
    wt = W.draw_weights(12, 1, 1)
    T = W.synth_timings(F, wt, 1)
    rc, rep, Wg = _fit(ctx, dev, F, T, steps=5)
    wref, rank, cond, res = oracle.fit(F, T[:, 0], "relative")
    assert rep[0]["rank"] == rank
    p, pref = oracle.predict(F, Wg[0][None])[:, 0], oracle.predict(F, wref[None])[:, 0]
    assert np.allclose(p, pref, rtol=1e-8, atol=0)
    if rank == 12 and cond <= 1e6:
        assert _scaled_err(F, T, 0, Wg[0], wref, "relative") <= 1e-8


def test_fit_rejects_bad_timings(env):
    ctx, dev = env
    F = W.fit_features(500, 32, 13)
    T = W.synth_timings(F, W.draw_weights(32, 1, 14), 15)
    T[7, 0] = -1.0
    with pytest.raises(B.PMError) as e:
        _fit(ctx, dev, F, T)
    assert e.value.code == -1


def test_fit_full_size_sampled_models(env):
    """200,000 rows x 32 features, 64 models in one call; 8 of the models checked
    against the QR oracle."""
    ctx, dev = env
    F = W.fit_features(200000, 32, 5)
    wt = W.draw_weights(32, 64, 6)
    T = W.synth_timings(F, wt, 6)
    rc, rep, Wg = _fit(ctx, dev, F, T)
    assert rc == 0
    for m in (0, 9, 21, 33, 40, 51, 60, 63):
        wref, rank, cond, res = oracle.fit(F, T[:, m], "relative")
        assert _scaled_err(F, T, m, Wg[m], wref, "relative") <= 1e-8


@pytest.mark.parametrize("R", [1, 63, 4097, 8192 + 130])
def test_fit_tensor_gram_ragged_rows_and_k12(env, R):
    """Row counts off the 64-row stages and 4096-row chunks (including a single row
    and fewer rows than columns), and a 12-column problem: the tensor-core Gram and
    the float-float Gram give the same fit (both refined against the exact residual)."""
    ctx, dev = env
    for k in (32, 12):
        F = W.fit_features(max(R, 40), 32, 20 + R)[:R, :k].copy()
        F[:, 0] += 1                                    # no all-zero row
        T = W.synth_timings(F, W.draw_weights(k, 3, 21), 22)
        rc1, rep1, W1 = _fit(ctx, dev, F, T, precision=B.PREC_BF16X3)
        rc2, rep2, W2 = _fit(ctx, dev, F, T, precision=B.PREC_FP64)
        if R >= k:
            assert rc1 == rc2
        for m in range(3):
            if R >= k:
                assert rep1[m]["rank"] == rep2[m]["rank"]
            p1, p2 = oracle.predict(F, W1[m][None])[:, 0], oracle.predict(F, W2[m][None])[:, 0]
            assert np.allclose(p1, p2, rtol=1e-7, atol=0), (k, m)


def test_fit_ill_conditioned_uses_exact_gram(env):
    """Two nearly collinear columns (cond(A) ~ 1e4-1e5, so cond(G) 2^-24 > 1): refinement
    on the three-bf16-term Gram cannot converge, and PM_PREC_BF16X3 repeats the fit on
    the exact digit Gram; the weights must still match the QR fit to 1e-8."""
    ctx, dev = env
    rng = np.random.default_rng(31)
    F = W.fit_features(20000, 32, 31)
    F[:, 9] = 2 * F[:, 8] + rng.integers(0, 4, size=len(F))   # almost dependent columns
    wt = W.draw_weights(32, 3, 32)
    T = W.synth_timings(F, wt, 33)
    rc, rep, Wg = _fit(ctx, dev, F, T)
    checked = 0
    for m in range(3):
        wref, rank, cond, res = oracle.fit(F, T[:, m], "relative")
        if rank == 32 and cond <= 1e6:
            assert cond > 1e3
            assert _scaled_err(F, T, m, Wg[m], wref, "relative") <= 1e-8
            assert rep[m]["status"] == 0
            checked += 1
    assert checked > 0
