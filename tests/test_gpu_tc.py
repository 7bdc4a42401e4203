"""Tensor-core prediction (three-term bf16 split, FP32 accumulation) against the
oracle's compensated FP64 prediction: |T - T_ref| <= 1e-5 * sum_i |F_i w_i|."""
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


def _predict(ctx, dev, F, Wm):
    import torch
    T = torch.full((F.shape[0], Wm.shape[0]), -1.0, dtype=torch.float64, device=dev)
    ctx.predict(torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev), T, B.PREC_BF16X3)
    ctx.sync_status()
    return T.cpu().numpy()


@pytest.mark.parametrize("R,M", [(128, 64), (1, 64), (129, 17), (1000, 1), (5003, 64)])
def test_tc_predict_small(env, R, M):
    ctx, dev = env
    F = W.fit_features(R, 32, R + M)
    Wm = W.draw_weights(32, M, M + 3)
    T = _predict(ctx, dev, F, Wm)
    ref, mag = oracle.predict(F, Wm), oracle.predict_abs(F, Wm)
    assert (np.abs(T - ref) <= 1e-5 * mag).all()


def test_tc_predict_negative_weights_and_counts(env):
    ctx, dev = env
    rng = np.random.default_rng(4)
    F = rng.integers(-2 ** 40, 2 ** 40, size=(777, 32), dtype=np.int64)
    Wm = rng.uniform(-1e-6, 1e-6, size=(64, 32))
    T = _predict(ctx, dev, F, Wm)
    ref, mag = oracle.predict(F, Wm), oracle.predict_abs(F, Wm)
    assert (np.abs(T - ref) <= 1e-5 * mag).all()


def test_tc_argmin(env):
    import torch
    ctx, dev = env
    F = W.fit_features(20000, 32, 9)
    Wm = W.draw_weights(32, 64, 10)
    ref, mag = oracle.predict(F, Wm), oracle.predict_abs(F, Wm)
    arg = torch.empty(64, dtype=torch.int64, device=dev)
    mn = torch.empty(64, dtype=torch.float64, device=dev)
    ctx.predict_argmin(torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev), arg, mn, B.PREC_BF16X3)
    ctx.sync_status()
    a, m = arg.cpu().numpy(), mn.cpu().numpy()
    for j in range(64):
        best = ref[:, j].min()
        # the returned row is a minimiser within the reduced-precision tolerance
        assert ref[a[j], j] - best <= 2e-5 * mag[a[j], j]
        assert abs(m[j] - ref[a[j], j]) <= 1e-5 * mag[a[j], j]


def test_tc_argmin_many_tiles_per_cta(env):
    """300,007 rows: every CTA streams many row tiles through both buffers; ragged last tile."""
    import torch
    ctx, dev = env
    F = W.fit_features(300_007, 32, 11)
    Wm = W.draw_weights(32, 40, 12)
    ref, mag = oracle.predict(F, Wm), oracle.predict_abs(F, Wm)
    arg = torch.empty(40, dtype=torch.int64, device=dev)
    mn = torch.empty(40, dtype=torch.float64, device=dev)
    ctx.predict_argmin(torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev), arg, mn, B.PREC_BF16X3)
    ctx.sync_status()
    a, m = arg.cpu().numpy(), mn.cpu().numpy()
    for j in range(40):
        assert ref[a[j], j] - ref[:, j].min() <= 2e-5 * mag[a[j], j]
        assert abs(m[j] - ref[a[j], j]) <= 1e-5 * mag[a[j], j]


def test_tc_empty_and_misaligned(env):
    import torch
    ctx, dev = env
    Wt = torch.from_numpy(W.draw_weights(32, 8, 1)).to(dev)
    arg = torch.zeros(8, dtype=torch.int64, device=dev)
    mn = torch.zeros(8, dtype=torch.float64, device=dev)
    F0 = torch.zeros(64, dtype=torch.int64, device=dev)[:0].view(0, 32)   # empty, non-null pointer
    ctx.predict_argmin(F0, Wt, arg, mn, B.PREC_BF16X3)
    ctx.sync_status()
    assert (arg.cpu().numpy() == -1).all() and np.isinf(mn.cpu().numpy()).all()
    buf = torch.zeros(129 * 32 + 1, dtype=torch.int64, device=dev)
    Fm = buf[1:].view(129, 32)          # 8 bytes past a 16-byte boundary
    T = torch.zeros((129, 8), dtype=torch.float64, device=dev)
    with pytest.raises(B.PMError) as e:
        ctx.predict(Fm, Wt, T, B.PREC_BF16X3)
    assert e.value.code == -1


def test_tc_predict_full_size_sampled(env):
    """1,000,000 rows x 32 features x 64 models, sampled rows checked."""
    ctx, dev = env
    F = W.fit_features(1_000_000, 32, 7)
    Wm = W.draw_weights(32, 64, 8)
    T = _predict(ctx, dev, F, Wm)
    rows = np.random.default_rng(1).choice(len(F), 2000, replace=False)
    ref, mag = oracle.predict(F[rows], Wm), oracle.predict_abs(F[rows], Wm)
    assert (np.abs(T[rows] - ref) <= 1e-5 * mag).all()
    assert (T[-1] > 0).all() and (T[0] > 0).all()
