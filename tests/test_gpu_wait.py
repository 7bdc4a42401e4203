"""The give-up path of the bounded mbarrier waits used by the tensor-core kernels
(prediction and the fit's Gram): a wait on a phase that nothing completes must return
after its limit with a timeout, and the context must stay usable.  No kernel is broken
on purpose: the probe waits on a barrier that expects an arrival nobody makes."""
import ctypes

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
    ctx = B.Context(0)
    yield ctx, torch.device("cuda:0")
    ctx.close()


def _probe(limit_ns, complete):
    import torch
    f = B.lib().pmx_wait_probe
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_ulonglong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    out = torch.full((2,), -1, dtype=torch.int64, device="cuda:0")
    assert f(limit_ns, complete, out.data_ptr(), None) == B.PM_OK
    torch.cuda.synchronize()
    gave_up, waited = out.cpu().tolist()
    return gave_up, waited


def test_wait_completes(env):
    gave_up, waited = _probe(10_000_000, 1)
    assert gave_up == 0
    assert 0 <= waited < 10_000_000


def test_wait_gives_up_and_context_survives(env):
    ctx, dev = env
    import torch
    gave_up, waited = _probe(2_000_000, 0)          # 2 ms, nothing arrives
    assert gave_up == 1
    assert 2_000_000 <= waited < 100_000_000
    # the context still runs the tensor-core prediction correctly afterwards
    F = _rand_features(1000, 32, 5)
    Wm = W.draw_weights(32, 8, 6)
    T = torch.empty((1000, 8), dtype=torch.float64, device=dev)
    ctx.predict(torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev), T, precision=B.PREC_BF16X3)
    ctx.sync_status()
    ref = oracle.predict(F, Wm)
    scale = oracle.predict_abs(F, Wm)
    assert (np.abs(T.cpu().numpy() - ref) <= 1e-5 * scale).all()
    assert _probe(10_000_000, 1)[0] == 0


def test_wait_probe_rejects_bad_limits(env):
    f = B.lib().pmx_wait_probe
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_ulonglong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    assert B.ERRORS[f(0, 1, 16, None)] == "PM_ERR_INVALID_ARG"
    assert B.ERRORS[f(200_000_000, 1, 16, None)] == "PM_ERR_INVALID_ARG"
    assert B.ERRORS[f(1000, 1, None, None)] == "PM_ERR_INVALID_ARG"
