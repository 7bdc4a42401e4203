"""pm_predict_argmin_static: the argmin entry point for callers that cannot allocate
device memory (it uses a fixed array inside the library and needs no context).  Its
results must equal those of pm_predict_argmin on the same inputs bit for bit (the two
share their arithmetic), on consecutive calls that reuse the shared array, and agree
with the oracle's FP64-accurate times.  Collected last so that a failure here comes
after every other test has run."""
import numpy as np
import pytest

import oracle
from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _inputs(R, M, seed):
    F = W.fit_features(R, 32, seed)
    F[R // 2] = F[3]                 # an exact tie between two rows: the smaller row wins
    return F, W.draw_weights(32, M, seed + 1)


def test_static_argmin_matches_allocating_entry_point():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    dev = torch.device("cuda:0")
    ctx = B.Context(0)
    try:
        for R, M, seed in ((100003, 64, 21), (4099, 17, 22)):   # two calls in a row
            F, Wm = _inputs(R, M, seed)
            dF, dW = torch.from_numpy(F).to(dev), torch.from_numpy(Wm).to(dev)
            a_ref = torch.empty(M, dtype=torch.int64, device=dev)
            m_ref = torch.empty(M, dtype=torch.float64, device=dev)
            ctx.predict_argmin(dF, dW, a_ref, m_ref)
            a = torch.full((M,), -3, dtype=torch.int64, device=dev)
            m = torch.full((M,), -3.0, dtype=torch.float64, device=dev)
            B.predict_argmin_static(dF, dW, a, m)
            torch.cuda.synchronize()
            a_ref, m_ref, a, m = (x.cpu().numpy() for x in (a_ref, m_ref, a, m))
            assert np.array_equal(a, a_ref)
            assert np.array_equal(m, m_ref)
            # the oracle: the returned row's time is the minimum, within the FP64 path's 1e-9
            T = oracle.predict(F, Wm)
            tmin = T.min(axis=0)
            assert np.all(np.abs(m - tmin) <= 1e-9 * np.abs(tmin))
            assert np.all(np.abs(T[a, np.arange(M)] - tmin) <= 1e-9 * np.abs(tmin))
        # no rows: every model gets row -1 and time +inf
        a0 = torch.zeros(3, dtype=torch.int64, device=dev)
        m0 = torch.zeros(3, dtype=torch.float64, device=dev)
        B.predict_argmin_static(torch.zeros((0, 32), dtype=torch.int64, device=dev), dW[:3], a0, m0)
        torch.cuda.synchronize()
        assert (a0.cpu().numpy() == -1).all() and np.isinf(m0.cpu().numpy()).all()
        with pytest.raises(B.PMError) as e:     # more models than the fixed array is sized for
            B.predict_argmin_static(dF, torch.zeros((65, 32), dtype=torch.float64, device=dev), a_ref, m_ref)
        assert e.value.code == -1
    finally:
        ctx.close()
