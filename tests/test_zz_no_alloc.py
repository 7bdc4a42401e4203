"""pm_predict_argmin_static: the argmin entry point for callers that cannot allocate
device memory (it uses a fixed array inside the library and needs no context).  Its
results must equal those of pm_predict_argmin on the same inputs, on consecutive
calls that reuse the shared array.  Collected last so that a failure here comes
after every other test has run."""
import numpy as np
import pytest

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
            assert np.all(np.abs(m - m_ref) <= 1e-12 * np.abs(m_ref))
        with pytest.raises(B.PMError) as e:     # more models than the fixed array is sized for
            B.predict_argmin_static(dF, torch.zeros((65, 32), dtype=torch.float64, device=dev), a_ref, m_ref)
        assert e.value.code == -1
    finally:
        ctx.close()
