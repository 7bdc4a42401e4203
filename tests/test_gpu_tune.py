"""The autotuner of the fused ranking launch (pm_tune): every candidate launch shape
(variants per work unit, warps per CTA, CTAs per SM) must give the same rankings, bit
for bit, as the default shape; the tuning log lists every candidate; a tuning cache
written by one context is read back by another without re-timing."""
import os
import tempfile

import numpy as np
import pytest

from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import tuning
from paper_1604_04997_gb300 import workloads as W
from test_gpu_eval import _check_topk, _run_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def test_tuned_shape_ranks_like_the_default(dev):
    w = W.draw_weights(32, 1, 4)[0]
    plain = B.Context(0)
    plain.tune(False)
    bp0 = tuning.build(plain, n_variants=3000, n_points=300, variant_seed=31, point_seed=32)
    idx0, t0 = _run_topk(plain, dev, bp0, w, 16)
    info0 = plain.plan_info(bp0.tables, bp0.var_off, bp0.pt_off)
    assert not info0["tuned"]
    plain.close()

    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "tune.json")
        tuned = B.Context(0)
        tuned.tune(True, cache)
        bp = tuning.build(tuned, n_variants=3000, n_points=300, variant_seed=31, point_seed=32)
        idx, t = _run_topk(tuned, dev, bp, w, 16)
        info = tuned.plan_info(bp.tables, bp.var_off, bp.pt_off)
        log = tuned.plan_tune_log(bp.tables, bp.var_off, bp.pt_off)
        tuned.close()
        assert info["tuned"]
        # every slice (whole group, 2048, 1024, 512) x warps per CTA (4, 8) x up to three CTA counts
        assert len({(r[0], r[1]) for r in log}) == 8 and 8 <= len(log) <= 24
        assert all(r[3] > 0 for r in log)
        assert np.array_equal(idx, idx0) and np.array_equal(t.view(np.int64), t0.view(np.int64))
        _check_topk(bp, idx, t, w, 16, range(0, bp.points.shape[0], 7))

        # a second context takes the shape from the cache: no timing, same rankings
        again = B.Context(0)
        again.tune(True, cache)
        bp2 = tuning.build(again, n_variants=3000, n_points=300, variant_seed=31, point_seed=32)
        idx2, t2 = _run_topk(again, dev, bp2, w, 16)
        info2 = again.plan_info(bp2.tables, bp2.var_off, bp2.pt_off)
        log2 = again.plan_tune_log(bp2.tables, bp2.var_off, bp2.pt_off)
        again.close()
        assert info2["tuned"] and not log2
        assert (info2["nw"], info2["grid"], info2["slice"]) == (info["nw"], info["grid"], info["slice"])
        assert np.array_equal(idx2, idx0) and np.array_equal(t2.view(np.int64), t0.view(np.int64))
