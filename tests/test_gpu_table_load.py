"""Resume from a saved tuning space on the GPU: tables written by checkpoint.save and
registered in a fresh context through pm_table_load give the same counts and the same
fused top-k ranking, bit for bit, as the tables compiled from the IR."""
import dataclasses
import os

import numpy as np
import pytest

from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import checkpoint as CK
from paper_1604_04997_gb300 import tuning
from paper_1604_04997_gb300 import workloads as W
from test_gpu_eval import _eval, _run_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    ctx = B.Context(0, 64 << 20)
    yield ctx, torch.device("cuda:0")
    ctx.close()


@pytest.mark.parametrize("coupled", [False, True])
def test_resumed_space_ranks_identically(env, tmp_path, coupled):
    ctx, dev = env
    bp = tuning.build(ctx, n_variants=300, n_points=100, variant_seed=71, point_seed=72, coupled=coupled)
    w = W.draw_weights(32, 2, 73)
    distinct = sorted(set(bp.tables.tolist()))
    path = os.path.join(tmp_path, "space.pmck")
    CK.save(path, ctx, distinct, weights=w)

    ctx2 = B.Context(0, 64 << 20)
    try:
        ck = CK.load(path, ctx2)
        remap = dict(zip(distinct, ck.table_ids))
        bp2 = dataclasses.replace(bp, tables=np.array([remap[t] for t in bp.tables.tolist()], dtype=np.int32))
        idx, tt = _run_topk(ctx, dev, bp, w[0], 16)
        idx2, tt2 = _run_topk(ctx2, dev, bp2, ck.weights[0], 16)
        assert np.array_equal(idx, idx2) and np.array_equal(tt, tt2)
        t = W.COUPLED_TEMPLATES[1] if coupled else "stencil"
        t0 = bp.templates.index(t)
        P = len(W.TEMPLATE_PARAMS[t])
        own = sorted(set(bp.tables[bp.var_off[t0]:bp.var_off[t0 + 1]].tolist()))[:12]
        pts = np.ascontiguousarray(bp.points[bp.pt_off[t0]:bp.pt_off[t0 + 1], :P])
        a = _eval(ctx, dev, own, pts)
        b = _eval(ctx2, dev, [remap[i] for i in own], pts)
        assert len(own) > 0 and np.array_equal(a, b)
    finally:
        ctx2.close()
