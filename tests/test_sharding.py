"""Multi-process path on CPU: point sharding, the gather of per-rank result rows and
the max-over-ranks timing reduction, with world_size 2 over gloo.  Each rank ranks
its own rows with the oracle; the gathered result must equal one process ranking
everything."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1604_04997_gb300 import sharding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_points_partitions_every_template():
    pt_off = [0, 5, 5, 37, 38, 1000]
    for world in (1, 2, 3, 4, 7):
        seen = []
        for rank in range(world):
            loc, rows = sharding.split_points(pt_off, world, rank)
            assert loc[0] == 0 and len(loc) == len(pt_off) and loc[-1] == len(rows)
            for t in range(len(pt_off) - 1):
                r = rows[loc[t]:loc[t + 1]]
                assert ((r >= pt_off[t]) & (r < pt_off[t + 1])).all()
                assert (np.diff(r) == 1).all()
            seen.append(rows)
        allr = np.sort(np.concatenate(seen))
        assert (allr == np.arange(pt_off[-1])).all()
    with pytest.raises(ValueError):
        sharding.split_points(pt_off, 2, 2)


def test_rank_point_seeds_differ():
    assert sharding.rank_point_seed(3, 0) == 3
    assert len({sharding.rank_point_seed(3, r) for r in range(8)}) == 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle
    from paper_1604_04997_gb300 import sharding as S
    from paper_1604_04997_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # small batched problem: six strided-copy variants at 40 log-uniform points
        vs = [v for v in W.all_variants() if v.template == "copy"][::7][:6]
        ks = [oracle.Kernel(W.variant_ir(v)) for v in vs]
        pts = W.draw_points(1, 40, 11)
        loc, rows = S.split_points([0, len(pts)], world, rank)
        w = W.draw_weights(32, 1, 4)[0]
        idx, val = oracle.eval_predict_topk(ks, pts[rows], w, 4, 1)
        full_idx = S.gather_rows(idx, rows, len(pts))
        full_val = S.gather_rows(val, rows, len(pts))
        ref_idx, ref_val = oracle.eval_predict_topk(ks, pts, w, 4, 1)
        ok = (full_idx == ref_idx).all() and (full_val == ref_val).all()
        m = S.max_over_ranks(1.5 + rank)
        ok = ok and m == 1.5 + world - 1
        open(os.path.join(out_dir, f"rank{rank}"), "w").write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        assert (tmp_path / f"rank{r}").read_text() == "ok"
