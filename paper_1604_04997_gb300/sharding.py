"""Host-side logic of the multi-GPU path: one process per GPU, no collective on the
data path.

The batched evaluation is a set of independent (template, point) units, so N GPUs
either run N independent batches (weak scaling: each rank its own point set) or split
one batch by points (each rank ranks its own rows of every template; the results are
disjoint row ranges that only need to be gathered).  The only collectives are the
timing reduction (max over ranks) and, when a caller wants the full answer on one
rank, the gather of the per-rank result rows.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def split_points(pt_off: Sequence[int], world: int, rank: int) -> Tuple[np.ndarray, np.ndarray]:
    """Split every template's point range [pt_off[t], pt_off[t+1]) into `world`
    contiguous parts and return this rank's part: (local CSR offsets int64 [T+1],
    global row index of each local row int64 [n_local])."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    off = np.asarray(pt_off, dtype=np.int64)
    rows: List[np.ndarray] = []
    local = [0]
    for t in range(len(off) - 1):
        n = int(off[t + 1] - off[t])
        lo = off[t] + (n * rank) // world
        hi = off[t] + (n * (rank + 1)) // world
        rows.append(np.arange(lo, hi, dtype=np.int64))
        local.append(local[-1] + int(hi - lo))
    return np.asarray(local, dtype=np.int64), (np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64))


def rank_point_seed(seed: int, rank: int) -> int:
    """Point seed of a rank's own batch under weak scaling (rank 0 keeps `seed`)."""
    return seed + 7919 * rank


def max_over_ranks(x: float, device=None) -> float:
    """The largest of the ranks' values (a step time), on the default process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local: np.ndarray, global_rows: np.ndarray, total_rows: int) -> np.ndarray:
    """Assemble per-rank result rows (local [n_local, ...], indexed by global_rows)
    into the full [total_rows, ...] array on every rank (object all-gather: host
    memory only, used off the timed path)."""
    import torch.distributed as dist
    parts = [(global_rows, local)]
    if dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, (global_rows, local))
    out = np.empty((total_rows,) + local.shape[1:], dtype=local.dtype)
    seen = np.zeros(total_rows, dtype=bool)
    for rows, vals in parts:
        if seen[rows].any():
            raise ValueError("ranks returned overlapping rows")
        out[rows] = vals
        seen[rows] = True
    if not seen.all():
        raise ValueError("some rows were returned by no rank")
    return out
