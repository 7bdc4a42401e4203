"""Batched tuning problems: compile a set of kernel variants and lay out the
per-template variant and point lists that pm_eval_predict_topk consumes."""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import binding as B
from . import workloads as W


@dataclasses.dataclass
class Batched:
    templates: List[str]
    variants: List[W.Variant]          # in template-major order
    tables: np.ndarray                 # int32 [n_variants] table ids (duplicates share a table)
    var_off: np.ndarray                # int32 [T+1]
    points: np.ndarray                 # int64 [total][4]
    pt_off: np.ndarray                 # int64 [T+1]
    n_distinct: int

    @property
    def total_evals(self) -> int:
        return int(sum((self.var_off[t + 1] - self.var_off[t]) * (self.pt_off[t + 1] - self.pt_off[t])
                       for t in range(len(self.templates))))


def compile_variants(ctx: B.Context, variants: Sequence[W.Variant], lo: int, hi: int, layout: int = 32,
                     cache: Dict = None) -> List[int]:
    cache = {} if cache is None else cache
    ids = []
    for v in variants:
        if v.key not in cache:
            P = len(W.TEMPLATE_PARAMS[v.template])
            cache[v.key] = ctx.compile_counts(W.variant_ir(v), layout, [lo] * P, [hi] * P)[0]
        ids.append(cache[v.key])
    return ids


def build(ctx: B.Context, n_variants: int = 10000, n_points: int = 4096, variant_seed: int = 2,
          point_seed: int = 3, lo: int = W.BOX_LO, hi: int = W.BOX_HI, coupled: bool = False) -> Batched:
    """The batched tuning workload of workloads.batched_space, compiled in ctx
    (duplicate variants share one table)."""
    sp = W.batched_space(n_variants, n_points, variant_seed, point_seed, lo, hi, coupled)
    cache: Dict = {}
    tables = compile_variants(ctx, sp.variants, lo, hi, 32, cache)
    return Batched(sp.templates, sp.variants, np.array(tables, dtype=np.int32), sp.var_off, sp.points, sp.pt_off,
                   len(cache))


def save_space(path: str, ctx: B.Context, b: Batched, weights: np.ndarray = None) -> None:
    """Write a built tuning space (each distinct table once, the variants, both CSR
    offset arrays and the points) and optionally its fitted weights to one
    checksummed file (checkpoint.py)."""
    from . import checkpoint as CK
    distinct = sorted(set(int(t) for t in b.tables))
    slot = {t: i for i, t in enumerate(distinct)}
    knobs = np.array([[b.templates.index(v.template), v.tx, v.ty, v.unroll, int(v.prefetch), v.wg, v.stride]
                      for v in b.variants], dtype=np.int64).reshape(-1, 7)
    CK.save(path, ctx, distinct, names=[str(t) for t in distinct], weights=weights, arrays={
        "templates": np.frombuffer("\n".join(b.templates).encode(), dtype=np.uint8),
        "variant_knobs": knobs,
        "variant_table": np.array([slot[int(t)] for t in b.tables], dtype=np.int64),
        "var_off": np.asarray(b.var_off, dtype=np.int32),
        "points": np.asarray(b.points, dtype=np.int64),
        "pt_off": np.asarray(b.pt_off, dtype=np.int64)})


def load_space(path: str, ctx: B.Context) -> Tuple[Batched, np.ndarray]:
    """Resume a space written by save_space into ctx: its tables are registered anew
    (pm_table_load checks each image) and the variants point at the new ids.
    Returns the space and the weights (None if none were saved)."""
    from . import checkpoint as CK
    ck = CK.load(path, ctx)
    a = ck.arrays
    templates = bytes(a["templates"]).decode().split("\n") if a["templates"].size else []
    variants = [W.Variant(templates[int(k[0])], int(k[1]), int(k[2]), int(k[3]), bool(k[4]), int(k[5]), int(k[6]))
                for k in a["variant_knobs"]]
    tables = np.array([ck.table_ids[int(i)] for i in a["variant_table"]], dtype=np.int32)
    if len(variants) != len(tables) or a["var_off"][-1] != len(tables) or a["pt_off"][-1] != len(a["points"]):
        raise ValueError(f"{path}: inconsistent tuning space")
    return Batched(templates, variants, tables, a["var_off"].astype(np.int32), a["points"].astype(np.int64),
                   a["pt_off"].astype(np.int64), len(ck.table_ids)), ck.weights


def query_arrays(b: Batched, q: W.QueryDraw):
    """Candidate tables (int32 [n]) and points (int64 [n][4]) of one drawn query."""
    t = q.template
    tables = np.ascontiguousarray(b.tables[b.var_off[t] + q.variant], dtype=np.int32)
    points = np.ascontiguousarray(b.points[b.pt_off[t] + q.point], dtype=np.int64)
    return tables, points
