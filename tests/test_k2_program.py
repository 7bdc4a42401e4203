"""The fused ranking kernel's per-table programs, checked on the CPU.

A program replaces a table's column sums and weight dot product by one dot product
over the piece's slots (sum_col W_col sum_e coef_e slot_e = sum_slot Weff_slot slot)
and folds every post-op min(A, B) whose smaller operand is fixed over the box.  The
program's value must equal sum_col W_col p_col(n) exactly, with p_col(n) from the
table (itself checked against the oracle in test_compile.py), for any weights,
including negative ones, at points all over the box (corners included, where a fold
decision is tightest)."""
import ctypes

import numpy as np
import pytest

from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import workloads as W
from table_interp import Table, _s64, program_dot


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build_library()
    c = B.Context(-1)
    yield c
    c.close()


def k2_program(words):
    L = B.lib()
    f = L.pmx_k2_program
    sz = ctypes.c_size_t
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, sz, ctypes.c_void_p, sz, ctypes.POINTER(sz), ctypes.c_void_p, sz,
                  ctypes.POINTER(sz), ctypes.c_void_p, sz, ctypes.POINTER(sz)]
    words = np.ascontiguousarray(words, dtype=np.uint32)
    prog = np.zeros(8192, dtype=np.uint32)
    tgt = np.zeros((1024, 4), dtype=np.uint32)
    con = np.zeros((8192, 4), dtype=np.uint32)
    npw, nt, nc = sz(), sz(), sz()
    rc = f(words.ctypes.data, len(words), prog.ctypes.data, len(prog), ctypes.byref(npw), tgt.ctypes.data, len(tgt),
           ctypes.byref(nt), con.ctypes.data, len(con), ctypes.byref(nc))
    assert rc == 0
    return prog[:npw.value].astype(np.int64).tolist(), tgt[:nt.value], con[:nc.value]


def fill(prog, targets, contrib, Wcol):
    """What the weight prepass computes: Weff = sum W_col * coef, modulo 2^128."""
    for word, first, count, _ in targets:
        v = sum(Wcol[int(contrib[i][0])] * _s64(contrib[i][2], contrib[i][3]) for i in range(first, first + count))
        v &= (1 << 128) - 1
        for j in range(4):
            prog[int(word) + j] = (v >> (32 * j)) & 0xFFFFFFFF


def _runtime_posts(prog, T):
    """Post-ops left to the runtime min, summed over the table's pieces."""
    I = (T.w[14] + 3) & ~3   # the table's entry offset, rounded up to 4 words
    return sum(prog[I + 8 * p + 7] for p in range(T.w[5]))


def _check(ctx, v, lo, hi, rng, n_points=24):
    P = len(W.TEMPLATE_PARAMS[v.template])
    tid, _ = ctx.compile_counts(W.variant_ir(v), 32, [lo] * P, [hi] * P)
    words = ctx.table_image(tid)
    T = Table(words)
    prog, tgt, con = k2_program(words)
    corners = [[lo if (m >> i) & 1 else hi for i in range(P)] for m in range(1 << P)]
    pts = corners + [[int(x) for x in p] for p in W.draw_points(P, n_points, int(rng.integers(1 << 30)), lo, hi)]
    for trial in range(2):
        Wcol = [int(x) for x in rng.integers(-(1 << 55), 1 << 55, size=32)]
        if trial == 0:
            Wcol = [abs(x) for x in Wcol]   # non-negative weights, as fitted times usually are
        fill(prog, tgt, con, Wcol)
        for n in pts:
            ref = sum(Wcol[c] * x for c, x in enumerate(T.evaluate(n, check_magic=False)))
            assert program_dot(prog, T, n) == ref, (v.name, n)
    return _runtime_posts(prog, T), 2 * T.w[5]


@pytest.mark.parametrize("t", W.TEMPLATES)
def test_program_equals_weighted_counts(ctx, t):
    rng = np.random.default_rng(17)
    vs = [v for v in W.all_variants() if v.template == t]
    left = total = 0
    for v in [W.canonical(t, 2 if t == "copy" else 1)] + [vs[i] for i in rng.choice(len(vs), 6, replace=False)]:
        a, b = _check(ctx, v, 64, 65536, rng)
        left, total = left + a, total + b
    assert left < total   # some post-ops are decided over the box


def test_program_small_box_keeps_runtime_post_ops(ctx):
    """On [1, 96] tiles are partly empty and remainders dominate, so some post-ops
    cannot be decided over the box; the runtime min must then give the same value."""
    rng = np.random.default_rng(18)
    left = 0
    for v in W.tiny_variants() + [v for v in W.all_variants() if v.template in ("stencil", "transpose")][:6]:
        left += _check(ctx, v, 1, 96, rng, n_points=40)[0]
    assert left > 0   # and some are not


@pytest.mark.parametrize("t", W.COUPLED_TEMPLATES)
def test_program_coupled_denominator(ctx, t):
    """Tables with a denominator D (coupled domains): the program's 128-bit sum is
    D times the prediction and divides exactly."""
    rng = np.random.default_rng(19)
    vs = [v for v in W.coupled_variants() if v.template == t]
    for v in [vs[i] for i in rng.choice(len(vs), 5, replace=False)]:
        _check(ctx, v, 1, 65536, rng, n_points=16)


def test_program_random_kernels(ctx):
    """Random kernels (tiled axes, sequential loops, guards over one to three
    indices, strided accesses) on random boxes: each table's program equals the
    weighted counts at the box corners and inside, for signed and unsigned weights."""
    from test_compile_fuzz import _random_kernel
    rng = np.random.default_rng(72)
    checked = 0
    for _ in range(120):
        ir, P = _random_kernel(rng)
        lo, hi = int(rng.choice([0, 1, 64])), int(rng.choice([96, 4096, 65536]))
        try:
            tid, _ = ctx.compile_counts(ir, 32, [lo] * P, [hi] * P)
        except B.PMError:
            continue
        words = ctx.table_image(tid)
        T = Table(words)
        prog, tgt, con = k2_program(words)
        corners = [[lo if (m >> i) & 1 else hi for i in range(P)] for m in range(1 << P)]
        pts = corners + [[int(x) for x in rng.integers(lo, hi + 1, size=P)] for _ in range(6)]
        for trial in range(2):
            Wcol = [int(x) for x in rng.integers(-(1 << 55), 1 << 55, size=32)]
            if trial == 0:
                Wcol = [abs(x) for x in Wcol]
            fill(prog, tgt, con, Wcol)
            for n in pts:
                ref = sum(Wcol[c] * x for c, x in enumerate(T.evaluate(n, check_magic=False)))
                assert program_dot(prog, T, n) == ref, (ir, lo, hi, n)
        checked += 1
    assert checked > 40
