"""The count compiler (host side of pm_compile_counts) against the oracle, on CPU.

Compiled tables are read back through the C ABI and evaluated by a test-only
interpreter; the oracle computes the same counts by brute force / per-axis.
"""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import workloads as W
from table_interp import Table, magic_div

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build_library()
    c = B.Context(-1)
    yield c
    c.close()


def test_library_exports_every_declared_symbol(ctx):
    decl = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", h)).read(), flags=re.S)
        decl |= set(re.findall(r"\b(pmm?_[a-z_0-9]+)\s*\(", text))
    L = B.lib()
    missing = [s for s in decl if not hasattr(L, s)]
    assert not missing and set(B.exported_symbols()) <= decl


@pytest.mark.parametrize("t", W.TEMPLATES)
def test_small_n_all_pieces(ctx, t):
    """Every n in [1, 96] on the box [1, 65536]: remainder tiles and small-n pieces."""
    for v in [W.canonical(t, 2 if t == "copy" else 1)] + [
            x for i, x in enumerate(v for v in W.all_variants() if v.template == t) if i % 37 == 3][:4]:
        ir = W.variant_ir(v)
        P = len(W.TEMPLATE_PARAMS[t])
        tid, info = ctx.compile_counts(ir, 32, [1] * P, [65536] * P)
        T = Table(ctx.table_image(tid))
        k = oracle.Kernel(ir)
        if P == 1:
            pts = np.arange(1, 97).reshape(-1, 1)
        else:
            vals = [1, 2, 15, 16, 17, 33, 64, 96]
            pts = np.array([(a, b, c) for a in vals for b in vals for c in vals])
        ref = k.features(pts, 32, "struct")
        for p, f in zip(pts, ref):
            assert T.evaluate([int(x) for x in p]) == list(f), (v.name, p)


def test_layout12_with_hidden_column(ctx):
    for v in W.tiny_variants():
        ir = W.variant_ir(v)
        P = len(W.TEMPLATE_PARAMS[v.template])
        tid, _ = ctx.compile_counts(ir, 12, [1] * P, [8192] * P)
        T = Table(ctx.table_image(tid))
        k = oracle.Kernel(ir)
        pts = W.tiny_points(v.template, 32, (64, 128, 256, 8192))
        ref = k.features(pts, 12, "struct")
        for p, f in zip(pts, ref):
            assert T.evaluate([int(x) for x in p]) == list(f)


def test_tuning_space_sample(ctx):
    """Random variants of the tuning space at log-uniform points of [64, 65536]."""
    allv = W.all_variants()
    rng = np.random.default_rng(5)
    for j in rng.choice(len(allv), 120, replace=False):
        v = allv[j]
        P = len(W.TEMPLATE_PARAMS[v.template])
        ir = W.variant_ir(v)
        tid, info = ctx.compile_counts(ir, 32, [64] * P, [65536] * P)
        assert info["n_words"] <= 1024
        T = Table(ctx.table_image(tid))
        pts = W.draw_points(P, 16, int(j))
        ref = oracle.Kernel(ir).features(pts, 32, "struct")
        for p, f in zip(pts, ref):
            assert T.evaluate([int(x) for x in p]) == list(f), v.name


def test_magic_division():
    """Granlund-Montgomery constants reproduce floor division for 32-bit numerators."""
    from table_interp import _s32
    rng = np.random.default_rng(1)
    ctx = B.Context(-1)
    for c in list(range(2, 70)) + [97, 255, 256, 1000, 4095, 4096, 65535, 65536, 1 << 20]:
        ir = f"kernel d\nparam n\ndim g g0 0 floor((n+7)/{c})\nstmt s g\nflop f32 add 1\nend\n"
        tid, _ = ctx.compile_counts(ir, 32, [0], [(1 << 30) - 8])
        T = Table(ctx.table_image(tid))
        (at,) = T.atoms()
        assert at["c"] == c or c % at["c"] == 0
        xs = np.concatenate([rng.integers(0, 1 << 31, 2000), np.arange(0, 3 * c), [(1 << 31) - 1]])
        for x in xs:
            assert magic_div(int(x), at["m"], at["sh2"]) == int(x) // at["c"]


@pytest.mark.parametrize("ir,code", [
    # coupled guard with no index of unit coefficient: no closed-form chamber sum
    ("kernel c\nparam n\ndim i g0 0 n\ndim j seq 0 n\nstmt s i,j\nguard 2*i+3*j < n\nflop f32 add 1\nend\n", -3),
    # a coupled triangle whose count reaches n^4 / 24 with n up to 2^20: beyond 2^62 / D
    ("kernel c\nparam n\ndim a g0 0 n\ndim b seq 0 n\ndim c seq 0 n\ndim d seq 0 n\n"
     "stmt s a,b,c,d\nguard b < a\nguard c < b\nguard d < c\nflop f32 add 1000\nend\n", -4),
    ("kernel c\nparam n\ndim i g0 0 n\nstmt s i\nload a[i]\nend\n", -2),
    # n^3 * n with n up to 2^20 leaves int64
    ("kernel c\nparam n\ndim a g0 0 n\ndim b seq 0 n\ndim c seq 0 n\ndim d seq 0 n\n"
     "stmt s a,b,c,d\nflop f32 add 1000\nend\n", -4),
])
def test_compile_errors(ir, code):
    ctx = B.Context(-1)
    with pytest.raises(B.PMError) as e:
        ctx.compile_counts(ir, 32, [1], [1 << 20])
    assert e.value.code == code


def test_loopy_example_table(ctx):
    ir = open(os.path.join(os.path.dirname(__file__), "golden", "loopy_double.ir")).read()
    tid, info = ctx.compile_counts(ir, 32, [1], [1 << 20])
    T = Table(ctx.table_image(tid))
    for n in (1, 7, 64, 65, 1000, 1 << 20):
        F = T.evaluate([n])
        assert (F[4], F[17], F[24], F[1]) == (n, n, n, -(-n // 64))


def test_measurement_config_checks_need_no_gpu(ctx):
    """pmm_time rejects bad configurations before touching the device."""
    for kw in (dict(kind="copy", n=0), dict(kind="vsa", variant=0, n=1024), dict(kind="arith", variant=7, k=8, n=64),
               dict(kind="matmul", gx=8, gy=8, n=64, m=64, l=64), dict(kind="reduction", variant=8, gx=256, n=4096),
               dict(kind="copy", n=1024, gx=2048)):
        with pytest.raises(B.PMError) as e:
            B.pmm_time(**kw, runs=5, skip=1)
        assert e.value.code == -1
    with pytest.raises(B.PMError):
        B.pmm_time("copy", n=1024, runs=4, skip=4)


def test_probe_tables_match_oracle(ctx):
    """The measurement and test kernels' IR (the CUDA kernels' operation counts),
    compiled, against the oracle's brute-force counting at small sizes."""
    from paper_1604_04997_gb300 import calibrate as C
    seen = set()
    for case in C.measurement_set(quick=True) + C.test_set(quick=True):
        p = case.probe
        if p in seen:
            continue
        seen.add(p)
        small = W.Probe(p.kind, p.variant, min(p.k, 4), min(p.gx, 16), min(p.gy, 16), p.f64) \
            if p.kind in ("arith", "filled", "empty") else p
        ir = W.probe_ir(small)
        P = small.n_params
        tid, _ = ctx.compile_counts(ir, 32, [1] * P, [4096] * P)
        T = Table(ctx.table_image(tid))
        sizes = [(40,), (64,), (70,)] if P == 1 else [(40, 24, 36), (64, 32, 64), (33, 17, 48)]
        for n in sizes:
            ref = oracle.Kernel(ir).features(np.array([n]), 32, "brute")[0]
            assert T.evaluate(list(n)) == list(ref), (small.name, n)


# ----------------------------------------------------------------------------- coupled domains

def _check_table(T, k, pts, method):
    ref = k.features(pts, 32, method)
    for p, f in zip(pts, ref):
        assert T.evaluate([int(x) for x in p]) == list(f), p


@pytest.mark.parametrize("t", W.COUPLED_TEMPLATES)
def test_coupled_templates(ctx, t):
    """Triangles and bands, every variant of the template on the box [1, 65536]: small
    sizes against brute force, log-uniform points against the per-axis oracle.  The
    counts are sums of powers over chambers, so the tables carry a denominator."""
    P = len(W.TEMPLATE_PARAMS[t])
    rng = np.random.default_rng(31)
    small = np.arange(1, 34).reshape(-1, 1) if P == 1 else \
        np.array([(a, b) for a in (1, 2, 5, 17, 33) for b in (1, 2, 9, 40)])
    vs = [v for v in W.coupled_variants() if v.template == t]
    for v in vs[::3] if t == "syrk" else vs:
        ir = W.variant_ir(v)
        tid, info = ctx.compile_counts(ir, 32, [1] * P, [65536] * P)
        T = Table(ctx.table_image(tid))
        assert T.den > 1 and info["n_pieces"] <= 8
        k = oracle.Kernel(ir)
        _check_table(T, k, small[::3] if t == "syrk" else small, "brute")
        _check_table(T, k, W.draw_points(P, 8, int(rng.integers(1 << 30)), 1, 65536), "struct")


_TET = """kernel tet
param n
array a global f32 n,n
dim i g0 0 n
dim j seq 0 n
dim k seq 0 n
stmt s i,j,k
guard j < i
guard k < j
load a[i,k]
flop f32 mul 1
end
"""

_BLOCKED = """kernel btr
param n
array a global f32 n,n
dim g g0 0 ceil(n/16)
dim jt seq 0 ceil(n/16)
dim l l0 0 16
dim jj seq 0 16
stmt s g,jt,l,jj
guard jt <= g
guard 16*g+l < n
guard 16*jt+jj < n
guard 16*jt+jj <= 16*g+l
load a[16*g+l,16*jt+jj]
flop f32 mul 1
end
"""


def test_coupled_shapes(ctx):
    """A three-index chain k < j < i (C(n,3) points: cubic, denominator 6), a guard with
    a non-unit coefficient on one index (2j < i), and a blocked triangle whose tile
    guard jt <= g is implied by the element guard (kept as one collapsed index pair)."""
    for ir, lo, hi, pieces in ((_TET, 1, 4096, None), (_TET.replace("guard k < j", "guard 2*k < j"), 1, 4096, None),
                               (_BLOCKED, 1, 65536, 1)):
        tid, info = ctx.compile_counts(ir, 32, [lo], [hi])
        T = Table(ctx.table_image(tid))
        assert pieces is None or info["n_pieces"] == pieces
        k = oracle.Kernel(ir)
        _check_table(T, k, np.arange(1, 30).reshape(-1, 1), "brute")
        _check_table(T, k, np.array([[97], [1000], [4095], [4096]] + ([[65535]] if hi > 4096 else [])), "struct")
    T = Table(ctx.table_image(ctx.compile_counts(_TET, 32, [1], [4096])[0]))
    assert T.den == 6 and T.evaluate([100])[4] == 100 * 99 * 98 // 6


def test_coupled_unsupported(ctx):
    """Guards that leave no index with unit coefficients are refused, not miscounted."""
    ir = _TET.replace("guard j < i\nguard k < j", "guard 2*i+3*j < n")
    with pytest.raises(B.PMError) as e:
        ctx.compile_counts(ir, 32, [1], [4096])
    assert e.value.code == -3


def test_coupled_layout12(ctx):
    """The 12-column layout of coupled-domain tables (denominator included) against the
    oracle's 12-column features."""
    for t in W.COUPLED_TEMPLATES:
        v = [v for v in W.coupled_variants() if v.template == t][5]
        ir = W.variant_ir(v)
        P = len(W.TEMPLATE_PARAMS[t])
        tid, _ = ctx.compile_counts(ir, 12, [1] * P, [65536] * P)
        T = Table(ctx.table_image(tid))
        pts = W.draw_points(P, 10, 77, 1, 4096)
        ref = oracle.Kernel(ir).features(pts, 12, "struct")
        for p, f in zip(pts, ref):
            assert T.evaluate([int(x) for x in p]) == list(f), (v.name, p)


def test_denominator_cancels(ctx):
    """Two triangles j < i and j > i feeding the same columns sum to n(n-1): integer
    coefficients, so the table's denominator reduces to 1; one triangle alone keeps 2."""
    body = """kernel offdiag
param n
array a global f32 n,n
dim i g0 0 n
dim j seq 0 n
stmt lo i,j
guard j < i
load a[i,j]
flop f32 add 1
end
stmt up i,j
guard j > i
load a[i,j]
flop f32 add 1
end
"""
    T = Table(ctx.table_image(ctx.compile_counts(body, 32, [1], [65536])[0]))
    assert T.den == 1
    k = oracle.Kernel(body)
    for n in (1, 2, 3, 100, 65536):
        assert T.evaluate([n]) == list(k.features([[n]], 32, "struct")[0])
        assert T.evaluate([n])[3] == n * (n - 1)
    one = body.split("stmt up")[0]
    assert Table(ctx.table_image(ctx.compile_counts(one, 32, [1], [65536])[0])).den == 2


def test_serve_stats_struct_matches_the_binding(ctx):
    """pm_serve_stats on a context without a serve loop clears the whole C struct:
    the binding's struct must cover it exactly (guard bytes past it stay intact) and
    every field reads zero."""
    import ctypes
    n = ctypes.sizeof(B.ServeStats)
    buf = (ctypes.c_uint8 * (n + 32))(*([0xAB] * (n + 32)))
    assert B.lib().pm_serve_stats(ctx.h, 0, ctypes.cast(buf, ctypes.POINTER(B.ServeStats))) == 0
    assert all(b == 0 for b in buf[:n]) and all(b == 0xAB for b in buf[n:])
    assert all(v == 0 for v in ctx.serve_stats().values()) and "n_rejected" in ctx.serve_stats()
