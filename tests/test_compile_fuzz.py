"""The count compiler on malformed and mutated IR, on CPU.

Every input ends in a status, never a crash or a hang; every table the compiler
accepts counts exactly what the oracle's brute-force enumeration counts.  Includes
the inputs that once broke it: an access with no cell at the classification
instance (a division by zero), a statement domain of ~10^13 points at that instance
(an endless walk), a coupled guard whose bound on one index was dropped by a proof
that used that same index's constraints (an extra group counted), and a count of
exactly 2^62 at a box corner (let through by the range check).
"""
import re

import numpy as np
import pytest

import oracle
from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import workloads as W
from table_interp import Table

STATUS = {-2, -3, -4}   # parse error, unsupported form, range overflow


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build_library()
    c = B.Context(-1)
    yield c
    c.close()


def _compile(ctx, ir, P=1, lo=1, hi=65536):
    return ctx.compile_counts(ir, 32, [lo] * P, [hi] * P)


def _exact_or_refused(ctx, ir, P, points):
    try:
        tid, _ = _compile(ctx, ir, P)
    except B.PMError as e:
        assert e.code in STATUS, e
        return False
    T = Table(ctx.table_image(tid))
    ref = oracle.Kernel(ir).features(np.array(points), 32, "brute")
    for p, f in zip(points, ref):
        assert T.evaluate(list(p)) == list(f), p
    return True


def test_empty_footprint_is_refused(ctx):
    ir = """kernel t
param n
array a global f32 n,n
dim g g0 0 ceil(n/64)
dim l l0 0 64
dim jo seq 0 n
dim ji seq 0 -21474836481
stmt mac g,l,jo,ji
load a[64*g+l,jo+ji]
end
"""
    with pytest.raises(B.PMError) as e:
        _compile(ctx, ir)
    assert e.value.code == -3 and "stride class" in str(e.value)


def test_huge_classification_domain_is_refused(ctx):
    ir = """kernel t
param n
array a global f32 n,n
dim g g0 0 ceil(n/128)
dim l l0 0 128
dim ti seq 0 6713769118
stmt mac g,l,ti
guard ti < n
load a[128*g+l,ti]
end
"""
    with pytest.raises(B.PMError) as e:
        _compile(ctx, ir)
    assert e.value.code == -3 and "too large" in str(e.value)


def test_bound_dominated_only_through_its_own_index(ctx):
    """256 g + 2 ro + l < n with ro in {0}: once counted one group too many."""
    ir = """kernel t
param n
array x global f64 n
dim g g0 0 ceil(n/256)
dim ro seq 0 1
dim l l0 0 256
stmt body g,ro,l
guard 256*g+2*ro+l < n
load x[256*g+l]
end
"""
    _exact_or_refused(ctx, ir, 1, [[n] for n in (1, 2, 3, 40, 255, 256, 257, 600)])


def test_coupled_guard_with_unequal_tile_coefficient(ctx):
    """Triangular matvec whose tile guard was mutated to g + l < n."""
    ir = W.variant_ir(W.Variant("trmv", 64, 1, 8, False, 64)).replace("guard 64*g+l < n", "guard 1*g+l < n", 1)
    assert "1*g+l" in ir
    _exact_or_refused(ctx, ir, 1, [[n] for n in (1, 9, 38, 64, 65, 130)])


_NUM = re.compile(r"(?<![A-Za-z_0-9])\d+")
_OPS = ["<", "<=", ">", ">="]


def _mutate(rng, text):
    lines = text.split("\n")
    for _ in range(rng.integers(1, 4)):
        k = rng.integers(len(lines))
        ln = lines[k]
        r = rng.random()
        if r < 0.6 and not ln.startswith("array"):
            ms = list(_NUM.finditer(ln))
            if ms:
                m = ms[rng.integers(len(ms))]
                v = int(rng.integers(0, 4)) if rng.random() < 0.4 else int(rng.integers(0, 40))
                ln = ln[:m.start()] + str(v) + ln[m.end():]
        elif r < 0.85 and ln.startswith("guard"):
            for o in ("<=", ">=", "<", ">"):
                if f" {o} " in ln:
                    ln = ln.replace(f" {o} ", f" {_OPS[rng.integers(4)]} ", 1)
                    break
        elif ln.startswith("guard"):
            ln = ln.replace("+", "-", 1) if rng.random() < 0.5 else ln.replace("-", "+", 1)
        lines[k] = ln
    return "\n".join(lines)


def test_mutated_templates_exact_or_refused(ctx):
    """Seeded mutations of template IR (constants, comparison operators, signs): each
    compiles to a table equal to brute force at random small points, or is refused."""
    rng = np.random.default_rng(2024)
    srcs = [W.variant_ir(W.canonical(t)) for t in W.TEMPLATES]
    srcs += [W.variant_ir(v) for v in W.coupled_variants()[::6]]
    accepted = 0
    for _ in range(160):
        ir = _mutate(rng, srcs[rng.integers(len(srcs))])
        P = len(re.search(r"^param (.*)$", ir, re.M).group(1).split())
        pts = rng.integers(1, 41, size=(3, P)).tolist()
        accepted += _exact_or_refused(ctx, ir, P, pts)
    assert accepted > 60


def test_garbled_text_always_gives_a_status(ctx):
    """Byte-level damage (deleted spans, inserted tokens, duplicated or dropped lines,
    huge numbers): every call returns, with a table or a status."""
    rng = np.random.default_rng(7)
    srcs = [W.variant_ir(W.canonical(t)) for t in W.TEMPLATES]
    toks = ["0", "-1", "n", "i", "+", "*", "/", "<", ">=", "floor(", ")", ",", "\n", "dim", "stmt", "end", "guard",
            "load", "param", "barrier", "x4", "1099511627776", "2147483648", "seq", "l0", "[", "]"]
    codes = set()
    for _ in range(400):
        s = srcs[rng.integers(len(srcs))]
        for _ in range(rng.integers(1, 4)):
            op = rng.integers(5)
            if op == 0:
                a = rng.integers(len(s))
                s = s[:a] + s[a + rng.integers(1, 8):]
            elif op == 1:
                a = rng.integers(len(s) + 1)
                s = s[:a] + toks[rng.integers(len(toks))] + s[a:]
            elif op == 2:
                a = rng.integers(len(s) + 1)
                s = s[:a] + str(int(rng.integers(-10 ** 12, 10 ** 12))) + s[a:]
            else:
                L = s.split("\n")
                k = rng.integers(len(L))
                L.insert(k, L[k]) if op == 3 else L.pop(k)
                s = "\n".join(L)
        try:
            _compile(ctx, s, 4)
            codes.add(0)
        except B.PMError as e:
            assert e.code in STATUS | {-1}, e
            codes.add(e.code)
    assert {0, -2} <= codes


def test_injected_coupled_guards_exact_or_refused(ctx):
    """Extra guards coupling two or three indices of a statement (coefficients in
    -2..2, a parameter, a shifted parameter or a constant on the right) added to the
    coupled and tiled templates: every accepted table equals brute force."""
    rng = np.random.default_rng(41)
    srcs = [W.variant_ir(v) for v in W.coupled_variants()[::5]]
    srcs += [W.variant_ir(W.canonical(t)) for t in ("matmul", "stencil", "transpose")]
    accepted = 0
    for _ in range(90):
        s = srcs[rng.integers(len(srcs))]
        lines = s.split("\n")
        params = re.search(r"^param (.*)$", s, re.M).group(1).split()
        stmts = [(i, ln.split()[2].split(",")) for i, ln in enumerate(lines) if ln.startswith("stmt ")]
        i, dims = stmts[rng.integers(len(stmts))]
        if len(dims) < 2:
            continue
        pick = rng.choice(dims, int(rng.integers(2, min(3, len(dims)) + 1)), replace=False)
        lhs = "+".join(f"{int(rng.choice([-2, -1, 1, 1, 2]))}*{d}" for d in pick).replace("+-", "-")
        p = params[rng.integers(len(params))]
        rhs = [p, f"{p}-{int(rng.integers(0, 5))}", str(int(rng.integers(0, 40))), f"2*{p}"][rng.integers(4)]
        lines.insert(i + 1, f"guard {lhs} {_OPS[rng.integers(4)]} {rhs}")
        ir = "\n".join(lines)
        accepted += _exact_or_refused(ctx, ir, len(params), rng.integers(1, 33, size=(3, len(params))).tolist())
    assert accepted > 10


def test_lane_mask_inside_a_tiled_axis(ctx):
    """64 g + l < n together with l < 20 (a lane mask) and l >= 3: the tiled axis is
    split into its indices and counted by the coupled-domain counter (such kernels
    were refused before); exact at ragged and full tiles."""
    ir = """kernel t
param n
array x global f32 n
dim g g0 0 ceil(n/64)
dim l l0 0 64
stmt body g,l
guard 64*g+l < n
guard l < 20
guard l >= 3
load x[64*g+l]
flop f32 add 1
end
"""
    assert _exact_or_refused(ctx, ir, 1, [[n] for n in (1, 3, 4, 19, 20, 21, 64, 65, 84, 100, 128, 1000)])


def _random_kernel(rng):
    P = int(rng.integers(1, 3))
    params = ["n", "m"][:P]
    pick = lambda: params[rng.integers(P)]
    T = int(rng.choice([4, 8, 16]))
    dims = [("g", "g0", "0", f"ceil({pick()}/{T})"), ("l", "l0", "0", str(T))]
    for i in range(int(rng.integers(1, 4))):
        hi = [pick(), str(int(rng.integers(1, 9))), f"ceil({pick()}/{int(rng.integers(2, 5))})",
              f"{pick()}+{int(rng.integers(0, 3))}"][rng.integers(4)]
        dims.append((f"s{i}", "seq", "0" if rng.random() < 0.8 else str(int(rng.integers(0, 3))), hi))
    ext = "64*n+64" if P == 1 else "64*n+64*m+64"
    lines = ["kernel r", "param " + " ".join(params), f"array a global f32 {ext}", f"array b global f32 {ext}"]
    lines += [f"dim {d[0]} {d[1]} {d[2]} {d[3]}" for d in dims]
    for si in range(int(rng.integers(1, 3))):
        used = ["g", "l"] + [d[0] for d in dims[2:] if rng.random() < 0.7]
        lines.append(f"stmt st{si} " + ",".join(used))
        if rng.random() < 0.8:
            lines.append(f"guard {T}*g+l < {pick()}")
        for _ in range(int(rng.integers(0, 3))):
            vs = rng.choice(used, int(rng.integers(1, min(3, len(used)) + 1)), replace=False)
            lhs = "+".join(f"{int(rng.choice([-1, 1, 1, 2]))}*{v}" for v in vs).replace("+-", "-")
            rhs = [pick(), f"{pick()}-{int(rng.integers(0, 4))}", str(int(rng.integers(0, 20))),
                   f"{pick()}+{int(rng.integers(0, 4))}"][rng.integers(4)]
            lines.append(f"guard {lhs} {_OPS[rng.integers(4)]} {rhs}")
        lines.append(f"flop f32 add {int(rng.integers(1, 3))}")
        idx = "+".join(f"{int(rng.integers(1, 3))}*{v}" for v in used)
        lines.append(f"load a[{T}*g+l]" if rng.random() < 0.5 else f"load a[{idx}]")
        if rng.random() < 0.5:
            lines.append(f"store b[{T}*g+l]")
        lines.append("end")
    return "\n".join(lines) + "\n", P


def test_random_kernels_exact_or_refused(ctx):
    """Random kernels (tiled group and local axes, sequential loops with affine,
    ceil or constant bounds, guards over one to three indices, strided accesses):
    each accepted table equals brute force."""
    rng = np.random.default_rng(62)
    accepted = 0
    for _ in range(150):
        ir, P = _random_kernel(rng)
        try:
            tid, _ = ctx.compile_counts(ir, 32, [1] * P, [4096] * P)
        except B.PMError as e:
            assert e.code in STATUS, e
            continue
        accepted += 1
        T = Table(ctx.table_image(tid))
        pts = rng.integers(1, 25, size=(3, P))
        for p, f in zip(pts, oracle.Kernel(ir).features(pts, 32, "brute")):
            assert T.evaluate([int(x) for x in p]) == list(f), (ir, p)
    assert accepted > 50


def test_count_of_exactly_2_62_is_refused(ctx):
    """A count that reaches 2^62 at the box corner (65,536 x 65,536 x 16,384 x 65,536
    points) is refused; one point less on n is accepted."""
    ir = """kernel r
param n m
array a global f32 64*n+64*m+64
dim g g0 0 ceil(m/8)
dim l l0 0 8
dim s0 seq 2 n+2
dim s1 seq 0 ceil(n/4)
dim s2 seq 0 n
stmt st0 g,l,s0,s1,s2
guard 8*g+l < n
flop f32 add 1
store a[8*g+l]
end
"""
    with pytest.raises(B.PMError) as e:
        ctx.compile_counts(ir, 32, [1, 1], [65536, 65536])
    assert e.value.code == -4
    tid, _ = ctx.compile_counts(ir, 32, [1, 1], [65535, 65536])
    assert Table(ctx.table_image(tid)).evaluate([65535, 65536])[3] == 65535 ** 3 * 16384   # (g, l), s0, s2: 65535; s1: 16384


def _rich_kernel(rng):
    P = int(rng.integers(1, 3))
    params = ["n", "m"][:P]
    pick = lambda: params[rng.integers(P)]
    T = int(rng.choice([4, 8, 16]))
    dims = [("g", "g0", "0", f"ceil({pick()}/{T})"), ("l", "l0", "0", str(T))]
    for i in range(int(rng.integers(1, 3))):
        hi = [pick(), str(int(rng.integers(1, 6))), f"ceil({pick()}/{int(rng.integers(2, 5))})"][rng.integers(3)]
        dims.append((f"s{i}", "seq", "0", hi))
    ext = "64*n+64" if P == 1 else "64*n+64*m+64"
    lines = ["kernel r", "param " + " ".join(params), f"array a global f32 {ext}", f"array d global f64 {ext}",
             f"array sh local f32 {4 * T}"]
    lines += [f"dim {d[0]} {d[1]} {d[2]} {d[3]}" for d in dims]
    seqs = [d[0] for d in dims[2:]]
    for si in range(int(rng.integers(1, 4))):
        used = ["g", "l"] + [x for x in seqs if rng.random() < 0.7]
        lines.append(f"stmt st{si} " + ",".join(used))
        if rng.random() < 0.8:
            lines.append(f"guard {T}*g+l < {pick()}")
        if rng.random() < 0.5:
            vs = rng.choice(used, int(rng.integers(1, min(3, len(used)) + 1)), replace=False)
            lhs = "+".join(f"{int(rng.choice([-1, 1, 1]))}*{v}" for v in vs).replace("+-", "-")
            lines.append(f"guard {lhs} {_OPS[rng.integers(4)]} {[pick(), str(int(rng.integers(0, 12)))][rng.integers(2)]}")
        for _ in range(int(rng.integers(1, 3))):
            lines.append(f"flop {rng.choice(['f32', 'f64'])} {rng.choice(['add', 'mul', 'div', 'pow', 'spec'])} "
                         f"{int(rng.integers(1, 4))}")
        lines.append([f"load a[{T}*g+l]", f"load d[{T}*g+l]", f"load a[{2 * T}*g+2*l] x2", f"load a[{4 * T}*g+4*l] x4",
                      f"load a[{int(rng.integers(2, 5))}*({T}*g+l)]"][rng.integers(5)])
        if rng.random() < 0.5:
            lines.append("store sh[l]")
        if rng.random() < 0.5:
            lines.append(f"load sh[{T}+l]")
        if rng.random() < 0.4:
            lines.append(f"store d[{T}*g+l]")
        lines.append("end")
        if rng.random() < 0.5 and seqs:
            lines.append(f"barrier b{si} " + ",".join(["g"] + [x for x in seqs if rng.random() < 0.6]))
    return "\n".join(lines) + "\n", P


def test_rich_random_kernels_exact_or_refused(ctx):
    """Random kernels with barriers, local memory, 64- and 128-bit and strided global
    accesses, f64 and every flop kind, in both layouts: each accepted table equals
    brute force."""
    rng = np.random.default_rng(91)
    accepted = 0
    for _ in range(100):
        ir, P = _rich_kernel(rng)
        layout = 32 if rng.random() < 0.7 else 12
        try:
            tid, _ = ctx.compile_counts(ir, layout, [1] * P, [4096] * P)
        except B.PMError as e:
            assert e.code in STATUS, e
            continue
        accepted += 1
        T = Table(ctx.table_image(tid))
        pts = rng.integers(1, 25, size=(3, P))
        for p, f in zip(pts, oracle.Kernel(ir).features(pts, layout, "brute")):
            assert T.evaluate([int(x) for x in p]) == list(f), (ir, layout, p)
    assert accepted > 40
