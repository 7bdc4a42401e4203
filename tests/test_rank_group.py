"""The fused ranking kernel's groups, checked on the CPU.

A ranking group gathers variants of one template: its basis holds every value their
tables use (parameters, atoms floor((a.n + b)/c), monomials, the constant), evaluated
once per point, and each table becomes a program whose piece is an exact dot product
of 128-bit weights with basis values (sum_col W_col sum_e coef_e slot_e = sum_slot
Weff_slot slot), plus the post-ops min(A, B) whose smaller operand depends on n.  A
test-only interpreter of the group image (the layout of csrc/kernels.h) must give
sum_col W_col p_col(n) exactly, p_col(n) from the table itself (checked against the
oracle in test_compile.py), for any weights, at points all over the box (corners
included, where a fold decision of a post-op is tightest)."""
import ctypes

import numpy as np
import pytest

from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import workloads as W
from table_interp import Table, _s32, _s64, _wide


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build_library()
    c = B.Context(-1)
    yield c
    c.close()


def rank_group(images):
    """pmx_rank_group: the group image of a list of table images and its weight-fill recipe."""
    L = B.lib()
    f = L.pmx_rank_group
    sz = ctypes.c_size_t
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, sz, ctypes.POINTER(sz),
                  ctypes.c_void_p, sz, ctypes.POINTER(sz), ctypes.c_void_p, sz, ctypes.POINTER(sz)]
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.uint32) for x in images]))
    words = np.array([len(x) for x in images], dtype=np.uint64)
    out = np.zeros(1 << 16, dtype=np.uint32)
    tgt = np.zeros((1 << 14, 4), dtype=np.uint32)
    con = np.zeros((1 << 15, 4), dtype=np.uint32)
    nw, nt, nc = sz(), sz(), sz()
    rc = f(flat.ctypes.data, words.ctypes.data, len(images), out.ctypes.data, len(out), ctypes.byref(nw),
           tgt.ctypes.data, len(tgt), ctypes.byref(nt), con.ctypes.data, len(con), ctypes.byref(nc))
    assert rc == 0, B.lib().pm_last_error().decode()
    return out[:nw.value].astype(np.int64).tolist(), tgt[:nt.value], con[:nc.value]


def fill(img, targets, contrib, Wcol):
    """What the weight prepass computes: Weff = sum W_col * coef, modulo 2^128; a 96-bit
    record (flag 1) keeps its fourth word (the term's basis entry), and its weight must
    fit in 96 signed bits."""
    for word, first, count, flags in targets:
        v = sum(Wcol[int(contrib[i][0])] * _s64(contrib[i][2], contrib[i][3]) for i in range(first, first + count))
        if flags & 1:
            assert -(1 << 95) <= v < (1 << 95)
        v &= (1 << 128) - 1
        for j in range(3 if flags & 1 else 4):
            img[int(word) + j] = (v >> (32 * j)) & 0xFFFFFFFF


def group_basis(img, n):
    """Basis values and the condition mask (bit q for condition q) of the group at n."""
    B_, nlev, ncond = img[0], img[1], img[2]
    off_b, off_c = img[12], img[13]
    n4 = list(n) + [0] * (4 - len(n))
    vals = []
    ends = img[4:4 + nlev]
    assert nlev == 0 or ends[-1] == B_
    for e in range(B_):
        d = img[off_b + 8 * e: off_b + 8 * e + 8]
        kind = d[7] & 3
        if kind == 0:
            vals.append(n4[d[0] & 3])
        elif kind == 1:
            vals.append(1)
        elif kind == 2:
            num = _s32(d[4]) + sum(_s32(d[q]) * n4[q] for q in range(4))
            vals.append(num // _s32(d[5]))
        else:
            assert d[0] < e and d[1] < e       # factors come first (levels)
            vals.append(vals[d[0]] * vals[d[1]])
        assert abs(vals[-1]) < (1 << 62)
    mask, o = 0, off_c
    assert ncond <= 64
    for q in range(ncond):
        nt = img[o]
        s = _s64(img[o + 1], img[o + 2]) + sum(_s64(img[o + 4 + 3 * k], img[o + 5 + 3 * k]) * vals[img[o + 3 + 3 * k]]
                                               for k in range(nt))
        assert abs(s) < (1 << 63)
        mask |= int(s >= 0) << q
        o += 3 + 3 * nt
    return vals, mask


def _w96(r):
    """A 96-bit signed weight from three words."""
    x = (r[0] & 0xFFFFFFFF) | ((r[1] & 0xFFFFFFFF) << 32) | ((r[2] & 0xFFFFFFFF) << 64)
    return x - (1 << 96) if x >= (1 << 95) else x


def _u16(img, off, i):
    return (img[off + i // 2] >> (16 * (i & 1))) & 0xFFFF


def positions(img):
    """The walk order: (position, variant index in the group) pairs, after checking
    that the runs cover every position once and that each program's leaves all have
    its run's shape."""
    n_runs, off_r = img[17], img[16]
    covered = []
    for r in range(n_runs):
        shape, first, count = img[off_r + 4 * r: off_r + 4 * r + 3]
        covered += list(range(first, first + count))
        for pos in range(first, first + count):
            if shape != 0xFFFF:
                for N in _leaves(img, _u16(img, img[14], pos)):
                    assert (N[0] >> 8) & 0xFF == shape & 0xFF and (N[0] >> 16) & 0xFF == shape >> 8
                    assert N[0] >> 24 == 0
    assert covered == list(range(len(covered)))
    vids = [_u16(img, img[15], p) for p in covered]
    assert sorted(vids) == list(range(len(vids)))
    return list(zip(covered, vids))


def _leaves(img, off):
    out, todo, seen = [], [off], set()
    while todo:
        o = todo.pop()
        if o in seen:
            continue
        seen.add(o)
        N = img[o: o + 4]
        if N[0] & 3 == 0:
            out.append(N)
        elif N[0] & 3 == 2:
            todo += [N[2] + 4 * i for i in range(1 << ((N[0] >> 8) & 0xFF))]
        else:
            nc = (N[0] >> 8) & 0xFF
            todo += [(N[0] >> 16) + 4 * ((img[N[3] + (b >> 2)] >> (8 * (b & 3))) & 0xFF) for b in range(1 << nc)]
    return out


def program_value(img, pos, vals, mask, den):
    """The kernel's exact value at walk position pos: D * prediction, divided by D."""
    off = _u16(img, img[14], pos)
    N = img[off: off + 4]
    while N[0] & 3:
        nc = (N[0] >> 8) & 0xFF
        bits = 0
        for c in range(nc):
            gi = (N[1] >> (6 * c)) & 63 if c < 5 else (N[2] >> (6 * (c - 5))) & 63
            bits |= ((mask >> gi) & 1) << c
        if N[0] & 3 == 1:
            piece = (img[N[3] + (bits >> 2)] >> (8 * (bits & 3))) & 0xFF
            off = (N[0] >> 16) + 4 * piece
        else:
            assert N[0] & 3 == 2
            off = N[2] + 4 * bits
        N = img[off: off + 4]
    n64, n32, nwide = (N[0] >> 8) & 0xFF, (N[0] >> 16) & 0xFF, N[0] >> 24
    r = N[1]
    assert N[3] == 1          # the constant's weight record is always present (zero if unused)
    S = _wide(img[r: r + 4])
    r += 4
    for i in range(n64 + n32):
        e = img[r + 3]
        if i >= n64 and _w96(img[r: r + 3]):
            assert 0 <= vals[e] < (1 << 32)      # the 32-bit class (padding terms weigh 0)
        S += _w96(img[r: r + 3]) * vals[e]
        r += 4
    for i in range(nwide):
        S += _wide(img[r: r + 4]) * vals[img[r + 4]]
        r += 8
    assert (N[2] != 0) == (den != 1)
    assert S % den == 0
    return S // den


def _check_group(images, pts, rng, trials=2):
    img, tgt, con = rank_group(images)
    tabs = [Table(x) for x in images]
    runtime = 0
    for trial in range(trials):
        Wcol = [int(x) for x in rng.integers(-(1 << 55), 1 << 55, size=32)]
        if trial == 0:
            Wcol = [abs(x) for x in Wcol]   # non-negative weights, as fitted times usually are
        fill(img, tgt, con, Wcol)
        walk = positions(img)
        assert len(walk) == len(tabs)
        for n in pts:
            vals, mask = group_basis(img, n)
            for pos, v in walk:
                T = tabs[v]
                ref = sum(Wcol[c] * x for c, x in enumerate(T.evaluate(n, check_magic=False)))
                assert program_value(img, pos, vals, mask, T.den) == ref, (v, n)
    return img


def _points(P, lo, hi, n, rng):
    corners = [[lo if (m >> i) & 1 else hi for i in range(P)] for m in range(1 << P)]
    if lo < 1:
        return corners + [[int(x) for x in rng.integers(lo, hi + 1, size=P)] for _ in range(n)]
    return corners + [[int(x) for x in p] for p in W.draw_points(P, n, int(rng.integers(1 << 30)), lo, hi)]


def _images(ctx, vs, lo, hi):
    out = []
    for v in vs:
        P = len(W.TEMPLATE_PARAMS[v.template])
        tid, _ = ctx.compile_counts(W.variant_ir(v), 32, [lo] * P, [hi] * P)
        out.append(ctx.table_image(tid))
    return out


@pytest.mark.parametrize("t", W.TEMPLATES)
def test_group_equals_weighted_counts(ctx, t):
    """One group over a template's canonical variant and six drawn ones (repeated, as
    duplicate variants are), on the batched workload's box."""
    rng = np.random.default_rng(17)
    vs = [v for v in W.all_variants() if v.template == t]
    pick = [W.canonical(t, 2 if t == "copy" else 1)] + [vs[i] for i in rng.choice(len(vs), 6, replace=False)]
    pick = pick + [pick[2], pick[0]]
    P = len(W.TEMPLATE_PARAMS[t])
    _check_group(_images(ctx, pick, 64, 65536), _points(P, 64, 65536, 16, rng), rng)


def _sub_nodes(img, n_var):
    """Sub nodes (leaves chosen by the signs of post-op differences) reachable from the
    variants' roots."""
    seen, count, todo = set(), 0, []
    for v in range(n_var):
        todo.append(_u16(img, img[14], v))
    while todo:
        off = todo.pop()
        if off in seen:
            continue
        seen.add(off)
        kind = img[off] & 3
        if kind == 1:
            nc = (img[off] >> 8) & 0xFF
            lut = img[off + 3]
            todo += list({(img[off] >> 16) + 4 * ((img[lut + (b >> 2)] >> (8 * (b & 3))) & 0xFF)
                          for b in range(1 << nc)})
        elif kind == 2:
            count += 1
    return count


def test_group_small_box_keeps_runtime_post_ops(ctx):
    """On [1, 96] tiles are partly empty and remainders dominate, so some post-ops
    cannot be decided over the box: their sign becomes a condition of the group and the
    piece a pair of leaves, which must give the same value as the runtime min."""
    rng = np.random.default_rng(18)
    subs = 0
    for t in ("stencil", "transpose", "matmul"):
        vs = [W.canonical(t)] + [v for v in W.all_variants() if v.template == t][:5]
        P = len(W.TEMPLATE_PARAMS[t])
        img = _check_group(_images(ctx, vs, 1, 96), _points(P, 1, 96, 24, rng), rng)
        subs += _sub_nodes(img, len(vs))
    assert subs > 0


@pytest.mark.parametrize("t", W.COUPLED_TEMPLATES)
def test_group_coupled_denominator(ctx, t):
    """Tables with a denominator D (coupled domains): the program's 128-bit sum is D
    times the prediction and divides exactly."""
    rng = np.random.default_rng(19)
    vs = [v for v in W.coupled_variants() if v.template == t]
    pick = [vs[i] for i in rng.choice(len(vs), 5, replace=False)]
    P = len(W.TEMPLATE_PARAMS[t])
    _check_group(_images(ctx, pick, 1, 65536), _points(P, 1, 65536, 10, rng), rng)


def test_group_whole_template_shares_the_basis(ctx):
    """All distinct matmul tables of the batched workload in one group: the basis
    holds each shared value once (far fewer entries than the tables' slots)."""
    rng = np.random.default_rng(20)
    vs = [v for v in W.all_variants() if v.template == "matmul"][::7][:40]
    imgs = _images(ctx, vs, 64, 65536)
    img = _check_group(imgs, _points(3, 64, 65536, 3, rng), rng, trials=1)
    slots = sum(Table(x).A + 3 for x in imgs)
    assert img[0] < slots / 4


def test_group_random_kernels(ctx):
    """Random kernels (tiled axes, sequential loops, guards over one to three indices,
    strided accesses) on random boxes, alone and three to a group: each program equals
    the weighted counts at the box corners and inside, for signed and unsigned weights."""
    from test_compile_fuzz import _random_kernel
    rng = np.random.default_rng(72)
    checked = 0
    by_box = {}
    for _ in range(150):
        ir, P = _random_kernel(rng)
        lo, hi = int(rng.choice([0, 1, 64])), int(rng.choice([96, 4096, 65536]))
        try:
            tid, _ = ctx.compile_counts(ir, 32, [lo] * P, [hi] * P)
        except B.PMError:
            continue
        words = ctx.table_image(tid)
        pts = _points(P, lo, hi, 4, rng)
        _check_group([words], pts, rng)
        by_box.setdefault((P, lo, hi), []).append(words)
        checked += 1
    assert checked > 40
    groups = 0
    for (P, lo, hi), ims in by_box.items():
        for k in range(0, len(ims) - 2, 3):
            _check_group(ims[k:k + 3], _points(P, lo, hi, 3, rng), rng, trials=1)
            groups += 1
    assert groups > 5


def rank_plan(ctx, b, slice_=0):
    """pmx_rank_plan: the host arrays of the fused ranking plan (before upload)."""
    L = B.lib()
    f = L.pmx_rank_plan
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    f.restype = ctypes.c_int
    f.argtypes = [vp, vp, vp, ctypes.c_int32, vp, ctypes.c_int32, vp, vp, sz, vp, sz, vp, sz, vp, sz, vp, sz, vp, sz,
                  vp, sz]
    t = np.ascontiguousarray(b.tables, dtype=np.int32)
    vo = np.ascontiguousarray(b.var_off, dtype=np.int32)
    po = np.ascontiguousarray(b.pt_off, dtype=np.int64)
    T = len(vo) - 1
    sizes = np.zeros(8, dtype=np.int64)
    rc = f(ctx.h, t.ctypes.data, vo.ctypes.data, T, po.ctypes.data, slice_, sizes.ctypes.data,
           None, 0, None, 0, None, 0, None, 0, None, 0, None, 0, None, 0)
    assert rc == 0, B.lib().pm_last_error().decode()
    img = np.zeros(sizes[0], dtype=np.uint32)
    tg = np.zeros((sizes[1], 4), dtype=np.uint32)
    cb = np.zeros((max(1, sizes[2]), 4), dtype=np.uint32)
    gr = np.zeros((sizes[3] * 2, 4), dtype=np.int32)
    tm = np.zeros((T * 3, 4), dtype=np.int32)
    ch = np.zeros((sizes[5], 4), dtype=np.int32)
    un = np.zeros((sizes[6], 2), dtype=np.int32)
    rc = f(ctx.h, t.ctypes.data, vo.ctypes.data, T, po.ctypes.data, slice_, sizes.ctypes.data,
           img.ctypes.data, len(img), tg.ctypes.data, len(tg), cb.ctypes.data, len(cb), gr.ctypes.data, len(gr),
           tm.ctypes.data, T * 3, ch.ctypes.data, len(ch), un.ctypes.data, len(un))
    assert rc == 0
    return dict(img=img.astype(np.int64).tolist(), targets=tg, contrib=cb, groups=gr.reshape(-1, 2, 4),
                tmpl=tm.reshape(-1, 3, 4), chunks=ch, units=un, slots=int(sizes[7]))


def _check_plan(ctx, b, slice_, rng, pts_per_template=3):
    pl = rank_plan(ctx, b, slice_)
    img = pl["img"]
    Wcol = [int(x) for x in rng.integers(-(1 << 56), 1 << 56, size=32)]
    fill(img, pl["targets"], pl["contrib"], Wcol)
    T = len(b.var_off) - 1
    # groups cover each template's variants contiguously, in order
    seen = {t: 0 for t in range(T)}
    for g0, g1 in pl["groups"]:
        t = int(g1[0])
        assert g0[2] == seen[t]
        seen[t] += int(g0[3])
    assert all(seen[t] == b.var_off[t + 1] - b.var_off[t] for t in range(T))
    # units cover every (chunk, group of its template) once; empty templates get one empty unit
    want = set()
    for c, (t, p0, n, slot) in enumerate(pl["chunks"]):
        gs = [g for g in range(len(pl["groups"])) if pl["groups"][g][1][0] == t]
        want |= {(c, g) for g in gs} if gs else {(c, -1)}
        assert (slot >= 0) == (len(gs) > 1)
    assert sorted(map(tuple, pl["units"].tolist())) == sorted(want)
    tabs = {}
    for gi, (g0, g1) in enumerate(pl["groups"]):
        t = int(g1[0])
        gimg = img[g0[0]: g0[0] + g0[1]]
        P = int(pl["tmpl"][t][0][0])
        for p in rng.choice(np.arange(b.pt_off[t], b.pt_off[t + 1]), pts_per_template, replace=False):
            n = [int(x) for x in b.points[p][:P]]
            vals, mask = group_basis(gimg, n)
            walk = positions(gimg)
            assert len(walk) == int(g0[3])
            for pos, v in walk:
                tid = int(b.tables[b.var_off[t] + g0[2] + v])
                if tid not in tabs:
                    tabs[tid] = Table(ctx.table_image(tid))
                T_ = tabs[tid]
                ref = sum(Wcol[c] * x for c, x in enumerate(T_.evaluate(n, check_magic=False)))
                assert program_value(gimg, pos, vals, mask, T_.den) == ref, (gi, v, n)
    return pl


def test_plan_batched_and_sliced(ctx):
    """The plan of a batched tuning space as uploaded: each template one group, and with a
    slice size of 100 several groups per template (partial slots for their chunks)."""
    from paper_1604_04997_gb300 import tuning
    rng = np.random.default_rng(30)
    b = tuning.build(ctx, n_variants=700, n_points=70, variant_seed=41, point_seed=42)
    pl = _check_plan(ctx, b, 0, rng)
    assert len(pl["groups"]) == len(b.templates) and pl["slots"] == 0
    pl = _check_plan(ctx, b, 100, rng, pts_per_template=2)
    assert len(pl["groups"]) > len(b.templates) and pl["slots"] > 0


def test_plan_coupled_and_empty_template(ctx):
    """Coupled-domain tables (denominators) and a template without variants."""
    from paper_1604_04997_gb300 import tuning
    rng = np.random.default_rng(31)
    b = tuning.build(ctx, n_variants=120, n_points=40, variant_seed=43, point_seed=44, coupled=True)
    _check_plan(ctx, b, 0, rng)
    # drop the variants of template 1
    vo = b.var_off.copy()
    keep = np.r_[b.tables[:vo[1]], b.tables[vo[2]:]]
    vo2 = vo.copy()
    vo2[2:] -= vo[2] - vo[1]
    b2 = tuning.Batched(b.templates, b.variants[:vo[1]] + b.variants[vo[2]:], keep.astype(np.int32), vo2,
                        b.points, b.pt_off, b.n_distinct)
    pl = _check_plan(ctx, b2, 0, rng)
    assert any(u[1] == -1 for u in pl["units"].tolist())


def test_plan_refuses_more_than_65536_variants(ctx):
    """A ranking entry keeps the variant index within its template in 16 bits: a
    template of 65,537 variants is refused before anything is built."""
    L = B.lib()
    f = L.pmx_rank_plan
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    f.restype = ctypes.c_int
    f.argtypes = [vp, vp, vp, ctypes.c_int32, vp, ctypes.c_int32, vp, vp, sz, vp, sz, vp, sz, vp, sz, vp, sz, vp, sz,
                  vp, sz]
    from paper_1604_04997_gb300 import tuning
    b = tuning.build(ctx, 16, 8)
    tid = int(b.tables[0])
    t = np.full(65537, tid, dtype=np.int32)
    vo = np.array([0, 65537], dtype=np.int32)
    po = np.array([0, 8], dtype=np.int64)
    sizes = np.zeros(8, dtype=np.int64)
    rc = f(ctx.h, t.ctypes.data, vo.ctypes.data, 1, po.ctypes.data, 0, sizes.ctypes.data,
           None, 0, None, 0, None, 0, None, 0, None, 0, None, 0, None, 0)
    assert B.ERRORS[rc] == "PM_ERR_INVALID_ARG"
    assert "65,536" in B.lib().pm_last_error().decode()
