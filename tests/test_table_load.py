"""Table images saved and loaded back (pm_table_load, checkpoint.py), on CPU.

Every table the compiler emits passes the host-side structural check and loads back
word for word; images with a broken header, offset, index, divisor magic or
denominator inverse are refused with PM_ERR_INVALID_ARG before anything reaches a
device; seeded single-word corruptions are either refused or, when accepted, still
index inside the image (the interpreter evaluates them without leaving it).
"""
import os

import numpy as np
import pytest

from paper_1604_04997_gb300 import binding as B
from paper_1604_04997_gb300 import checkpoint as CK
from paper_1604_04997_gb300 import workloads as W
from table_interp import Table

H_MAGIC, H_WORDS, H_NPARAMS, H_NATOMS, H_NCONDS, H_NPIECES, H_K = range(7)
H_OFF_ATOMS, H_OFF_CONDS, H_OFF_LUT, H_OFF_PIECES, H_OFF_PRODS, H_OFF_ENTRIES, H_OFF_POST = range(9, 16)
H_BOX_LO, H_DEN, H_DEN_SHIFT, H_DEN_INV = 16, 28, 29, 32


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build_library()
    c = B.Context(-1)
    yield c
    c.close()


def _compile(ctx, v, layout=32, lo=64, hi=65536):
    P = len(W.TEMPLATE_PARAMS[v.template])
    return ctx.compile_counts(W.variant_ir(v), layout, [lo] * P, [hi] * P)[0]


@pytest.fixture(scope="module")
def images(ctx):
    """Images of a sample of the tuning space, every coupled-domain variant, both
    layouts, and the measurement kernels."""
    from paper_1604_04997_gb300 import calibrate as C
    allv = W.all_variants()
    rng = np.random.default_rng(21)
    out = []
    for j in rng.choice(len(allv), 60, replace=False):
        out.append(ctx.table_image(_compile(ctx, allv[j])))
    for v in W.coupled_variants()[::4]:
        out.append(ctx.table_image(_compile(ctx, v, lo=1)))
    out.append(ctx.table_image(_compile(ctx, W.canonical("matmul"), layout=12)))
    for case in C.measurement_set(quick=True)[:12]:
        p = case.probe
        tid, _ = ctx.compile_counts(W.probe_ir(p), 32, [1] * p.n_params, [4096] * p.n_params)
        out.append(ctx.table_image(tid))
    return out


def _refused(ctx, img):
    with pytest.raises(B.PMError) as e:
        ctx.table_load(img)
    assert e.value.code == -1
    return str(e.value)


def test_every_compiled_table_loads_back(ctx, images):
    for img in images:
        tid = ctx.table_load(img)
        assert np.array_equal(ctx.table_image(tid), img)


def test_loaded_table_counts_equal(ctx):
    v = W.Variant("trmv", 256, 1, 2, False, 256)
    a = _compile(ctx, v, lo=1)
    b = ctx.table_load(ctx.table_image(a))
    ta, tb = Table(ctx.table_image(a)), Table(ctx.table_image(b))
    for n in W.draw_points(2, 32, 4):
        assert ta.evaluate([int(x) for x in n]) == tb.evaluate([int(x) for x in n])


def _first(img, pred, start, stop, step):
    for i in range(start, stop, step):
        if pred(i):
            return i
    pytest.skip("no such word in this image")


REFUSALS = [  # corruption, the check that refuses it
    ("magic", "magic or word count"),
    ("words", "magic or word count"),
    ("size", "magic or word count"),
    ("nparams", "header counts"),
    ("pieces", "header counts"),
    ("layout", "columns"),
    ("atoms_offset", "section offsets"),
    ("box", "parameter box"),
    ("atom_divisor", "atom divisor"),
    ("atom_magic", "atom magic"),
    ("atom_range", "atom range"),
    ("lut", "piece table"),
    ("product", "product operands"),
    ("entry_slot", "entry slot"),
    ("entry_col", "entry column or hold"),
    ("entry_flags", "entry flags"),
    ("unterminated", "unterminated column"),
    ("den", "denominator inverse"),
    ("den_shift", "denominator"),
    ("den_inv", "denominator inverse"),
]


@pytest.mark.parametrize("what,why", REFUSALS)
def test_corrupted_image_refused(ctx, what, why):
    # a table with an atom, conditions, several pieces, products and a denominator
    img = ctx.table_image(_compile(ctx, W.Variant("band", 256, 1, 2, False, 256), lo=1))
    w = img.copy()
    oa, ol, op, opr, oe = (int(w[k]) for k in (H_OFF_ATOMS, H_OFF_LUT, H_OFF_PIECES, H_OFF_PRODS, H_OFF_ENTRIES))
    A, NC, NP = int(w[H_NATOMS]), int(w[H_NCONDS]), int(w[H_NPIECES])
    assert A > 0 and NC > 0 and NP > 1 and int(w[H_DEN]) > 1
    if what == "magic":
        w[H_MAGIC] ^= 1
    elif what == "words":
        w[H_WORDS] += 4
    elif what == "size":
        w = w[:-4]
    elif what == "nparams":
        w[H_NPARAMS] = 5
    elif what == "pieces":
        w[H_NPIECES] = 0
    elif what == "layout":
        w[H_K] = 16
    elif what == "atoms_offset":
        w[H_OFF_ATOMS] = 8
    elif what == "box":
        w[H_BOX_LO] = 1 << 20
    elif what == "atom_divisor":
        w[oa + 5] = 1
    elif what == "atom_magic":
        w[oa + 6] ^= 2
    elif what == "atom_range":
        i = _first(w, lambda i: int(w[i]) != 0, oa, oa + 4, 1)
        w[i] = np.uint32(1 << 30)
    elif what == "lut":
        w[ol] = (int(w[ol]) & ~0xFF) | 0xFF
    elif what == "product":
        pn = int(w[op + 1])
        if pn == 0:
            pytest.skip("first piece has no products")
        w[opr + int(w[op])] |= 0xFF
    elif what == "entry_slot":
        w[oe + 2] = (int(w[oe + 2]) & ~0xFF00) | (22 << 8)
    elif what == "entry_col":
        w[oe + 2] = (int(w[oe + 2]) & ~0xFF) | 0x80
    elif what == "entry_flags":
        w[oe + 2] |= 1 << 24
    elif what == "unterminated":
        eb, en = int(w[op + 2]), int(w[op + 3])
        w[oe + 4 * (eb + en - 1) + 2] &= ~np.uint32(1 << 20)
    elif what == "den":
        w[H_DEN] = 6
    elif what == "den_shift":
        w[H_DEN_SHIFT] = 3
    elif what == "den_inv":
        w[H_DEN_INV] ^= 2
    assert _refused(ctx, w).endswith("rejected: " + why)


def test_post_offset_past_end_refused(ctx):
    img = ctx.table_image(_compile(ctx, W.Variant("matmul", 16, 16, 2, True, 256)))
    w = img.copy()
    w[H_OFF_POST] = w.size + 1
    assert "section offsets" in _refused(ctx, w)


def test_single_word_fuzz(ctx, images):
    """Seeded single-word corruptions of real images: each is refused, or accepted and
    then evaluable by the interpreter with every index inside the image."""
    rng = np.random.default_rng(99)
    accepted = refused = 0
    for img in images[::3]:
        for _ in range(40):
            w = img.copy()
            i = int(rng.integers(0, w.size))
            w[i] = np.uint32(rng.integers(0, 1 << 32)) if rng.random() < 0.5 else w[i] ^ np.uint32(1 << int(rng.integers(0, 32)))
            try:
                tid = ctx.table_load(w)
            except B.PMError as e:
                assert e.code == -1
                refused += 1
                continue
            accepted += 1
            T = Table(ctx.table_image(tid))
            P = int(w[H_NPARAMS])
            lo = [int(np.int32(w[H_BOX_LO + k])) for k in range(P)]
            hi = [int(np.int32(w[H_BOX_LO + 4 + k])) for k in range(P)]
            for _ in range(3):
                n = [int(rng.integers(a, b + 1)) for a, b in zip(lo, hi)]
                T.evaluate(n, check_exact=False)
    assert refused > 0 and accepted > 0


# ----------------------------------------------------------------------------- files

def test_checkpoint_round_trip(ctx, tmp_path):
    vs = [W.canonical(t) for t in ("copy", "matmul", "stencil")] + [W.Variant("band", 256, 1, 2, False, 256)]
    ids = [_compile(ctx, v, lo=1) for v in vs]
    wts = W.draw_weights(32, 3, 7)
    path = os.path.join(tmp_path, "space.pmck")
    CK.save(path, ctx, ids, names=[v.name for v in vs], weights=wts)
    ck = CK.load(path, ctx)
    assert ck.names == [v.name for v in vs]
    assert np.array_equal(ck.weights, wts)
    for a, b in zip(ids, ck.table_ids):
        assert np.array_equal(ctx.table_image(a), ctx.table_image(b))


def test_checkpoint_corruption_detected(ctx, tmp_path):
    path = os.path.join(tmp_path, "t.pmck")
    CK.save(path, ctx, [_compile(ctx, W.canonical("copy"))])
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x10
    bad = os.path.join(tmp_path, "bad.pmck")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(ValueError, match="checksum"):
        CK.load(bad, ctx)
    open(bad, "wb").write(bytes(raw[:20]))
    with pytest.raises(ValueError):
        CK.load(bad, ctx)


def test_named_arrays_round_trip(ctx, tmp_path):
    arrs = {"a": np.arange(12, dtype=np.int64).reshape(3, 4), "b": np.array([1.5, -2.0], dtype=np.float32),
            "c": np.zeros((0, 5), dtype=np.int32), "d": np.array(7, dtype=np.uint8), "e": np.array([True, False])}
    path = os.path.join(tmp_path, "arr.pmck")
    CK.save(path, ctx, [], arrays=arrs)
    ck = CK.load(path, ctx)
    assert ck.table_ids == [] and ck.weights is None and set(ck.arrays) == set(arrs)
    for k, v in arrs.items():
        assert ck.arrays[k].dtype == v.dtype and np.array_equal(ck.arrays[k], v), k
    with pytest.raises(ValueError, match="not storable"):
        CK.save(path, ctx, [], arrays={"s": np.array(["x"])})


def test_tuning_space_resumes(ctx, tmp_path):
    """A whole tuning space (variants of every template, duplicate draws sharing a
    table, both offset arrays, the points) and its weights, saved and loaded into a
    fresh context: the same space, each variant's table image unchanged."""
    from paper_1604_04997_gb300 import tuning
    b = tuning.build(ctx, n_variants=60, n_points=20, variant_seed=31, point_seed=32)
    w = W.draw_weights(32, 4, 33)
    path = os.path.join(tmp_path, "space.pmck")
    tuning.save_space(path, ctx, b, w)
    ctx2 = B.Context(-1)
    try:
        b2, w2 = tuning.load_space(path, ctx2)
        assert b2.templates == b.templates and b2.variants == b.variants
        assert np.array_equal(b2.var_off, b.var_off) and np.array_equal(b2.pt_off, b.pt_off)
        assert np.array_equal(b2.points, b.points) and np.array_equal(w2, w)
        assert b2.n_distinct == len(set(b.tables.tolist()))
        for t1, t2 in zip(b.tables, b2.tables):
            assert np.array_equal(ctx.table_image(int(t1)), ctx2.table_image(int(t2)))
        # duplicates still share one table
        assert len(set(b2.tables.tolist())) == len(set(b.tables.tolist()))
    finally:
        ctx2.close()
