"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the bench.

This module holds no counting, prediction or fitting arithmetic: it only writes
kernel descriptions in the affine loop-nest IR, draws tuning-space variants and
parameter points, and draws weights / noisy timings that stand in for the
paper's hardware measurement step (Fig. 1, "Hardware measurement").

IR text format (one directive per line, tokens separated by blanks,
expressions contain no blanks, ``#`` starts a comment)::

    kernel NAME
    param P1 [P2 ...]                       # at most 4 size parameters (Sec. 2, vector n)
    array NAME global|local f32|f64 EXT[,EXT...]   # row-major extents, affine in params
    dim NAME g0|g1|g2|l0|l1|l2|seq LO HI     # loop index range [LO, HI), quasi-affine in params
    stmt NAME DIM[,DIM...]                   # an instruction, run once per point of its dims
      guard LHS <|<=|>|>= RHS                # affine in the statement's dims and params
      flop f32|f64 add|mul|div|pow|spec COUNT
      load ARRAY[IDX,...] [x2|x4]
      store ARRAY[IDX,...] [x2|x4]
    end
    barrier NAME DIM[,DIM...]                # one barrier per point of its (group/seq) dims

The IR mirrors the Loopy model of a kernel (Sec. 3.1): a loop domain and scalar
instructions, each executed once per integer point of the projection of the
domain onto its own loop indices.  Barriers are explicit, as a schedule would
place them (Sec. 3.2, last paragraph).  Group dims (g*) form the launch grid;
local dims (l*) are work-item indices, l0 being the SIMD-lane axis used by the
amortized stride fraction (Sec. 2.1).

The eight templates follow the paper's measurement and test kernel families
(Sec. 4.1, Sec. 5): vector add, axpy, strided copy, local-tile transpose,
tiled matmul, 5-point stencil, local-memory tree reduction, batched matvec.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

TEMPLATES = ("vecadd", "axpy", "copy", "transpose", "matmul", "stencil", "reduction", "matvec")
# Kernels whose loop domains couple indices (triangles, bands): their counts are sums
# of powers over piece chambers rather than products of per-axis intervals.
COUPLED_TEMPLATES = ("trmv", "syrk", "band", "pairs")
TEMPLATE_PARAMS = {
    "vecadd": ("n",), "axpy": ("n",), "copy": ("n",), "transpose": ("n",),
    "matmul": ("n", "m", "l"), "stencil": ("n",), "reduction": ("n",), "matvec": ("b",),
    "trmv": ("n",), "syrk": ("n", "m"), "band": ("n", "w"), "pairs": ("n",),
}
TILES = (8, 16, 32, 64)
UNROLLS = (1, 2, 4, 8)
WGS = (64, 128, 256, 512)
STRIDES = (1, 2, 4, 8, 16)

# Paper-style parameter box of the batched tuning workload.
BOX_LO, BOX_HI = 64, 65536


@dataclasses.dataclass(frozen=True)
class Variant:
    template: str
    tx: int
    ty: int
    unroll: int
    prefetch: bool
    wg: int
    stride: int = 1  # only meaningful for the strided copy

    @property
    def key(self) -> Tuple:
        return (self.template, self.tx, self.ty, self.unroll, self.prefetch, self.wg, self.stride)

    @property
    def name(self) -> str:
        return (f"{self.template}_t{self.tx}x{self.ty}_u{self.unroll}_p{int(self.prefetch)}"
                f"_w{self.wg}" + (f"_s{self.stride}" if self.template == "copy" else ""))


def _lin(terms: Sequence[Tuple[int, str]], const: int = 0) -> str:
    """Render sum(coef*name) + const without blanks, dropping zero/empty terms."""
    out = []
    for c, v in terms:
        if c == 0:
            continue
        out.append(v if c == 1 else f"{c}*{v}")
    s = "+".join(out) if out else ""
    if const:
        s = f"{s}+{const}" if s else str(const) if const > 0 else str(const)
        s = s.replace("+-", "-")
    return s or "0"


# --------------------------------------------------------------------------- templates

def _one_d(v: Variant, dtype: str, body) -> str:
    """Shared 1-D blocking: E = tx*ty elements per group, wg items, E/wg per item."""
    E, W, u = v.tx * v.ty, v.wg, v.unroll
    R = E // W
    X = _lin([(E, "g"), (u * W, "ro"), (W, "ri"), (1, "l")])
    lines = [
        f"dim g g0 0 ceil(n/{E})",
        f"dim ro seq 0 {R // u}",
        f"dim ri seq 0 {u}",
        f"dim l l0 0 {W}",
        "stmt body g,ro,ri,l",
        f"guard {X} < n",
    ]
    lines += body(X)
    lines.append("end")
    return "\n".join(lines)


def ir_vecadd(v: Variant) -> str:
    head = [f"kernel {v.name}", "param n",
            "array a global f32 n", "array b global f32 n", "array c global f32 n"]
    body = lambda X: [f"load a[{X}]", f"load b[{X}]", "flop f32 add 1", f"store c[{X}]"]
    return "\n".join(head) + "\n" + _one_d(v, "f32", body) + "\n"


def ir_axpy(v: Variant) -> str:
    head = [f"kernel {v.name}", "param n", "array x global f64 n", "array y global f64 n"]
    body = lambda X: [f"load x[{X}]", f"load y[{X}]", "flop f64 mul 1", "flop f64 add 1",
                      f"store y[{X}]"]
    return "\n".join(head) + "\n" + _one_d(v, "f64", body) + "\n"


def ir_copy(v: Variant) -> str:
    s = v.stride
    head = [f"kernel {v.name}", "param n", f"array a global f32 {s}*n" if s > 1 else
            "array a global f32 n", "array b global f32 n"]
    body = lambda X: [f"load a[{s}*({X})]" if s > 1 else f"load a[{X}]", f"store b[{X}]"]
    return "\n".join(head) + "\n" + _one_d(v, "f32", body) + "\n"


def ir_reduction(v: Variant) -> str:
    E, W, u = v.tx * v.ty, v.wg, v.unroll
    R = E // W
    X = _lin([(E, "g"), (u * W, "ro"), (W, "ri"), (1, "l")])
    L = [f"kernel {v.name}", "param n",
         "array a global f32 n", f"array out global f32 ceil(n/{E})", f"array s local f32 {W}",
         f"dim g g0 0 ceil(n/{E})", f"dim ro seq 0 {R // u}", f"dim ri seq 0 {u}",
         f"dim l l0 0 {W}",
         "stmt acc g,ro,ri,l", f"guard {X} < n", f"load a[{X}]", "flop f32 add 1", "end",
         "stmt put g,l", "store s[l]", "end",
         "barrier b0 g"]
    stages = int(math.log2(W))
    S = W // 2
    for k in range(1, stages + 1):
        L += [f"stmt r{k} g,l", f"guard l < {S}", "load s[l]", f"load s[l+{S}]",
              "flop f32 add 1", "store s[l]", "end"]
        if k < stages:
            L.append(f"barrier b{k} g")
        S //= 2
    L += ["stmt fin g", "load s[0]", "store out[g]", "end"]
    return "\n".join(L) + "\n"


def ir_transpose(v: Variant) -> str:
    T, W, u = v.tx, v.wg, v.unroll
    WY = W // T
    RY = T // WY
    R = _lin([(u * WY, "ro"), (WY, "ri"), (1, "ly")])
    Y = _lin([(T, "gy"), (u * WY, "ro"), (WY, "ri"), (1, "ly")])
    X = _lin([(T, "gx"), (1, "lx")])
    Yt = _lin([(T, "gx"), (u * WY, "ro"), (WY, "ri"), (1, "ly")])   # output row
    Xt = _lin([(T, "gy"), (1, "lx")])                               # output col
    dims = "gx,gy,ro,ri,ly,lx"
    L = [f"kernel {v.name}", "param n", "array in global f32 n,n", "array out global f32 n,n"]
    if v.prefetch:
        L.append(f"array t local f32 {T},{T + 1}")
    L += [f"dim gx g0 0 ceil(n/{T})", f"dim gy g1 0 ceil(n/{T})",
          f"dim ro seq 0 {RY // u}", f"dim ri seq 0 {u}",
          f"dim ly l1 0 {WY}", f"dim lx l0 0 {T}"]
    if v.prefetch:
        L += [f"stmt ld {dims}", f"guard {Y} < n", f"guard {X} < n",
              f"load in[{Y},{X}]", f"store t[{R},lx]", "end",
              "barrier b1 gx,gy",
              f"stmt st {dims}", f"guard {Yt} < n", f"guard {Xt} < n",
              f"load t[lx,{R}]", f"store out[{Yt},{Xt}]", "end"]
    else:
        L += [f"stmt cp {dims}", f"guard {Y} < n", f"guard {X} < n",
              f"load in[{Y},{X}]", f"store out[{X},{Y}]", "end"]
    return "\n".join(L) + "\n"


def ir_matmul(v: Variant) -> str:
    TX, TY, W, u = v.tx, v.ty, v.wg, v.unroll
    WY = W // TX
    RY, RK = TY // WY, TX // WY
    Y = _lin([(TY, "gy"), (WY, "ry"), (1, "ly")])
    X = _lin([(TX, "gx"), (1, "lx")])
    L = [f"kernel {v.name}", "param n m l",
         "array A global f32 n,m", "array B global f32 m,l", "array C global f32 n,l"]
    if v.prefetch:
        L += [f"array As local f32 {TY},{TX}", f"array Bs local f32 {TX},{TX}"]
    L += [f"dim gx g0 0 ceil(l/{TX})", f"dim gy g1 0 ceil(n/{TY})",
          f"dim ry seq 0 {RY}", f"dim ly l1 0 {WY}", f"dim lx l0 0 {TX}"]
    if v.prefetch:
        K = _lin([(TX, "kt"), (u, "ko"), (1, "ki")])
        Kb = _lin([(TX, "kt"), (WY, "rk"), (1, "ly")])
        L += [f"dim kt seq 0 ceil(m/{TX})", f"dim rk seq 0 {RK}",
              f"dim ko seq 0 {TX // u}", f"dim ki seq 0 {u}",
              "stmt lda gx,gy,kt,ry,ly,lx", f"guard {Y} < n", f"guard {_lin([(TX, 'kt'), (1, 'lx')])} < m",
              f"load A[{Y},{_lin([(TX, 'kt'), (1, 'lx')])}]", f"store As[{_lin([(WY, 'ry'), (1, 'ly')])},lx]", "end",
              "stmt ldb gx,gy,kt,rk,ly,lx", f"guard {Kb} < m", f"guard {X} < l",
              f"load B[{Kb},{X}]", f"store Bs[{_lin([(WY, 'rk'), (1, 'ly')])},lx]", "end",
              "barrier b1 gx,gy,kt",
              "stmt mac gx,gy,kt,ry,ko,ki,ly,lx", f"guard {Y} < n", f"guard {X} < l", f"guard {K} < m",
              f"load As[{_lin([(WY, 'ry'), (1, 'ly')])},{_lin([(u, 'ko'), (1, 'ki')])}]",
              f"load Bs[{_lin([(u, 'ko'), (1, 'ki')])},lx]",
              "flop f32 mul 1", "flop f32 add 1", "end",
              "barrier b2 gx,gy,kt"]
    else:
        Km = _lin([(u, "ko"), (1, "ki")])
        L += [f"dim ko seq 0 floor(m/{u})", f"dim ki seq 0 {u}",
              f"dim kr seq {u}*floor(m/{u}) m" if u > 1 else "dim kr seq m m",
              "stmt mac gx,gy,ry,ko,ki,ly,lx", f"guard {Y} < n", f"guard {X} < l",
              f"load A[{Y},{Km}]", f"load B[{Km},{X}]", "flop f32 mul 1", "flop f32 add 1", "end",
              "stmt rem gx,gy,ry,kr,ly,lx", f"guard {Y} < n", f"guard {X} < l",
              f"load A[{Y},kr]", f"load B[kr,{X}]", "flop f32 mul 1", "flop f32 add 1", "end"]
    L += ["stmt st gx,gy,ry,ly,lx", f"guard {Y} < n", f"guard {X} < l",
          f"store C[{Y},{X}]", "end"]
    return "\n".join(L) + "\n"


def ir_stencil(v: Variant) -> str:
    TX, TY, W, u = v.tx, v.ty, v.wg, v.unroll
    WY = W // TX
    RY = TY // WY
    R = _lin([(u * WY, "ro"), (WY, "ri"), (1, "ly")])
    Y1 = _lin([(TY, "gy"), (u * WY, "ro"), (WY, "ri"), (1, "ly")], 1)   # interior row
    X1 = _lin([(TX, "gx"), (1, "lx")], 1)                               # interior col
    dims = "gx,gy,ro,ri,ly,lx"
    L = [f"kernel {v.name}", "param n", "array u global f32 n,n", "array v global f32 n,n"]
    if v.prefetch:
        L.append(f"array t local f32 {TY + 2},{TX + 2}")
    L += [f"dim gx g0 0 ceil((n-2)/{TX})", f"dim gy g1 0 ceil((n-2)/{TY})",
          f"dim ro seq 0 {RY // u}", f"dim ri seq 0 {u}",
          f"dim ly l1 0 {WY}", f"dim lx l0 0 {TX}"]
    flops = ["flop f32 add 4", "flop f32 mul 2"]
    if v.prefetch:
        L += [f"stmt c {dims}", f"guard {Y1} < n", f"guard {X1} < n",
              f"load u[{Y1},{X1}]", f"store t[{R}+1,lx+1]", "end",
              "stmt ht gx,gy,lx", f"guard {X1} < n",
              f"load u[{TY}*gy,{X1}]", "store t[0,lx+1]", "end",
              "stmt hb gx,gy,lx", f"guard {TY}*gy+{TY + 1} < n", f"guard {X1} < n",
              f"load u[{TY}*gy+{TY + 1},{X1}]", f"store t[{TY + 1},lx+1]", "end",
              "stmt hl gx,gy,ro,ri,ly", f"guard {Y1} < n",
              f"load u[{Y1},{TX}*gx]", f"store t[{R}+1,0]", "end",
              "stmt hr gx,gy,ro,ri,ly", f"guard {TX}*gx+{TX + 1} < n", f"guard {Y1} < n",
              f"load u[{Y1},{TX}*gx+{TX + 1}]", f"store t[{R}+1,{TX + 1}]", "end",
              "barrier b1 gx,gy",
              f"stmt pt {dims}", f"guard {Y1} < n-1", f"guard {X1} < n-1",
              f"load t[{R},lx+1]", f"load t[{R}+2,lx+1]", f"load t[{R}+1,lx]",
              f"load t[{R}+1,lx+2]", f"load t[{R}+1,lx+1]"] + flops + [f"store v[{Y1},{X1}]", "end"]
    else:
        L += [f"stmt pt {dims}", f"guard {Y1} < n-1", f"guard {X1} < n-1",
              f"load u[{Y1}-1,{X1}]", f"load u[{Y1}+1,{X1}]", f"load u[{Y1},{X1}-1]",
              f"load u[{Y1},{X1}+1]", f"load u[{Y1},{X1}]"] + flops + [f"store v[{Y1},{X1}]", "end"]
    return "\n".join(L) + "\n"


def ir_matvec(v: Variant) -> str:
    W, u = v.wg, v.unroll
    MPG = W // 32
    M = _lin([(MPG, "g"), (1, "lm")])
    K = _lin([(u, "ko"), (1, "ki")])
    L = [f"kernel {v.name}", "param b", "array A global f64 b,32,32",
         "array x global f64 b,32", "array y global f64 b,32"]
    if v.prefetch:
        L.append(f"array xs local f64 {MPG},32")
    L += [f"dim g g0 0 ceil(b/{MPG})", f"dim lm l1 0 {MPG}", "dim lr l0 0 32",
          f"dim ko seq 0 {32 // u}", f"dim ki seq 0 {u}"]
    if v.prefetch:
        L += ["stmt lx g,lm,lr", f"guard {M} < b", f"load x[{M},lr]", "store xs[lm,lr]", "end",
              "barrier b1 g",
              "stmt mac g,lm,lr,ko,ki", f"guard {M} < b", f"load A[{M},lr,{K}]",
              f"load xs[lm,{K}]", "flop f64 mul 1", "flop f64 add 1", "end"]
    else:
        L += ["stmt mac g,lm,lr,ko,ki", f"guard {M} < b", f"load A[{M},lr,{K}]",
              f"load x[{M},{K}]", "flop f64 mul 1", "flop f64 add 1", "end"]
    L += ["stmt st g,lm,lr", f"guard {M} < b", f"store y[{M},lr]", "end"]
    return "\n".join(L) + "\n"


# --------------------------------------------------------------------------- coupled domains

def _rows(v: Variant) -> Tuple[List[str], str, str]:
    """Row-per-work-item blocking of the 1-D coupled templates (wg rows per group) and
    an unrolled inner index J = u*jo + ji over [0, ceil(extent/u)*u)."""
    W, u = v.wg, v.unroll
    return [f"dim g g0 0 ceil(n/{W})", f"dim l l0 0 {W}"], _lin([(W, "g"), (1, "l")]), \
        _lin([(u, "jo"), (1, "ji")])


def ir_trmv(v: Variant) -> str:
    """y = L x with L lower triangular (diagonal included): row i sums over j <= i."""
    dims, I, J = _rows(v)
    u = v.unroll
    L = [f"kernel {v.name}", "param n", "array a global f32 n,n", "array x global f32 n",
         "array y global f32 n"] + dims + [
        f"dim jo seq 0 ceil(n/{u})", f"dim ji seq 0 {u}",
        "stmt mac g,l,jo,ji", f"guard {I} < n", f"guard {J} < n", f"guard {J} <= {I}",
        f"load a[{I},{J}]", f"load x[{J}]", "flop f32 mul 1", "flop f32 add 1", "end",
        "stmt st g,l", f"guard {I} < n", f"store y[{I}]", "end"]
    return "\n".join(L) + "\n"


def ir_pairs(v: Variant) -> str:
    """Pairwise interactions over j < i (each pair once, as in a symmetric n-body step):
    relative position, r^2 + eps, rsqrt, r^-3 m and the force accumulation."""
    dims, I, J = _rows(v)
    u = v.unroll
    L = [f"kernel {v.name}", "param n", "array p global f32 n,4", "array f global f32 n,4"] + dims + [
        f"dim jo seq 0 ceil(n/{u})", f"dim ji seq 0 {u}",
        "stmt own g,l", f"guard {I} < n", f"load p[{I},0]", f"load p[{I},1]", f"load p[{I},2]", "end",
        "stmt pair g,l,jo,ji", f"guard {I} < n", f"guard {J} < n", f"guard {J} < {I}",
        f"load p[{J},0]", f"load p[{J},1]", f"load p[{J},2]", f"load p[{J},3]",
        "flop f32 add 9", "flop f32 mul 9", "flop f32 spec 1", "end",
        "stmt st g,l", f"guard {I} < n", f"store f[{I},0]", f"store f[{I},1]", f"store f[{I},2]", "end"]
    return "\n".join(L) + "\n"


def ir_band(v: Variant) -> str:
    """y = A x for A banded with half-bandwidth w, stored as n x (2w+1): row i reads
    x[i - w + t] for the t in [0, 2w] that land inside [0, n)."""
    dims, I, T = _rows(v)
    T = _lin([(v.unroll, "to"), (1, "ti")])
    u = v.unroll
    L = [f"kernel {v.name}", "param n w", "array a global f32 n,2*w+1", "array x global f32 n",
         "array y global f32 n"] + dims + [
        f"dim to seq 0 ceil((2*w+1)/{u})", f"dim ti seq 0 {u}",
        "stmt mac g,l,to,ti", f"guard {I} < n", f"guard {T} < 2*w+1", f"guard {I}+{T} >= w",
        f"guard {I}+{T} < n+w", f"load a[{I},{T}]", f"load x[{I}+{T}-w]", "flop f32 mul 1", "flop f32 add 1",
        "end", "stmt st g,l", f"guard {I} < n", f"store y[{I}]", "end"]
    return "\n".join(L) + "\n"


def ir_syrk(v: Variant) -> str:
    """Lower triangle of C = A A^T (A: n x m): tx x ty tiles of C per group, column
    index on the lanes, the m-loop unrolled by u; only entries with j <= i."""
    tx, ty, u = v.tx, v.ty, v.unroll
    I, J, K = _lin([(ty, "gy"), (1, "ly")]), _lin([(tx, "gx"), (1, "lx")]), _lin([(u, "ko"), (1, "ki")])
    tri = [f"guard {J} < n", f"guard {I} < n", f"guard {J} <= {I}"]
    L = [f"kernel {v.name}", "param n m", "array A global f32 n,m", "array C global f32 n,n",
         f"dim gx g0 0 ceil(n/{tx})", f"dim gy g1 0 ceil(n/{ty})", f"dim ly l1 0 {ty}", f"dim lx l0 0 {tx}",
         f"dim ko seq 0 ceil(m/{u})", f"dim ki seq 0 {u}",
         "stmt mac gx,gy,ly,lx,ko,ki"] + tri + [f"guard {K} < m", f"load A[{I},{K}]", f"load A[{J},{K}]",
                                                "flop f32 mul 1", "flop f32 add 1", "end",
                                                "stmt st gx,gy,ly,lx"] + tri + [f"store C[{I},{J}]", "end"]
    return "\n".join(L) + "\n"


_IR = {"vecadd": ir_vecadd, "axpy": ir_axpy, "copy": ir_copy, "transpose": ir_transpose,
       "matmul": ir_matmul, "stencil": ir_stencil, "reduction": ir_reduction, "matvec": ir_matvec,
       "trmv": ir_trmv, "pairs": ir_pairs, "band": ir_band, "syrk": ir_syrk}


def variant_ir(v: Variant) -> str:
    if not valid(v):
        raise ValueError(f"invalid variant {v}")
    return _IR[v.template](v)


def valid(v: Variant) -> bool:
    """Which knob combinations are meaningful for each template (others are redrawn)."""
    t, tx, ty, u, p, W = v.template, v.tx, v.ty, v.unroll, v.prefetch, v.wg
    if v.stride != 1 and t != "copy":
        return False
    if t in ("vecadd", "axpy", "copy", "reduction"):
        E = tx * ty
        return (not p) and E % W == 0 and (E // W) % u == 0
    if t == "transpose":
        if tx != ty or W > tx * tx or W % tx:
            return False
        WY = W // tx
        return tx % WY == 0 and (tx // WY) % u == 0
    if t == "matmul":
        if W % tx:
            return False
        WY = W // tx
        if WY > ty or ty % WY or tx % WY:
            return False
        return (tx % u == 0) if p else True
    if t == "stencil":
        if W % tx:
            return False
        WY = W // tx
        return WY <= ty and ty % WY == 0 and ((ty // WY) % u == 0)
    if t == "matvec":
        return (tx, ty) == (8, 8) and 32 % u == 0
    if t in ("trmv", "pairs", "band"):
        return (not p) and tx == W and ty == 1
    if t == "syrk":
        return (not p) and tx * ty == W
    return False


def canonical(template: str, stride: int = 1) -> Variant:
    """The fixed small-workload instance: 16x16 tile, 256-item groups, no unroll,
    local prefetch where it applies."""
    pre = template in ("transpose", "matmul", "stencil", "matvec")
    tx, ty = (8, 8) if template == "matvec" else (16, 16)
    return Variant(template, tx, ty, 1, pre, 256, stride)


def all_variants() -> List[Variant]:
    out = []
    for t in TEMPLATES:
        for tx in TILES:
            for ty in TILES:
                for u in UNROLLS:
                    for p in (False, True):
                        for W in WGS:
                            for s in (STRIDES if t == "copy" else (1,)):
                                v = Variant(t, tx, ty, u, p, W, s)
                                if valid(v):
                                    out.append(v)
    return out


def coupled_variants() -> List[Variant]:
    """The tuning space of the coupled-domain templates: rows per group (trmv, pairs,
    band) or the C tile (syrk) and the inner unroll."""
    out = []
    for t in COUPLED_TEMPLATES:
        for W in WGS:
            for u in UNROLLS:
                if t == "syrk":
                    out += [Variant(t, tx, W // tx, u, False, W) for tx in TILES if W // tx in TILES]
                else:
                    out.append(Variant(t, W, 1, u, False, W))
    return out


def draw_coupled_variants(n_variants: int, seed: int = 12) -> List[Variant]:
    """Coupled-domain variants drawn uniformly with replacement (duplicates tie)."""
    allv = coupled_variants()
    rng = np.random.default_rng(seed)
    return [allv[i] for i in rng.integers(len(allv), size=n_variants)]


def draw_variants(n_variants: int, seed: int = 2) -> List[Variant]:
    """Draw variants with replacement from the tuning space: template, tile in
    {8..64}^2, unroll in {1,2,4,8}, prefetch on/off, work-group size in {64..512}.
    Invalid combinations are redrawn, so duplicates occur (exact prediction ties)."""
    rng = np.random.default_rng(seed)
    out: List[Variant] = []
    while len(out) < n_variants:
        t = TEMPLATES[rng.integers(len(TEMPLATES))]
        v = Variant(t, int(rng.choice(TILES)), int(rng.choice(TILES)), int(rng.choice(UNROLLS)),
                    bool(rng.integers(2)), int(rng.choice(WGS)),
                    int(rng.choice(STRIDES)) if t == "copy" else 1)
        if valid(v):
            out.append(v)
    return out


def group_by_template(variants: Sequence[Variant], templates: Sequence[str] = TEMPLATES) -> Dict[str, List[int]]:
    g: Dict[str, List[int]] = {t: [] for t in templates}
    for i, v in enumerate(variants):
        g[v.template].append(i)
    return g


def draw_points(n_params: int, n_points: int, seed: int, lo: int = BOX_LO, hi: int = BOX_HI) -> np.ndarray:
    """Log-uniform integer parameter points in [lo, hi], int64 [n_points][n_params]."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size=(n_points, n_params)))
    return np.clip(np.floor(x), lo, hi).astype(np.int64)


def template_points(seed: int, n_points: int, lo: int = BOX_LO, hi: int = BOX_HI,
                    templates: Sequence[str] = TEMPLATES) -> Dict[str, np.ndarray]:
    """One independent point set per template (seed offset by template index)."""
    return {t: draw_points(len(TEMPLATE_PARAMS[t]), n_points, seed * 1000 + i, lo, hi)
            for i, t in enumerate(templates)}


@dataclasses.dataclass
class Space:
    """A batched tuning space before compilation: variants in template-major order,
    CSR offsets per template, and each template's points padded to 4 parameters."""
    templates: List[str]
    variants: List[Variant]
    var_off: np.ndarray      # int32 [T+1]
    points: np.ndarray       # int64 [total][4]
    pt_off: np.ndarray       # int64 [T+1]


def batched_space(n_variants: int = 10000, n_points: int = 4096, variant_seed: int = 2, point_seed: int = 3,
                  lo: int = BOX_LO, hi: int = BOX_HI, coupled: bool = False) -> Space:
    """The batched tuning workload: variants drawn with replacement from the tuning
    space over the eight templates (or, with coupled=True, over the coupled-domain
    templates), grouped by template; n_points log-uniform points per template."""
    templates = COUPLED_TEMPLATES if coupled else TEMPLATES
    drawn = draw_coupled_variants(n_variants, variant_seed) if coupled else draw_variants(n_variants, variant_seed)
    groups = group_by_template(drawn, templates)
    pts = template_points(point_seed, n_points, lo, hi, templates)
    variants, var_off, rows, pt_off = [], [0], [], [0]
    for t in templates:
        variants += [drawn[i] for i in groups[t]]
        var_off.append(len(variants))
        p = np.zeros((n_points, 4), dtype=np.int64)
        p[:, :pts[t].shape[1]] = pts[t]
        rows.append(p)
        pt_off.append(pt_off[-1] + n_points)
    return Space(list(templates), variants, np.array(var_off, dtype=np.int32), np.concatenate(rows),
                 np.array(pt_off, dtype=np.int64))


def draw_weights(k: int, n_models: int, seed: int, lo: float = 1e-12, hi: float = 1e-9) -> np.ndarray:
    """Per-device weight vectors, uniform in [lo, hi] (units: seconds per operation)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n_models, k))


@dataclasses.dataclass
class QueryDraw:
    arrival_s: float          # arrival time from the start of the stream
    template: int             # index into TEMPLATES
    model: int
    variant: np.ndarray       # int64 [n] variant index within the template's list
    point: np.ndarray         # int64 [n] point index within the template's point set


def draw_queries(n_queries: int, rate_per_s: float, n_variants: Sequence[int], n_points: int, n_models: int = 64,
                 seed: int = 9, max_cand: int = 50000) -> List[QueryDraw]:
    """Autotuner query stream: Poisson arrivals at rate_per_s; each query picks a
    template and a model uniformly and n candidates log-uniform in [1, max_cand],
    each a (variant, point) pair drawn uniformly from that template's variants
    (n_variants[t] of them) and its n_points points."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_queries)
    live = [t for t in range(len(n_variants)) if n_variants[t] > 0]
    out = []
    t_arr = 0.0
    for i in range(n_queries):
        t_arr += float(gaps[i])
        t = live[int(rng.integers(len(live)))]
        n = int(min(max_cand, math.floor(math.exp(rng.uniform(0.0, math.log(max_cand + 1))))))
        n = max(1, n)
        out.append(QueryDraw(t_arr, t, int(rng.integers(n_models)), rng.integers(n_variants[t], size=n),
                             rng.integers(n_points, size=n)))
    return out


# --------------------------------------------------------------------------- measurement kernels

PROBE_KINDS = ("empty", "copy", "sum4", "index", "vsa", "filled", "arith", "transpose_p", "transpose_r",
               "transpose_w", "matmul", "matmul_naive", "stencil", "matvec", "reduction", "axpy", "vecadd",
               "nbody", "conv5")
ARITH_TYPES = ("add", "mul", "div", "pow", "spec")


@dataclasses.dataclass(frozen=True)
class Probe:
    """One measurement or test kernel configuration (Sec. 4.1, Sec. 5): its kind, a
    kind-specific variant (stride for vsa/filled, index into ARITH_TYPES for arith,
    tile for the 2-D tiled kinds), an inner trip count k (arith, filled) and the
    work-group size gx (x gy)."""
    kind: str
    variant: int = 0
    k: int = 0
    gx: int = 256
    gy: int = 1
    f64: bool = False   # fp64 data and arithmetic (copy, vsa, arith add/mul/div)

    @property
    def n_params(self) -> int:
        return 3 if self.kind in ("matmul", "matmul_naive") else 1

    @property
    def name(self) -> str:
        return f"{self.kind}{'64' if self.f64 else ''}_v{self.variant}_k{self.k}_g{self.gx}x{self.gy}"


def _probe_1d(p: Probe, head: List[str], body: List[str]) -> str:
    W = p.gx
    X = f"{W}*g+l"
    L = [f"kernel {p.name}", "param n"] + head + [f"dim g g0 0 ceil(n/{W})", f"dim l l0 0 {W}",
                                                  "stmt s g,l", f"guard {X} < n"]
    return "\n".join(L + [b.replace("X", X) for b in body] + ["end"]) + "\n"


def probe_ir(p: Probe) -> str:
    """The IR of a measurement/test kernel; the CUDA kernel of the same Probe performs
    exactly these loads, stores, flops and barriers per work-item."""
    k, s, W = p.kind, p.variant, p.gx
    dt = "f64" if p.f64 else "f32"
    if k == "copy":
        return _probe_1d(p, [f"array a global {dt} n", f"array b global {dt} n"], ["load a[X]", "store b[X]"])
    if k == "sum4":
        return _probe_1d(p, [f"array a{i} global {dt} n" for i in range(4)] + [f"array c global {dt} n"],
                         [f"load a{i}[X]" for i in range(4)] + [f"flop {dt} add 3", "store c[X]"])
    if k == "index":
        return _probe_1d(p, [f"array a global {dt} n"], ["store a[X]"])
    if k == "vsa":
        ext = f"{s}*n" if s > 1 else "n"
        idx = f"{s}*(X)" if s > 1 else "X"
        return _probe_1d(p, [f"array a global {dt} {ext}", f"array b global {dt} {ext}", f"array c global {dt} {ext}"],
                         [f"load a[{idx}]", f"load b[{idx}]", f"flop {dt} mul 2", f"flop {dt} add 1", f"store c[{idx}]"])
    if k == "filled":
        X = f"{W}*g+l"
        return "\n".join([f"kernel {p.name}", "param n", f"array a global f32 {p.k},{s}*n", "array o global f32 n",
                          f"dim g g0 0 ceil(n/{W})", f"dim l l0 0 {W}", f"dim k seq 0 {p.k}", f"dim j seq 0 {s}",
                          "stmt acc g,k,j,l", f"guard {X} < n", f"load a[k,{s}*({X})+j]", "flop f32 add 1", "end",
                          "stmt st g,l", f"guard {X} < n", f"store o[{X}]", "end"]) + "\n"
    if k in ("arith", "empty"):
        X, Y = f"{p.gx}*gx+lx", f"{p.gy}*gy+ly"
        L = [f"kernel {p.name}", "param n"] + ([f"array o global {dt} n,n"] if k == "arith" else []) + [
            f"dim gx g0 0 ceil(n/{p.gx})", f"dim gy g1 0 ceil(n/{p.gy})", f"dim lx l0 0 {p.gx}",
            f"dim ly l1 0 {p.gy}"]
        if k == "empty":
            return "\n".join(L + ["stmt s gx,gy,lx,ly", "end"]) + "\n"
        t = ARITH_TYPES[s]
        ops = {"add": [f"flop {dt} add 8"], "mul": [f"flop {dt} mul 8"], "div": [f"flop {dt} div 8"],
               "pow": ["flop f32 pow 8", "flop f32 add 8"], "spec": ["flop f32 spec 8", "flop f32 add 8"]}[t]
        return "\n".join(L + [f"dim k seq 0 {p.k}", "stmt a gx,gy,ly,lx,k", f"guard {Y} < n", f"guard {X} < n"]
                         + ops + ["end", "stmt st gx,gy,ly,lx", f"guard {Y} < n", f"guard {X} < n",
                                  f"store o[{Y},{X}]", "end"]) + "\n"
    if k == "nbody":
        X = f"{W}*g+l"
        return "\n".join([f"kernel {p.name}", "param n"] + [f"array {a} global f32 n" for a in
                                                             ("x", "y", "z", "m", "ax", "ay", "az")] + [
            f"dim g g0 0 ceil(n/{W})", f"dim l l0 0 {W}", "dim j seq 0 n",
            "stmt own g,l", f"guard {X} < n", f"load x[{X}]", f"load y[{X}]", f"load z[{X}]", "end",
            "stmt pair g,l,j", f"guard {X} < n", "load x[j]", "load y[j]", "load z[j]", "load m[j]",
            "flop f32 add 9", "flop f32 mul 9", "flop f32 spec 1", "end",
            "stmt st g,l", f"guard {X} < n", f"store ax[{X}]", f"store ay[{X}]", f"store az[{X}]", "end"]) + "\n"
    if k == "conv5":
        X, Y = f"{p.gx}*gx+lx", f"{p.gy}*gy+ly"
        return "\n".join([f"kernel {p.name}", "param n", "array in global f32 n,n", "array w global f32 5,5",
                          "array out global f32 n,n", f"dim gx g0 0 ceil((n-4)/{p.gx})",
                          f"dim gy g1 0 ceil((n-4)/{p.gy})", f"dim lx l0 0 {p.gx}", f"dim ly l1 0 {p.gy}",
                          "dim fy seq 0 5", "dim fx seq 0 5",
                          "stmt mac gx,gy,ly,lx,fy,fx", f"guard {Y} < n-4", f"guard {X} < n-4",
                          f"load in[{Y}+fy,{X}+fx]", "load w[fy,fx]", "flop f32 mul 1", "flop f32 add 1", "end",
                          "stmt st gx,gy,ly,lx", f"guard {Y} < n-4", f"guard {X} < n-4", f"store out[{Y},{X}]",
                          "end"]) + "\n"
    if k == "transpose_w":
        T = p.gx
        X, Y = f"{T}*gx+lx", f"{T}*gy+ly"
        return "\n".join([f"kernel {p.name}", "param n", "array in global f32 n,n", "array out global f32 n,n",
                          f"dim gx g0 0 ceil(n/{T})", f"dim gy g1 0 ceil(n/{T})", f"dim ly l1 0 {T}",
                          f"dim lx l0 0 {T}", "stmt cp gx,gy,ly,lx", f"guard {Y} < n", f"guard {X} < n",
                          f"load in[{X},{Y}]", f"store out[{Y},{X}]", "end"]) + "\n"
    return variant_ir(probe_variant(p))


def probe_variant(p: Probe) -> Variant:
    """The template variant behind a template-shaped probe (tile p.gx, one item per
    element for the 2-D kinds)."""
    T = p.gx
    if p.kind == "transpose_p":
        return Variant("transpose", T, T, 1, True, T * T)
    if p.kind == "transpose_r":
        return Variant("transpose", T, T, 1, False, T * T)
    if p.kind == "matmul":
        return Variant("matmul", T, T, 1, True, T * T)
    if p.kind == "matmul_naive":
        return Variant("matmul", T, T, 1, False, T * T)
    if p.kind == "stencil":
        return Variant("stencil", T, T, 1, False, T * T)
    if p.kind == "matvec":
        return Variant("matvec", 8, 8, 1, False, 256)
    if p.kind in ("reduction", "axpy", "vecadd"):
        return Variant(p.kind, p.variant, p.variant, 1, False, p.gx)   # tile variant x variant elements per group
    raise ValueError(p.kind)


# --------------------------------------------------------------------------- small workload

POW2_SMALL = (64, 128, 256)


def tiny_points(template: str, n_points: int = 32, sizes: Sequence[int] = POW2_SMALL,
                seed: int = 1) -> np.ndarray:
    """Points of the small workload: powers of two from ``sizes``, taken from the
    product grid for multi-parameter templates and cycled/padded otherwise."""
    P = len(TEMPLATE_PARAMS[template])
    grid = np.array(np.meshgrid(*([list(sizes)] * P), indexing="ij")).reshape(P, -1).T
    rng = np.random.default_rng(seed)
    if len(grid) >= n_points:
        idx = rng.choice(len(grid), n_points, replace=False)
        return grid[np.sort(idx)].astype(np.int64)
    reps = int(math.ceil(n_points / len(grid)))
    return np.tile(grid, (reps, 1))[:n_points].astype(np.int64)


def tiny_variants() -> List[Variant]:
    """The eight templates of the small workload; the strided copy takes s = 4."""
    return [canonical(t, 4 if t == "copy" else 1) for t in TEMPLATES]


# --------------------------------------------------------------------------- fit inputs

def fit_features(rows: int, k: int = 32, seed: int = 5) -> np.ndarray:
    """Feature rows shaped like the paper's measurement-kernel families (Sec. 4.1):
    each row belongs to one family whose nonzero columns and size scaling
    (n, n^2 or n^3 with log-uniform n) mimic that family's counts.  int64 [rows][k].
    Column magnitudes span roughly 1e2..1e13."""
    rng = np.random.default_rng(seed)
    F = np.zeros((rows, k), dtype=np.int64)
    fam = rng.integers(0, 8, size=rows)
    n = np.exp(rng.uniform(math.log(2**8), math.log(2**13), size=rows))
    n1 = np.floor(n * 64).astype(np.int64)            # 1-D sizes up to ~5e5
    n2 = np.floor(n).astype(np.int64)                 # 2-D sizes
    wg = rng.choice([128, 256, 512], size=rows)
    F[:, 0] = 1
    def put(mask, col, val):
        F[mask, col] = np.asarray(val)[mask]
    for f in range(8):
        msk = fam == f
        if f == 0:   # stride-1 streaming (copy / add arrays)
            nl = rng.integers(0, 5, size=rows)
            put(msk, 17, n1 * np.maximum(nl, 1)); put(msk, 24, n1); put(msk, 3, n1 * np.maximum(nl - 1, 0))
            put(msk, 1, (n1 + wg - 1) // wg)
        elif f == 1:  # strided vector scale-add (stride 2 or 3)
            put(msk, 19, 2 * n1); put(msk, 24, n1); put(msk, 4, 2 * n1); put(msk, 3, n1)
            put(msk, 1, (n1 + wg - 1) // wg)
        elif f == 2:  # transpose, no prefetch
            put(msk, 17, n2 * n2); put(msk, 26, n2 * n2); put(msk, 1, (n2 * n2 + 255) // 256)
        elif f == 3:  # transpose, prefetch
            put(msk, 17, n2 * n2); put(msk, 24, n2 * n2); put(msk, 13, n2 * n2); put(msk, 15, n2 * n2)
            put(msk, 2, (n2 * n2 + 255) // 256); put(msk, 1, (n2 * n2 + 255) // 256)
        elif f == 4:  # tiled matmul
            nn = np.minimum(n2, 2048)
            put(msk, 3, nn ** 3); put(msk, 4, nn ** 3); put(msk, 13, 2 * nn ** 3)
            put(msk, 17, 2 * nn ** 3 // 16); put(msk, 15, 2 * nn ** 3 // 16); put(msk, 24, nn * nn)
            put(msk, 2, 2 * (nn // 16) ** 3); put(msk, 1, (nn // 16) ** 2)
        elif f == 5:  # naive matmul
            nn = np.minimum(n2, 1024)
            put(msk, 3, nn ** 3); put(msk, 4, nn ** 3); put(msk, 16, nn ** 3); put(msk, 17, nn ** 3)
            put(msk, 24, nn * nn); put(msk, 1, (nn * nn + 255) // 256)
        elif f == 6:  # arithmetic kernels (one op kind each)
            kk = rng.choice([256, 512, 728], size=rows)
            col = rng.choice([3, 4, 5, 6, 7], size=rows)
            nn = np.minimum(n2, 1024)
            for c in (3, 4, 5, 6, 7):
                put(msk & (col == c), c, nn * nn * kk * rng.integers(6, 11, size=rows))
            put(msk, 24, nn * nn); put(msk, 1, (nn * nn + 255) // 256)
        else:         # empty kernel
            put(msk, 1, (n2 * n2 + 255) // 256)
    # Sparse remaining columns get an independent small family so every column is informative.
    extra = rng.integers(0, k, size=rows)
    for c in range(k):
        msk = (extra == c) & (F[:, c] == 0)
        F[msk, c] = n1[msk] * rng.integers(1, 4, size=rows)[msk]
    return F


def synth_timings(F: np.ndarray, w_true: np.ndarray, seed: int = 6, sigma: float = 0.05) -> np.ndarray:
    """Stand-in for timing measurement kernels on hardware: t = (F w_true) * exp(e),
    e ~ N(0, sigma^2), one column per device model.  fp64 [rows][models]."""
    rng = np.random.default_rng(seed)
    clean = F.astype(np.float64) @ np.asarray(w_true, dtype=np.float64).T
    e = rng.normal(0.0, sigma, size=clean.shape)
    return clean * np.exp(e)
