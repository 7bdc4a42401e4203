"""Test-only reader of compiled count tables (the layout of csrc/pm_table.h).

It lets the CPU tests check the compiler's output against the oracle without a
GPU.  It is never imported by the library, so it cannot act as a CPU fallback.
"""
import numpy as np

H_MAGIC, H_WORDS, H_NPARAMS, H_NATOMS, H_NCONDS, H_NPIECES, H_K, H_NHIDDEN, H_NPOST = range(9)
H_OFF_ATOMS, H_OFF_CONDS, H_OFF_LUT, H_OFF_PIECES, H_OFF_PRODS, H_OFF_ENTRIES, H_OFF_POST = range(9, 16)
H_BOX_LO, H_BOX_HI = 16, 20
H_DEN = 28


def _s32(x):
    x = int(x) & 0xFFFFFFFF
    return x - (1 << 32) if x >= (1 << 31) else x


def _s64(lo, hi):
    x = (int(lo) & 0xFFFFFFFF) | ((int(hi) & 0xFFFFFFFF) << 32)
    return x - (1 << 64) if x >= (1 << 63) else x


def magic_div(x, m, sh2):
    """The kernels' unsigned division by an invariant (32-bit arithmetic)."""
    t = (m * x) >> 32
    return ((t + ((x - t) >> 1)) & 0xFFFFFFFF) >> sh2


class Table:
    def __init__(self, words):
        self.w = [int(x) for x in np.asarray(words, dtype=np.uint32)]
        w = self.w
        assert w[H_MAGIC] == 0x31544D50
        self.P, self.A, self.C = w[H_NPARAMS], w[H_NATOMS], w[H_NCONDS]
        self.k, self.hidden = w[H_K], w[H_NHIDDEN]
        self.box_lo = [_s32(w[H_BOX_LO + i]) for i in range(self.P)]
        self.box_hi = [_s32(w[H_BOX_HI + i]) for i in range(self.P)]
        self.den = w[H_DEN]   # entries hold den * count

    def atoms(self):
        w, o = self.w, self.w[H_OFF_ATOMS]
        out = []
        for a in range(self.A):
            q = w[o + 8 * a: o + 8 * a + 8]
            out.append(dict(a=[_s32(x) for x in q[:4]], b=_s32(q[4]), c=_s32(q[5]), m=q[6],
                            sh2=(q[7] >> 8) & 0xFF, neg=(q[7] >> 16) & 1))
        return out

    def slots_and_piece(self, n):
        """Evaluation slots (parameters, atoms, products, constant) and the piece at n."""
        w = self.w
        vals = list(n[:self.P])
        for at in self.atoms():
            vals.append((at["b"] + sum(at["a"][i] * n[i] for i in range(self.P))) // at["c"])
        bits, o = 0, w[H_OFF_CONDS]
        for c in range(self.C):
            nt = w[o]
            s = _s64(w[o + 1], w[o + 2])
            for t in range(nt):
                s += _s32(w[o + 4 + 2 * t]) * vals[w[o + 3 + 2 * t]]
            bits |= int(s >= 0) << c
            o += 3 + 2 * nt
        piece = (w[w[H_OFF_LUT] + (bits >> 2)] >> (8 * (bits & 3))) & 0xFF
        p0, n_prod = w[w[H_OFF_PIECES] + 4 * piece], w[w[H_OFF_PIECES] + 4 * piece + 1]
        slots = list(vals) + [0] * (24 - len(vals))
        slots[23] = 1
        V = len(vals)
        for j in range(n_prod):
            x = w[w[H_OFF_PRODS] + p0 + j]
            slots[V + j] = slots[x & 0xFF] * slots[(x >> 8) & 0xFF]
        return slots, piece

    def evaluate(self, n, check_magic=True, check_exact=True):
        """Exact feature columns at point n (Python integers).  check_exact=False skips
        the exact-division and 62-bit checks (an image with altered coefficients)."""
        w = self.w
        P = self.P
        for i in range(P):
            assert self.box_lo[i] <= n[i] <= self.box_hi[i]
        vals = list(n[:P])
        for at in self.atoms():
            num = at["b"] + sum(at["a"][i] * n[i] for i in range(P))
            f = num // at["c"]
            if check_magic:
                if num >= 0:
                    g = magic_div(num, at["m"], at["sh2"])
                else:
                    assert at["neg"]
                    g = -magic_div(-num + at["c"] - 1, at["m"], at["sh2"])
                assert g == f, (num, at)
            vals.append(f)
        bits, o = 0, w[H_OFF_CONDS]
        for c in range(self.C):
            nt = w[o]
            s = _s64(w[o + 1], w[o + 2])
            for t in range(nt):
                s += _s32(w[o + 4 + 2 * t]) * vals[w[o + 3 + 2 * t]]
            bits |= int(s >= 0) << c
            o += 3 + 2 * nt
        lut = w[H_OFF_LUT]
        piece = (w[lut + (bits >> 2)] >> (8 * (bits & 3))) & 0xFF
        assert piece < w[H_NPIECES]
        pb = w[H_OFF_PIECES] + 4 * piece
        p0, n_prod, e0, n_ent = w[pb:pb + 4]
        slots = list(vals) + [None] * (24 - len(vals))
        slots[23] = 1
        V = len(vals)
        for j in range(n_prod):
            x = w[w[H_OFF_PRODS] + p0 + j]
            a, b = x & 0xFF, (x >> 8) & 0xFF
            assert a < V + j and b < V + j
            slots[V + j] = slots[a] * slots[b]
        cols = [0] * (self.k + self.hidden)
        hold = [0, 0, 0, 0]
        acc = 0
        for e in range(n_ent):
            eo = w[H_OFF_ENTRIES] + 4 * (e0 + e)
            coef = _s64(w[eo], w[eo + 1])
            pk = w[eo + 2]
            sl = (pk >> 8) & 0xFF
            assert sl < V + n_prod or sl == 23
            acc += coef * slots[sl]
            if pk & (1 << 20):
                col, h = pk & 0xFF, (pk >> 16) & 0xF
                assert not check_exact or (acc % self.den == 0 and abs(acc) < (1 << 62))
                acc //= self.den
                cols[col] = acc
                if h:
                    hold[h - 1] = acc
                acc = 0
        assert acc == 0
        po = w[H_OFF_POST]
        for q in range(w[H_NPOST]):
            x = w[po + q]
            cols[x & 0xFF] = min(hold[(x >> 8) & 0xFF], hold[(x >> 16) & 0xFF])
        return cols[:self.k]


def _wide(words):
    """Four 32-bit words -> signed 128-bit integer."""
    x = sum((int(words[i]) & 0xFFFFFFFF) << (32 * i) for i in range(4))
    return x - (1 << 128) if x >= (1 << 127) else x


def program_dot(prog, table, n):
    """The fused ranking kernel's value of a K2 program at n: sum over the piece's
    weighted slots, then the runtime post-ops (signed 128-bit result)."""
    slots, piece = table.slots_and_piece(n)
    I = (table.w[H_OFF_ENTRIES] + 3) & ~3
    dot_w, n_dot, dot_s, flags, hold_off, n_hold, post_off, n_post = prog[I + 8 * piece: I + 8 * piece + 8]
    S = 0
    for d in range(n_dot):
        S += _wide(prog[dot_w + 4 * d: dot_w + 4 * d + 4]) * slots[prog[dot_s + d]]
    if n_post:
        hold = [0, 0, 0, 0]
        for h in range(n_hold):
            e = prog[hold_off + 4 * h: hold_off + 4 * h + 4]
            hold[(e[0] >> 8) & 3] += _s64(e[2], e[3]) * slots[e[0] & 0xFF]
        for q in range(n_post):
            e = prog[post_off + 8 * q: post_off + 8 * q + 8]
            S += _wide(e[:4]) * min(hold[e[4] & 3], hold[(e[4] >> 8) & 3])
    assert S % table.den == 0
    return S // table.den
