// Compiled count table: the device-resident form of one kernel's piecewise
// quasi-polynomial properties (Sec. 3.2: a key -> piecewise quasi-polynomial
// mapping, here with keys already folded into feature columns).
//
// All fields are 32-bit words.  A table is evaluated at a parameter point n by
//   1. values v[0..P)   = n (the parameters),
//      values v[P..P+A) = atoms floor((a . n + b) / c), c >= 2;
//   2. bits: condition j holds iff const_j + sum_t coef_jt * v[idx_jt] >= 0;
//   3. piece = lut[bits];
//   4. the piece's products (monomials of degree >= 2) are formed once, then each
//      column value = sum of integer coef * (value or product) over its entries (exact int64),
//      divided exactly by the table's denominator D (usually 1);
//   5. post-ops: column = min(held value A, held value B)   (min(loads, stores)).
// Columns that no segment names are zero.  Hidden columns (index >= k) only feed
// post-ops.
#pragma once
#include <stdint.h>

namespace pmt {

constexpr uint32_t MAGIC = 0x31544d50u;  // "PMT1"
constexpr int MAX_VALUES = 32;
constexpr int MAX_CONDS = 10;
constexpr int MAX_DEGREE = 4;
constexpr int MAX_HOLD = 4;
constexpr int MAX_COLS = 40;           // visible + hidden
constexpr int MAX_TABLE_WORDS = 4096;  // 16 KB

enum Header {
  H_MAGIC = 0, H_WORDS, H_NPARAMS, H_NATOMS, H_NCONDS, H_NPIECES, H_K, H_NHIDDEN, H_NPOST,
  H_OFF_ATOMS, H_OFF_CONDS, H_OFF_LUT, H_OFF_PIECES, H_OFF_PRODS, H_OFF_ENTRIES, H_OFF_POST,
  H_BOX_LO = 16, H_BOX_HI = 20, H_NENTRIES = 24, H_DEGREE = 25, H_NPRODS = 26, H_MAXPROD = 27,
  H_DEN = 28, H_DEN_SHIFT = 29, H_DEN_INV = 32, HEADER_WORDS = 36
};

// Denominator.  Counts over coupled domains (j < i, bands, ...) are sums of powers with
// rational coefficients, so entries hold D * count and each column value is divided
// exactly by D = 2^t d (d odd): shifted right by t, then multiplied by d^-1 mod 2^128
// (H_DEN_INV, four words; its low 64 bits are d^-1 mod 2^64).  D = 1 for most kernels.
// A column's D * count stays below 2^62.

// Per-lane evaluation slots (int64): values 0..V-1 (parameters, then atoms), the
// piece's products V..V+J-1, four slots that hold post-op inputs, and the constant 1.
constexpr int MAX_SLOTS = 24;
constexpr int HOLD_SLOT = 19;          // 19..22
constexpr int MAX_PRODS = HOLD_SLOT;   // V + J <= 19
constexpr uint32_t CONST_SLOT = 23;    // always 1

// Atom: 8 words  a0 a1 a2 a3 b c magic packed
//   packed: bits 0..7 shift1, 8..15 shift2, bit 16: numerator may be negative
constexpr int ATOM_WORDS = 8;
// Condition: [n_terms, const_lo, const_hi, (idx, coef) * n_terms]
// LUT: 2^n_conds bytes (piece ids), packed 4 per word.
// Piece: 4 words [prod_begin, n_prods, entry_begin, n_entries]
// Product: 1 word [a | b << 8]: slot V+j = slot a * slot b, with a, b < V+j (the
//   monomials of degree >= 2 of the piece and the prefixes they are built from).
// Entry: 4 words [coef_lo, coef_hi, packed, 0]; entries are sorted by column and
//   column value = sum of coef * slot over its entries (slot 23 = the constant 1).
//   packed: col (8) | slot << 8 | (hold+1) << 16 (4 bits) | last-of-column << 20
constexpr int ENTRY_WORDS = 4;
constexpr uint32_t ENTRY_LAST = 1u << 20;
// Post-op: 1 word [out_col | holdA << 8 | holdB << 16]

}  // namespace pmt
