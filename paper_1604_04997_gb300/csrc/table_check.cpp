// Structural check of a compiled count table supplied from outside the compiler
// (pm_table_load: a saved image loaded back).  Everything the evaluators index is
// bounded here, so a corrupted or foreign image is refused with a status instead of
// reaching a kernel: header limits, section offsets inside the image, condition terms,
// the piece LUT, product operands, entry slots and columns, post-op holds, the atoms'
// divisors and magic numbers and their numerator range over the declared box, and the
// denominator's inverse.  The counts' values themselves are those of the compiled
// table the image came from.
#include <cstdint>
#include <string>

#include "pm_table.h"

namespace {

uint32_t magic_of(int64_t c, int &sh2) {   // as the compiler derives it (division by an invariant)
  int l = 0;
  while ((int64_t(1) << l) < c) l++;
  unsigned __int128 m = ((unsigned __int128)1 << 32) * (((unsigned __int128)1 << l) - (unsigned __int128)c) /
                        (unsigned __int128)c + 1;
  sh2 = l - 1;
  return (uint32_t)m;
}

bool fail(std::string &why, const char *m) {
  why = m;
  return false;
}

}  // namespace

bool pm_table_valid(const uint32_t *w, size_t n, std::string &why) {
  using namespace pmt;
  if (!w || n < (size_t)HEADER_WORDS || n > (size_t)MAX_TABLE_WORDS || n % 4) return fail(why, "image size");
  if (w[H_MAGIC] != MAGIC || w[H_WORDS] != n) return fail(why, "magic or word count");
  const uint32_t P = w[H_NPARAMS], A = w[H_NATOMS], NC = w[H_NCONDS], NP = w[H_NPIECES];
  const uint32_t K = w[H_K], HID = w[H_NHIDDEN], NPOST = w[H_NPOST];
  if (P < 1 || P > 4 || P + A > (uint32_t)MAX_VALUES || NC > (uint32_t)MAX_CONDS || NP < 1 || NP > 256)
    return fail(why, "header counts");
  if ((K != 12 && K != 32) || K + HID > (uint32_t)MAX_COLS || NPOST > 8) return fail(why, "columns");
  // sections in order, each inside the image (64-bit sums: no wrap-around)
  const uint64_t oa = w[H_OFF_ATOMS], oc = w[H_OFF_CONDS], ol = w[H_OFF_LUT], op = w[H_OFF_PIECES];
  const uint64_t opr = w[H_OFF_PRODS], oe = w[H_OFF_ENTRIES], opo = w[H_OFF_POST];
  const uint64_t NE = w[H_NENTRIES], NPR = w[H_NPRODS];
  if (oa < (uint64_t)HEADER_WORDS || oa + 8 * A > oc || oc > ol || ol + ((1u << NC) + 3) / 4 > op || op % 4 ||
      op + 4 * NP > opr || opr + NPR > oe || oe % 4 || oe + 4 * NE > opo || opo + NPOST > n)
    return fail(why, "section offsets");
  int64_t lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
  for (uint32_t i = 0; i < P; i++) {
    lo[i] = (int32_t)w[H_BOX_LO + i];
    hi[i] = (int32_t)w[H_BOX_HI + i];
    if (lo[i] > hi[i]) return fail(why, "parameter box");
  }
  // atoms: floor((a . n + b) / c) with the compiler's divisor magic and an int32 numerator
  for (uint32_t a = 0; a < A; a++) {
    const uint32_t *t = w + oa + 8 * a;
    const int64_t c = (int32_t)t[5];
    if (c < 2) return fail(why, "atom divisor");
    int sh2;
    if (t[6] != magic_of(c, sh2) || ((t[7] >> 8) & 0xFF) != (uint32_t)sh2) return fail(why, "atom magic");
    int64_t nl = (int32_t)t[4], nh = (int32_t)t[4];
    for (uint32_t i = 0; i < P; i++) {
      const int64_t x = (int64_t)(int32_t)t[i] * lo[i], y = (int64_t)(int32_t)t[i] * hi[i];
      nl += x < y ? x : y;
      nh += x < y ? y : x;
    }
    if (nl < INT32_MIN || nh > INT32_MAX || (nl < 0 && !((t[7] >> 16) & 1))) return fail(why, "atom range");
  }
  // conditions: terms over the values
  uint64_t o = oc;
  for (uint32_t q = 0; q < NC; q++) {
    if (o + 3 > ol) return fail(why, "condition bounds");
    const uint32_t nt = w[o];
    if (nt > P + A || o + 3 + 2 * nt > ol) return fail(why, "condition terms");
    for (uint32_t t = 0; t < nt; t++)
      if (w[o + 3 + 2 * t] >= P + A) return fail(why, "condition value index");
    o += 3 + 2 * nt;
  }
  // LUT: every reachable bit pattern names a piece
  for (uint32_t b = 0; b < (1u << NC); b++)
    if (((w[ol + (b >> 2)] >> (8 * (b & 3))) & 0xFF) >= NP) return fail(why, "piece table");
  // pieces: products, entries
  const uint32_t V = P + A;
  for (uint32_t p = 0; p < NP; p++) {
    const uint32_t *pc = w + op + 4 * p;
    const uint32_t pb = pc[0], pn = pc[1], eb = pc[2], en = pc[3];
    if ((uint64_t)pb + pn > NPR || pn > (uint32_t)MAX_PRODS || V + pn > (uint32_t)MAX_PRODS || (uint64_t)eb + en > NE)
      return fail(why, "piece ranges");
    for (uint32_t j = 0; j < pn; j++) {
      const uint32_t x = w[opr + pb + j];
      if ((x & 0xFF) >= V + j || ((x >> 8) & 0xFF) >= V + j || (x >> 16)) return fail(why, "product operands");
    }
    for (uint32_t e = 0; e < en; e++) {
      const uint32_t pk = w[oe + 4 * (eb + e) + 2];
      const uint32_t col = pk & 0xFF, slot = (pk >> 8) & 0xFF, hold = (pk >> 16) & 0xF;
      if (col >= K + HID || hold > (uint32_t)MAX_HOLD) return fail(why, "entry column or hold");
      if (slot >= V + pn && slot != CONST_SLOT) return fail(why, "entry slot");
      if (pk >> 21) return fail(why, "entry flags");
    }
    if (en && !(w[oe + 4 * (eb + en - 1) + 2] & ENTRY_LAST)) return fail(why, "unterminated column");
  }
  for (uint32_t q = 0; q < NPOST; q++) {
    const uint32_t x = w[opo + q];
    if ((x & 0xFF) >= K + HID || ((x >> 8) & 0xFF) >= (uint32_t)MAX_HOLD || ((x >> 16) & 0xFF) >= (uint32_t)MAX_HOLD)
      return fail(why, "post-op");
  }
  // denominator D = 2^t d with its inverse d^-1
  const uint64_t D = w[H_DEN];
  const uint32_t t = w[H_DEN_SHIFT];
  if (D < 1 || D > 4096 || t > 12 || (D >> t) << t != D || ((D >> t) & 1) == 0) return fail(why, "denominator");
  unsigned __int128 inv = 0;   // d^-1 mod 2^128 (the ranking kernel divides its 128-bit sums)
  for (int i = 3; i >= 0; i--) inv = (inv << 32) | w[H_DEN_INV + i];
  if ((unsigned __int128)(D >> t) * inv != 1) return fail(why, "denominator inverse");
  return true;
}
