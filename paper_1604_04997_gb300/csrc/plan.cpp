// Schedules for the persistent fused launch (pm_eval_predict_topk): ranking groups
// with a shared per-point basis, work units in longest-processing-time order,
// launch-shape tuning and CUDA-graph replay.
//
// Sec. 2 observes that the properties p_i(n) are "cheaply reevaluated for changed
// values of n".  Across the variants of one kernel template the same sub-expressions
// recur: floor(n / 16) appears in every table with a 16-wide tile, n * m in every
// table with an n x m domain.  A ranking group gathers the variants of one template
// whose tables together need at most BASIS_MAX distinct values (parameters, atoms
// floor((a.n + b)/c), monomials, the constant) and GCOND_MAX distinct piece
// conditions.  The kernel evaluates that basis once per point, and each variant's
// prediction becomes one exact dot product of its piece's weights with basis values.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "kernels.h"
#include "pm.h"
#include "pm_internal.h"
#include "pm_table.h"

#define CU(x)                                                                                          \
  do {                                                                                                 \
    cudaError_t e__ = (x);                                                                             \
    if (e__ != cudaSuccess) return pm_set_error(PM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e__)); \
  } while (0)

using pmd::RankLayout;

// Value ranges of a piece's evaluation slots over the table's parameter box (interval
// arithmetic, wide integers): parameters, atoms floor((a.n + b)/c), the constant 1 and
// the piece's products.
using i128 = __int128;
struct Range { i128 lo, hi; };
// Slot values and coefficients of a valid table stay below 2^63, so products stay
// below 2^126; anything wider is clamped to +-2^120 and never used in a proof.
static constexpr i128 WIDE_LIM = (i128)1 << 120;
static i128 clamp_wide(i128 v) { return v > WIDE_LIM ? WIDE_LIM : (v < -WIDE_LIM ? -WIDE_LIM : v); }
static i128 floor_div_wide(i128 a, i128 c) { return a >= 0 ? a / c : -((-a + c - 1) / c); }
static Range mul_range(Range x, Range y) {
  const i128 q[4] = {clamp_wide(x.lo * y.lo), clamp_wide(x.lo * y.hi), clamp_wide(x.hi * y.lo), clamp_wide(x.hi * y.hi)};
  return Range{*std::min_element(q, q + 4), *std::max_element(q, q + 4)};
}
static Range atom_range(const uint32_t *at, int P, const i128 *lo, const i128 *hi) {
  i128 mn = (int32_t)at[4], mx = (int32_t)at[4];
  for (int p = 0; p < P; p++) {
    const i128 k = (int32_t)at[p];
    mn += k >= 0 ? k * lo[p] : k * hi[p];
    mx += k >= 0 ? k * hi[p] : k * lo[p];
  }
  const i128 c = at[5] ? (i128)at[5] : 1;
  return Range{floor_div_wide(mn, c), floor_div_wide(mx, c)};
}
static std::vector<Range> slot_ranges(const std::vector<uint32_t> &T, const uint32_t *pc) {
  std::vector<Range> r(pmt::MAX_SLOTS, Range{0, 0});
  const int P = (int)T[pmt::H_NPARAMS], A = (int)T[pmt::H_NATOMS];
  i128 lo[4], hi[4];
  for (int p = 0; p < 4; p++) {
    lo[p] = (int32_t)T[pmt::H_BOX_LO + p];
    hi[p] = (int32_t)T[pmt::H_BOX_HI + p];
    if (p < P) r[p] = Range{lo[p], hi[p]};
  }
  const uint32_t *at = T.data() + T[pmt::H_OFF_ATOMS];
  for (int a = 0; a < A && P + a < pmt::MAX_SLOTS; a++, at += pmt::ATOM_WORDS) r[P + a] = atom_range(at, P, lo, hi);
  r[pmt::CONST_SLOT] = Range{1, 1};
  const uint32_t *pr = T.data() + T[pmt::H_OFF_PRODS] + pc[0];
  for (uint32_t j = 0; j < pc[1] && P + A + (int)j < pmt::MAX_SLOTS; j++)
    r[P + A + j] = mul_range(r[std::min<uint32_t>(pr[j] & 0xFF, pmt::MAX_SLOTS - 1)],
                             r[std::min<uint32_t>((pr[j] >> 8) & 0xFF, pmt::MAX_SLOTS - 1)]);
  return r;
}

// ------------------------------------------------------------------ ranking groups

namespace {

constexpr int BASIS_MAX = 128;        // basis values per group (one byte per term index)
constexpr int GCOND_MAX = 64;         // distinct conditions per group (two 32-bit masks per point)
constexpr int LEVEL_MAX = 8;          // product depth of the basis
constexpr int GROUP_MAX_WORDS = 12288; // a group's image, staged in shared memory (48 KB)
constexpr int PROG_MAX_WORDS = 6144;  // one table's program (24 KB)
constexpr i128 VALUE_LIM = (i128)1 << 62;

enum { BK_PARAM = 0, BK_CONST = 1, BK_ATOM = 2, BK_PROD = 3 };

struct BEntry {
  int kind = BK_PARAM;
  int i = 0, j = 0;      // PARAM: parameter index; PROD: factor entries
  uint32_t atom[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  Range range{0, 0};
  int level = 0;
};

using Contribs = std::vector<std::pair<uint32_t, uint64_t>>;   // (column, coefficient)

// One leaf of a program: an exact dot product of 128-bit weights with basis values.
struct LeafForm {
  bool const_first = false;
  Contribs const_c;
  std::vector<std::pair<int, Contribs>> t64, t32, twide;   // (basis entry, contributions)
};

// One piece of a table: its leaves, one per sign pattern of the post-op differences
// A - B (group conditions, bit q of the leaf index) that the box leaves undecided.
struct PieceForm {
  std::vector<int> sub_conds;
  std::vector<LeafForm> leaves;
};

struct ProgForm {
  int ncond = 0;
  int gcond[pmt::MAX_CONDS] = {0};
  std::vector<uint8_t> lut;
  bool den = false;
  uint32_t den_shift = 0, den_inv[4] = {0, 0, 0, 0};
  std::vector<PieceForm> pieces;
  double work = 0;       // algorithmic integer operations per evaluation (average over pieces)
};

struct Group {
  int P = 0;
  i128 lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
  std::vector<BEntry> ents;
  std::map<std::vector<uint32_t>, int> atom_idx;
  std::map<std::pair<int, int>, int> prod_idx;
  std::vector<std::vector<int64_t>> conds;           // [const, (entry, coef)*]
  std::map<std::vector<int64_t>, int> cond_idx;
  std::vector<ProgForm> progs;
  std::map<int, int> prog_of_table;                   // table id -> program
  std::vector<int> var_prog;                          // per variant of the group
  int var_begin = 0;                                  // template-relative index of the first variant
};

struct BuildError { pm_status code; std::string msg; };

int entry_param(Group &g, int p) { return p; }   // parameters are entries 0..P-1

int entry_const(Group &g) {
  for (size_t e = 0; e < g.ents.size(); e++)
    if (g.ents[e].kind == BK_CONST) return (int)e;
  BEntry b;
  b.kind = BK_CONST;
  b.range = Range{1, 1};
  g.ents.push_back(b);
  return (int)g.ents.size() - 1;
}

int entry_atom(Group &g, const uint32_t *at) {
  std::vector<uint32_t> key(at, at + 6);
  auto it = g.atom_idx.find(key);
  if (it != g.atom_idx.end()) return it->second;
  BEntry b;
  b.kind = BK_ATOM;
  std::memcpy(b.atom, at, sizeof b.atom);
  b.range = atom_range(at, g.P, g.lo, g.hi);
  g.ents.push_back(b);
  g.atom_idx[key] = (int)g.ents.size() - 1;
  return (int)g.ents.size() - 1;
}

int entry_prod(Group &g, int a, int b) {
  const std::pair<int, int> key(std::min(a, b), std::max(a, b));
  auto it = g.prod_idx.find(key);
  if (it != g.prod_idx.end()) return it->second;
  BEntry e;
  e.kind = BK_PROD;
  e.i = key.first;
  e.j = key.second;
  e.range = mul_range(g.ents[a].range, g.ents[b].range);
  e.level = 1 + std::max(g.ents[a].level, g.ents[b].level);
  if (e.range.lo <= -VALUE_LIM || e.range.hi >= VALUE_LIM)
    throw BuildError{PM_ERR_UNSUPPORTED, "a monomial of the table can reach 2^62 over its box"};
  if (e.level >= LEVEL_MAX) throw BuildError{PM_ERR_UNSUPPORTED, "monomial degree above the ranking kernel's limit"};
  g.ents.push_back(e);
  g.prod_idx[key] = (int)g.ents.size() - 1;
  return (int)g.ents.size() - 1;
}

bool fits_u32(const Range &r) { return r.lo >= 0 && r.hi < ((i128)1 << 32); }

// Add one table to the group (its basis values, conditions and program).  The
// caller keeps a copy of the group to roll back when the limits are exceeded.
void add_table(Group &g, int table_id, const std::vector<uint32_t> &T) {
  if (g.prog_of_table.count(table_id)) return;
  const int P = (int)T[pmt::H_NPARAMS], A = (int)T[pmt::H_NATOMS], NC = (int)T[pmt::H_NCONDS];
  const uint32_t npieces = T[pmt::H_NPIECES], npost = T[pmt::H_NPOST];
  if (P != g.P || P + A > pmt::MAX_VALUES || NC > pmt::MAX_CONDS || npieces < 1 || npieces > 255)
    throw BuildError{PM_ERR_INVALID_ARG, "malformed table"};
  std::vector<int> vmap(pmt::MAX_SLOTS, -1);
  for (int p = 0; p < P; p++) vmap[p] = entry_param(g, p);
  const uint32_t *at = T.data() + T[pmt::H_OFF_ATOMS];
  for (int a = 0; a < A; a++, at += pmt::ATOM_WORDS) {
    const int e = entry_atom(g, at);
    if (g.ents[e].range.lo <= -VALUE_LIM || g.ents[e].range.hi >= VALUE_LIM)
      throw BuildError{PM_ERR_UNSUPPORTED, "an atom of the table can reach 2^62 over its box"};
    vmap[P + a] = e;
  }
  vmap[pmt::CONST_SLOT] = entry_const(g);
  ProgForm pf;
  // conditions: sum of coefficient x value + constant >= 0, deduplicated per group
  pf.ncond = NC;
  const uint32_t *cd = T.data() + T[pmt::H_OFF_CONDS];
  for (int c = 0; c < NC; c++) {
    const int nt = (int)cd[0];
    std::map<int, int64_t> terms;
    for (int t = 0; t < nt; t++) {
      const uint32_t sl = cd[3 + 2 * t];
      if (sl >= (uint32_t)(P + A)) throw BuildError{PM_ERR_INVALID_ARG, "malformed table condition"};
      terms[vmap[sl]] += (int64_t)(int32_t)cd[4 + 2 * t];
    }
    std::vector<int64_t> key{(int64_t)((uint64_t)cd[1] | ((uint64_t)cd[2] << 32))};
    for (auto &kv : terms)
      if (kv.second) { key.push_back(kv.first); key.push_back(kv.second); }
    auto it = g.cond_idx.find(key);
    int q;
    if (it == g.cond_idx.end()) {
      q = (int)g.conds.size();
      g.conds.push_back(key);
      g.cond_idx[key] = q;
    } else {
      q = it->second;
    }
    pf.gcond[c] = q;
    cd += 3 + 2 * nt;
  }
  const uint32_t *lut = T.data() + T[pmt::H_OFF_LUT];
  pf.lut.resize((size_t)1 << NC);
  for (size_t b = 0; b < pf.lut.size(); b++) {
    pf.lut[b] = (uint8_t)((lut[b >> 2] >> (8 * (b & 3))) & 0xFF);
    // the kernel indexes the piece records with it: every bit pattern must name a piece
    if (pf.lut[b] >= npieces) throw BuildError{PM_ERR_INVALID_ARG, "malformed table: a LUT entry names no piece"};
  }
  pf.den = T[pmt::H_DEN] != 1;
  pf.den_shift = T[pmt::H_DEN_SHIFT] & 63;
  for (int q = 0; q < 4; q++) pf.den_inv[q] = T[pmt::H_DEN_INV + q];
  // pieces: the products as basis monomials, then the weighted dot over basis values.
  // A post-op min(hold A, hold B) whose sign of A - B is fixed over the box (interval
  // arithmetic on the piece's slots, like terms combined) is folded into the dot as
  // the smaller column; the others stay runtime post-ops with their held columns.
  double work = 0;
  for (uint32_t p = 0; p < npieces; p++) {
    const uint32_t *pc = T.data() + T[pmt::H_OFF_PIECES] + 4 * p;
    if (P + A + pc[1] > (uint32_t)pmt::MAX_PRODS) throw BuildError{PM_ERR_INVALID_ARG, "malformed table piece"};
    std::vector<int> pmap = vmap;
    const uint32_t *pr = T.data() + T[pmt::H_OFF_PRODS] + pc[0];
    for (uint32_t j = 0; j < pc[1]; j++) {
      const uint32_t a = pr[j] & 0xFF, b = (pr[j] >> 8) & 0xFF;
      if (a >= (uint32_t)(P + A + j) || b >= (uint32_t)(P + A + j) || pmap[a] < 0 || pmap[b] < 0)
        throw BuildError{PM_ERR_INVALID_ARG, "malformed table product"};
      pmap[P + A + j] = entry_prod(g, pmap[a], pmap[b]);
    }
    const uint32_t *en = T.data() + T[pmt::H_OFF_ENTRIES] + pmt::ENTRY_WORDS * pc[2];
    std::map<uint32_t, Contribs> by_slot;
    std::vector<std::vector<std::pair<uint32_t, int64_t>>> held(pmt::MAX_HOLD);
    std::vector<std::pair<uint32_t, int64_t>> col_entries;
    for (uint32_t e = 0; e < pc[3]; e++, en += pmt::ENTRY_WORDS) {
      const uint32_t col = en[2] & 0xFF, slot = (en[2] >> 8) & 0xFF;
      if (slot >= (uint32_t)pmt::MAX_SLOTS || pmap[slot] < 0) throw BuildError{PM_ERR_INVALID_ARG, "malformed table entry"};
      const uint64_t coef = (uint64_t)en[0] | ((uint64_t)en[1] << 32);
      if (col < 32) by_slot[slot].push_back({col, coef});
      col_entries.push_back({slot, (int64_t)coef});
      if (en[2] & pmt::ENTRY_LAST) {
        const uint32_t hold = (en[2] >> 16) & 0xF;
        if (hold) {
          if (hold > (uint32_t)pmt::MAX_HOLD) throw BuildError{PM_ERR_INVALID_ARG, "malformed table hold"};
          held[hold - 1] = col_entries;
        }
        col_entries.clear();
      }
    }
    const std::vector<Range> rg = slot_ranges(T, pc);
    std::vector<std::array<uint32_t, 3>> runtime;   // (output column, hold A, hold B)
    for (uint32_t q = 0; q < npost; q++) {
      const uint32_t w = T[T[pmt::H_OFF_POST] + q];
      const uint32_t out_col = w & 0xFF, ha = (w >> 8) & 3, hb = (w >> 16) & 3;
      std::map<uint32_t, i128> d;   // A - B per slot
      for (auto &x : held[ha]) d[x.first] += (i128)x.second;
      for (auto &x : held[hb]) d[x.first] -= (i128)x.second;
      i128 mn = 0, mx = 0;
      bool sound = true;
      for (auto &kv : d) {
        const Range r = rg[kv.first];
        const i128 lim = (i128)1 << 63;
        if (kv.second >= lim || kv.second <= -lim || r.lo <= -lim || r.hi >= lim) { sound = false; break; }
        const i128 a = kv.second * r.lo, b = kv.second * r.hi;
        mn += std::min(a, b);
        mx += std::max(a, b);
      }
      int pick = -1;
      if (sound && mn >= 0) pick = (int)hb;        // A >= B everywhere: min = B
      else if (sound && mx <= 0) pick = (int)ha;   // A <= B everywhere: min = A
      if (pick >= 0 && out_col < 32) {
        for (auto &x : held[pick]) by_slot[x.first].push_back({out_col, (uint64_t)x.second});
      } else if (out_col < 32) {
        runtime.push_back({out_col, ha, hb});
      }
    }
    // The others: the sign of A - B (a linear form over basis values, exact in 64 bits
    // since both are counts below 2^62) becomes a condition of the group, evaluated
    // once per point; the piece gets one leaf per sign pattern with the min folded.
    if (runtime.size() > 4) throw BuildError{PM_ERR_UNSUPPORTED, "more than four undecided post-ops in a piece"};
    PieceForm f;
    for (auto &q : runtime) {
      std::map<int, int64_t> terms;
      for (auto &x : held[q[1]]) terms[pmap[x.first]] += x.second;
      for (auto &x : held[q[2]]) terms[pmap[x.first]] -= x.second;
      std::vector<int64_t> key{0};
      for (auto &kv : terms)
        if (kv.second) { key.push_back(kv.first); key.push_back(kv.second); }
      auto it = g.cond_idx.find(key);
      if (it == g.cond_idx.end()) {
        it = g.cond_idx.emplace(key, (int)g.conds.size()).first;
        g.conds.push_back(key);
      }
      f.sub_conds.push_back(it->second);
    }
    double leaf_work = 0;
    for (uint32_t sp = 0; sp < (1u << runtime.size()); sp++) {
      std::map<uint32_t, Contribs> bs = by_slot;
      for (size_t q = 0; q < runtime.size(); q++) {
        const uint32_t pick = ((sp >> q) & 1) ? runtime[q][2] : runtime[q][1];   // bit set: A >= B, min = B
        for (auto &x : held[pick]) bs[x.first].push_back({runtime[q][0], (uint64_t)x.second});
      }
      // slots -> basis entries (two slots naming one entry merge their contributions)
      std::map<int, Contribs> by_entry;
      for (auto &kv : bs) {
        Contribs &cs = by_entry[pmap[kv.first]];
        cs.insert(cs.end(), kv.second.begin(), kv.second.end());
      }
      LeafForm lf;
      for (auto &kv : by_entry) {
        const BEntry &b = g.ents[kv.first];
        // a term's weight sum_col W_col coefsum_col has |.| <= 2^62.01 max |coefsum|
        // (sum |W| <= 2^62 + 16): below 2^95, it fits a 96-bit record
        std::map<uint32_t, i128> cs;
        for (auto &c : kv.second) cs[c.first] += (i128)(int64_t)c.second;
        i128 mx = 0;
        for (auto &c : cs) mx = std::max(mx, c.second < 0 ? -c.second : c.second);
        const bool narrow = mx < ((i128)1 << 32);
        if (b.kind == BK_CONST) { lf.const_first = true; lf.const_c = kv.second; }
        else if (!narrow) lf.twide.push_back(kv);
        else if (fits_u32(b.range)) lf.t32.push_back(kv);
        else lf.t64.push_back(kv);
      }
      if (lf.t64.size() > 255 || lf.t32.size() > 255 || lf.twide.size() > 255)
        throw BuildError{PM_ERR_UNSUPPORTED, "too many terms in a piece"};
      // exact integer operations of one evaluation: 32-bit multiply-adds of the 128-bit
      // products (12 for a 64-bit value, 7 for a 32-bit one), the constant's 128-bit
      // add, 2 per condition bit, the exact division, the threshold compare
      leaf_work += 4.0 * lf.const_first + 12.0 * (lf.t64.size() + lf.twide.size()) + 7.0 * lf.t32.size() +
                   2.0 * (NC + runtime.size()) + (pf.den ? 8.0 : 0.0) + 4.0;
      f.leaves.push_back(std::move(lf));
    }
    work += leaf_work / f.leaves.size();
    pf.pieces.push_back(std::move(f));
  }
  pf.work = work / npieces;
  g.prog_of_table[table_id] = (int)g.progs.size();
  g.progs.push_back(std::move(pf));
}

void check_limits(const Group &g) {
  if ((int)g.ents.size() > BASIS_MAX) throw BuildError{PM_ERR_BUSY, "basis"};
  if ((int)g.conds.size() > GCOND_MAX) throw BuildError{PM_ERR_BUSY, "conditions"};
}

void pad4(std::vector<uint32_t> &o) {
  while (o.size() % 4) o.push_back(0);
}

// The group's image: header, basis definitions (ordered by level), condition
// definitions, programs and the variant -> program map (layout in kernels.h).
// Weight words are left zero; `targets`/`contrib` say how to fill them per call
// (word offsets relative to the image start).
size_t emit_group(const Group &g0, std::vector<uint32_t> &img, std::vector<uint4> &targets,
                  std::vector<uint4> &contrib, std::vector<double> &prog_work) {
  // order the basis by level, so that every product follows its factors
  const int B = (int)g0.ents.size();
  std::vector<int> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return g0.ents[a].level < g0.ents[b].level; });
  std::vector<int> remap(B);
  for (int k = 0; k < B; k++) remap[order[k]] = k;
  int nlev = 0;
  for (auto &e : g0.ents) nlev = std::max(nlev, e.level + 1);
  img.assign(RankLayout::HDR_WORDS, 0);
  img[RankLayout::H_B] = (uint32_t)B;
  img[RankLayout::H_NLEV] = (uint32_t)nlev;
  img[RankLayout::H_NCOND] = (uint32_t)g0.conds.size();
  for (int L = 0; L < nlev; L++) {
    int end = 0;
    for (int k = 0; k < B; k++)
      if (g0.ents[order[k]].level <= L) end = k + 1;
    img[RankLayout::H_LEVEL_END + L] = (uint32_t)end;
  }
  img[RankLayout::H_OFF_BASIS] = (uint32_t)img.size();
  for (int k = 0; k < B; k++) {
    const BEntry &e = g0.ents[order[k]];
    uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (e.kind == BK_ATOM) {
      // a0..a3, b, c, magic, and the kind word: kind | shift2 << 8 | numerator-may-be-negative << 16
      std::memcpy(w, e.atom, 7 * 4);
      w[7] = (uint32_t)BK_ATOM | (((e.atom[7] >> 8) & 0xFF) << 8) | (((e.atom[7] >> 16) & 1) << 16);
    } else {
      w[0] = (uint32_t)(e.kind == BK_PROD ? remap[e.i] : e.i);
      w[1] = (uint32_t)(e.kind == BK_PROD ? remap[e.j] : 0);
      w[7] = (uint32_t)e.kind;
    }
    img.insert(img.end(), w, w + 8);
  }
  img[RankLayout::H_OFF_COND] = (uint32_t)img.size();
  for (auto &cnd : g0.conds) {
    const int nt = (int)(cnd.size() - 1) / 2;
    img.push_back((uint32_t)nt);
    img.push_back((uint32_t)cnd[0]);
    img.push_back((uint32_t)((uint64_t)cnd[0] >> 32));
    for (int t = 0; t < nt; t++) {
      img.push_back((uint32_t)remap[(int)cnd[1 + 2 * t]]);
      img.push_back((uint32_t)cnd[2 + 2 * t]);
      img.push_back((uint32_t)((uint64_t)cnd[2 + 2 * t] >> 32));
    }
  }
  pad4(img);
  // flags of a target: 1 = a 96-bit weight (three words; the fourth holds the term's
  // basis entry)
  auto add_target = [&](uint32_t word, const Contribs &cs, uint32_t flags) {
    targets.push_back(make_uint4(word, (uint32_t)contrib.size(), (uint32_t)cs.size(), flags));
    for (auto &cc : cs) contrib.push_back(make_uint4(cc.first, 0, (uint32_t)cc.second, (uint32_t)(cc.second >> 32)));
  };
  auto cond_ids = [&](const int *ids, int n, int first) {
    uint32_t x = 0;
    for (int c = first; c < n && c < first + 5; c++) x |= (uint32_t)ids[c] << (6 * (c - first));
    return x;
  };
  // a leaf record [n64 << 8 | n32 << 16 | nwide << 24, term records, denominator block
  // or 0, constant present] and its term records
  auto emit_leaf = [&](uint32_t rec, const LeafForm &lf, uint32_t den_off) {
    const uint32_t toff = (uint32_t)img.size();
    // the constant's weight comes first, zero when the leaf has no constant term
    add_target(toff, lf.const_first ? lf.const_c : Contribs{}, 0);
    img.resize(img.size() + 4, 0);
    for (auto *cls : {&lf.t64, &lf.t32})
      for (auto &t : *cls) {
        add_target((uint32_t)img.size(), t.second, 1);
        img.insert(img.end(), {0u, 0u, 0u, (uint32_t)remap[t.first]});   // padding: entry 0, weight 0
      }
    for (auto &t : lf.twide) {
      add_target((uint32_t)img.size(), t.second, 0);
      img.insert(img.end(), {0u, 0u, 0u, 0u, (uint32_t)remap[t.first], 0u, 0u, 0u});
    }
    img[rec + 0] = ((uint32_t)lf.t64.size() << 8) | ((uint32_t)lf.t32.size() << 16) | ((uint32_t)lf.twide.size() << 24);
    img[rec + 1] = toff;
    img[rec + 2] = den_off;
    img[rec + 3] = 1;
  };
  // Every leaf of a program is padded to the program's widest shape (zero weights on
  // basis entry 0), so that a program has one shape: its 64-bit- and 32-bit-class term
  // counts, or no shape (0xFFFF) when it has 128-bit weights.  Variants are walked in
  // runs of one shape, each run by a loop with fixed term counts.
  std::vector<ProgForm> progs = g0.progs;
  std::vector<uint32_t> shape(progs.size());
  for (size_t pi = 0; pi < progs.size(); pi++) {
    size_t n64 = 0, n32 = 0, nw = 0;
    for (auto &pc : progs[pi].pieces)
      for (auto &lf : pc.leaves) {
        n64 = std::max(n64, lf.t64.size());
        n32 = std::max(n32, lf.t32.size());
        nw = std::max(nw, lf.twide.size());
      }
    for (auto &pc : progs[pi].pieces)
      for (auto &lf : pc.leaves) {
        while (lf.t64.size() < n64) lf.t64.push_back({0, Contribs{}});
        while (lf.t32.size() < n32) lf.t32.push_back({0, Contribs{}});
      }
    shape[pi] = nw ? 0xFFFFu : (uint32_t)(n64 | (n32 << 8));
  }
  std::vector<uint32_t> prog_off(progs.size());
  prog_work.clear();
  for (size_t pi = 0; pi < progs.size(); pi++) {
    const ProgForm &pf = progs[pi];
    const uint32_t base = (uint32_t)img.size();
    prog_off[pi] = base;
    prog_work.push_back(pf.work);
    const uint32_t np = (uint32_t)pf.pieces.size();
    // nodes: a condition node [1 | ncond << 8 | piece records << 16, condition ids 0-4,
    // ids 5-9 (6 bits each), LUT offset] over the table's conditions (omitted for one
    // piece without conditions); piece records: a leaf, or a sub node [2 | nsub << 8,
    // post-condition ids (6 bits each), children, 0] over 2^nsub leaves
    const bool cond_node = pf.ncond > 0 || np > 1;
    if (cond_node) img.resize(img.size() + 4, 0);
    uint32_t den_off = 0;
    if (pf.den) {
      den_off = (uint32_t)img.size();
      const uint32_t d[8] = {pf.den_shift, 0, 0, 0, pf.den_inv[0], pf.den_inv[1], pf.den_inv[2], pf.den_inv[3]};
      img.insert(img.end(), d, d + 8);
    }
    const uint32_t precs = (uint32_t)img.size();
    img.resize(img.size() + 4 * np, 0);
    if (cond_node) {
      if (precs > 0xFFFF) throw BuildError{PM_ERR_UNSUPPORTED, "ranking group image too large"};
      img[base + 0] = 1u | ((uint32_t)pf.ncond << 8) | (precs << 16);
      img[base + 1] = cond_ids(pf.gcond, pf.ncond, 0);
      img[base + 2] = cond_ids(pf.gcond, pf.ncond, 5);
      img[base + 3] = (uint32_t)img.size();
      for (size_t b = 0; b < pf.lut.size(); b += 4) {
        uint32_t x = 0;
        for (size_t q = 0; q < 4 && b + q < pf.lut.size(); q++) x |= (uint32_t)pf.lut[b + q] << (8 * q);
        img.push_back(x);
      }
      pad4(img);
    }
    for (uint32_t p = 0; p < np; p++) {
      const PieceForm &f = pf.pieces[p];
      const uint32_t rec = precs + 4 * p;
      if (f.sub_conds.empty()) {
        emit_leaf(rec, f.leaves[0], den_off);
        continue;
      }
      const uint32_t kids = (uint32_t)img.size();
      img.resize(img.size() + 4 * f.leaves.size(), 0);
      img[rec + 0] = 2u | ((uint32_t)f.sub_conds.size() << 8);
      img[rec + 1] = cond_ids(f.sub_conds.data(), (int)f.sub_conds.size(), 0);
      img[rec + 2] = kids;
      img[rec + 3] = 0;
      for (size_t l = 0; l < f.leaves.size(); l++) emit_leaf(kids + 4 * (uint32_t)l, f.leaves[l], den_off);
    }
    if (!cond_node) prog_off[pi] = precs;   // the program's root is its only piece record
    if (img.size() - base > (size_t)PROG_MAX_WORDS)
      throw BuildError{PM_ERR_UNSUPPORTED, "a table's ranking program exceeds " + std::to_string(PROG_MAX_WORDS * 4) +
                                               " bytes"};
  }
  // walk order: variants by shape (stable), as runs [shape, first position, count]; per
  // position the program's root record and the variant's index in the group (16 bits each)
  const size_t nvar = g0.var_prog.size();
  std::vector<uint32_t> walk(nvar);
  std::iota(walk.begin(), walk.end(), 0u);
  std::stable_sort(walk.begin(), walk.end(),
                   [&](uint32_t a, uint32_t b) { return shape[g0.var_prog[a]] < shape[g0.var_prog[b]]; });
  auto put16 = [&](auto value_of) {
    for (size_t q = 0; q < nvar; q += 2) {
      uint32_t x = value_of(walk[q]);
      if (q + 1 < nvar) x |= value_of(walk[q + 1]) << 16;
      img.push_back(x);
    }
    pad4(img);
  };
  img[RankLayout::H_OFF_VARMAP] = (uint32_t)img.size();
  put16([&](uint32_t v) { return prog_off[g0.var_prog[v]]; });
  img[RankLayout::H_OFF_VIDMAP] = (uint32_t)img.size();
  put16([&](uint32_t v) { return v; });
  img[RankLayout::H_OFF_RUNS] = (uint32_t)img.size();
  uint32_t nruns = 0;
  for (size_t q = 0; q < nvar;) {
    size_t e = q;
    const uint32_t sh = shape[g0.var_prog[walk[q]]];
    while (e < nvar && shape[g0.var_prog[walk[e]]] == sh) e++;
    img.insert(img.end(), {sh, (uint32_t)q, (uint32_t)(e - q), 0u});
    nruns++;
    q = e;
  }
  img[RankLayout::H_NRUNS] = nruns;
  img[RankLayout::H_WORDS] = (uint32_t)img.size();
  return img.size();
}

}  // namespace

// Test hook, not part of the C ABI in pm.h: the ranking group of a list of compiled
// tables (all of one parameter count and box, each one variant), for host-side checks
// of the group builder.  tables: n images concatenated; out: the group's image;
// targets: 4 words each (image word, first contribution, count, 0); contrib: 4 words
// each (column, 0, coef_lo, coef_hi).  Returns 0, 1 if a buffer is too small (sizes
// are still reported), -1 for tables that do not form one group (with the reason in
// pm_last_error).
extern "C" int pmx_rank_group(const uint32_t *tables, const size_t *words, int n, uint32_t *out, size_t out_cap,
                              size_t *out_words, uint32_t *tgt, size_t tgt_cap, size_t *n_tgt, uint32_t *con,
                              size_t con_cap, size_t *n_con) {
  Group g;
  std::vector<uint32_t> img;
  std::vector<uint4> targets, contrib;
  std::vector<double> work;
  try {
    size_t off = 0;
    for (int i = 0; i < n; i++) {
      std::vector<uint32_t> T(tables + off, tables + off + words[i]);
      off += words[i];
      if (T.size() < (size_t)pmt::HEADER_WORDS || T[pmt::H_MAGIC] != pmt::MAGIC || T[pmt::H_WORDS] != T.size())
        throw BuildError{PM_ERR_INVALID_ARG, "not a table image"};
      if (i == 0) {
        g.P = (int)T[pmt::H_NPARAMS];
        if (g.P > 4) throw BuildError{PM_ERR_INVALID_ARG, "malformed table"};
        for (int p = 0; p < 4; p++) { g.lo[p] = (int32_t)T[pmt::H_BOX_LO + p]; g.hi[p] = (int32_t)T[pmt::H_BOX_HI + p]; }
        g.ents.resize(g.P);
        for (int p = 0; p < g.P; p++) {
          g.ents[p].kind = BK_PARAM;
          g.ents[p].i = p;
          g.ents[p].range = Range{g.lo[p], g.hi[p]};
        }
      }
      add_table(g, i, T);
      check_limits(g);
      g.var_prog.push_back(g.prog_of_table[i]);
    }
    emit_group(g, img, targets, contrib, work);
  } catch (const BuildError &e) {
    pm_set_error(e.code, e.msg);
    return -1;
  }
  *out_words = img.size();
  *n_tgt = targets.size();
  *n_con = contrib.size();
  if (img.size() > out_cap || targets.size() > tgt_cap || contrib.size() > con_cap) return 1;
  std::memcpy(out, img.data(), img.size() * 4);
  std::memcpy(tgt, targets.data(), targets.size() * 16);
  std::memcpy(con, contrib.data(), contrib.size() * 16);
  return 0;
}

// ------------------------------------------------------------------ plans

static std::string plan_key(const int32_t *tables, const int32_t *var_off, int T, const int64_t *pt_off, int slice) {
  std::string key;
  key.append((const char *)&T, sizeof T);
  key.append((const char *)&slice, sizeof slice);
  key.append((const char *)tables, sizeof(int32_t) * var_off[T]);
  key.append((const char *)var_off, sizeof(int32_t) * (T + 1));
  key.append((const char *)pt_off, sizeof(int64_t) * (T + 1));
  return key;
}

// The host side of a plan: what the launch reads, before it is uploaded.
struct HostPlan {
  std::vector<uint32_t> img;                 // every group's image, 16-byte aligned
  std::vector<uint4> targets, contrib;       // weight-fill recipe (absolute image words)
  std::vector<int4> groups;                  // per group: two int4 (see RankArgs)
  std::vector<int4> tmpl;                    // per template: three int4 (see RankArgs)
  std::vector<int4> chunks;
  std::vector<int2> units;
  int slots = 0, max_words = 0, max_basis = 0;
  int64_t evals = 0;
  double total_work = 0;
};

static pm_status build_host_plan(pm_ctx *c, const int32_t *tables, const int32_t *var_off, int T,
                                 const int64_t *pt_off, int slice_max, HostPlan &hp) {
  std::vector<uint32_t> &img = hp.img;
  std::vector<uint4> &targets = hp.targets, &contrib = hp.contrib;
  std::vector<int4> &groups = hp.groups;
  std::vector<int4> &tmpl = hp.tmpl;
  tmpl.assign(3 * T, make_int4(0, 0, 0, 0));
  std::vector<std::vector<double>> gwork;    // per group: average work of one evaluation per variant
  std::vector<int> gbasis;                   // per group: basis entries + conditions
  std::vector<int> first_group(T + 1, 0);
  int &max_words = hp.max_words, &max_basis = hp.max_basis;
  double &total_work = hp.total_work;
  int64_t &evals = hp.evals;
  // a ranking entry keeps the variant's index within its template in 16 bits
  for (int t = 0; t < T; t++)
    if (var_off[t + 1] < var_off[t] || var_off[t + 1] - var_off[t] > 65536)
      return pm_set_error(PM_ERR_INVALID_ARG, "at most 65,536 variants per template");
  // Tables with the same image evaluate alike; they share one program in a group.
  std::map<std::vector<uint32_t>, int> image_id;
  std::vector<int> canon(c->tables.size(), -1);
  auto canonical = [&](int id) {
    if (canon[id] < 0) {
      auto it = image_id.find(c->tables[id]);
      if (it == image_id.end()) it = image_id.emplace(c->tables[id], id).first;
      canon[id] = it->second;
    }
    return canon[id];
  };
  try {
    for (int t = 0; t < T; t++) {
      first_group[t] = (int)groups.size() / 2;
      const int v0 = var_off[t], v1 = var_off[t + 1];
      if (v1 == v0) { first_group[t + 1] = first_group[t]; continue; }
      const auto &w0 = c->tables[tables[v0]];
      Group cur;
      auto start = [&](int vb) {
        cur = Group();
        cur.P = (int)w0[pmt::H_NPARAMS];
        for (int p = 0; p < 4; p++) { cur.lo[p] = (int32_t)w0[pmt::H_BOX_LO + p]; cur.hi[p] = (int32_t)w0[pmt::H_BOX_HI + p]; }
        cur.ents.resize(cur.P);
        for (int p = 0; p < cur.P; p++) {
          cur.ents[p].kind = BK_PARAM;
          cur.ents[p].i = p;
          cur.ents[p].range = Range{cur.lo[p], cur.hi[p]};
        }
        cur.var_begin = vb;
      };
      auto finish = [&]() {
        std::vector<uint32_t> gi;
        std::vector<uint4> tg;
        std::vector<double> pw;
        emit_group(cur, gi, tg, contrib, pw);
        const uint32_t base = (uint32_t)img.size();
        for (auto &x : tg) targets.push_back(make_uint4(x.x + base, x.y, x.z, x.w));
        img.insert(img.end(), gi.begin(), gi.end());
        max_words = std::max(max_words, (int)gi.size());
        max_basis = std::max(max_basis, (int)cur.ents.size());
        const int nvar = (int)cur.var_prog.size();
        const int gidx = (int)groups.size() / 2;
        groups.push_back(make_int4((int)base, (int)gi.size(), cur.var_begin, nvar));
        groups.push_back(make_int4(t, gidx - first_group[t], 0, 0));
        std::vector<double> vw(nvar);
        for (int v = 0; v < nvar; v++) vw[v] = pw[cur.var_prog[v]];
        gwork.push_back(vw);
        gbasis.push_back((int)cur.ents.size() + (int)cur.conds.size());
      };
      // image words of the group without its variant map, refreshed when a program is added
      int fixed_words = 0;
      auto map_words = [](size_t nvar) { return (int)(((nvar + 1) / 2 + 3) & ~(size_t)3); };
      start(0);
      for (int v = v0; v < v1; v++) {
        const int id = tables[v];
        if (id < 0 || id >= (int)c->tables.size()) return pm_set_error(PM_ERR_NOT_FOUND, "unknown table id");
        const auto &w = c->tables[id];
        if ((int)w[pmt::H_K] != 32) return pm_set_error(PM_ERR_INVALID_ARG, "fused ranking needs PM_LAYOUT_32 tables");
        if (w[pmt::H_NPARAMS] != w0[pmt::H_NPARAMS])
          return pm_set_error(PM_ERR_INVALID_ARG, "variants of one template differ in parameter count");
        if (std::memcmp(&w[pmt::H_BOX_LO], &w0[pmt::H_BOX_LO], 8 * sizeof(uint32_t)))
          return pm_set_error(PM_ERR_UNSUPPORTED, "variants of one template must share one parameter box");
        const int cid = canonical(id);
        if ((int)cur.var_prog.size() >= slice_max && !cur.var_prog.empty()) {
          finish();
          start(v - v0);
          fixed_words = 0;
        }
        Group saved = cur;
        bool ok = true;
        try {
          add_table(cur, cid, c->tables[cid]);
          check_limits(cur);
        } catch (const BuildError &e) {
          if (e.code != PM_ERR_BUSY) throw;
          ok = false;
        }
        int fixed_new = fixed_words;
        if (ok && cur.progs.size() != saved.progs.size()) {
          std::vector<uint32_t> gi;
          std::vector<uint4> tg, cb;
          std::vector<double> pw;
          emit_group(cur, gi, tg, cb, pw);
          fixed_new = (int)gi.size() - map_words(cur.var_prog.size());
        }
        if (ok && fixed_new + map_words(cur.var_prog.size() + 1) > GROUP_MAX_WORDS) ok = false;
        if (ok) {
          fixed_words = fixed_new;
          cur.var_prog.push_back(cur.prog_of_table[cid]);
          continue;
        }
        // this variant opens a new group
        if (saved.var_prog.empty()) return pm_set_error(PM_ERR_UNSUPPORTED, "a table too large for the ranking kernel");
        cur = saved;
        finish();
        start(v - v0);
        add_table(cur, cid, c->tables[cid]);
        check_limits(cur);
        {
          std::vector<uint32_t> gi;
          std::vector<uint4> tg, cb;
          std::vector<double> pw;
          emit_group(cur, gi, tg, cb, pw);
          fixed_words = (int)gi.size() - map_words(0);
          if (fixed_words + map_words(1) > GROUP_MAX_WORDS)
            return pm_set_error(PM_ERR_UNSUPPORTED, "a table too large for the ranking kernel");
        }
        cur.var_prog.push_back(cur.prog_of_table[cid]);
      }
      finish();
      first_group[t + 1] = (int)groups.size() / 2;
      tmpl[3 * t] = make_int4((int)w0[pmt::H_NPARAMS], first_group[t + 1] - first_group[t], 0, 0);
      tmpl[3 * t + 1] = make_int4((int)w0[pmt::H_BOX_LO], (int)w0[pmt::H_BOX_LO + 1], (int)w0[pmt::H_BOX_LO + 2],
                                  (int)w0[pmt::H_BOX_LO + 3]);
      tmpl[3 * t + 2] = make_int4((int)w0[pmt::H_BOX_HI], (int)w0[pmt::H_BOX_HI + 1], (int)w0[pmt::H_BOX_HI + 2],
                                  (int)w0[pmt::H_BOX_HI + 3]);
    }
  } catch (const BuildError &e) {
    return pm_set_error(e.code == PM_ERR_BUSY ? PM_ERR_UNSUPPORTED : e.code, e.msg);
  }
  // Work units: (point chunk of 32, group).  A chunk whose template has S > 1 groups
  // is finished by the last of its S units (partial lists in scratch).  Units are
  // ordered most expensive first (longest processing time first).
  struct U { int chunk, group; double cost; };
  std::vector<int4> &chunks = hp.chunks;
  std::vector<U> units;
  int &slots = hp.slots;
  for (int t = 0; t < T; t++) {
    const int S = first_group[t + 1] - first_group[t];
    for (int64_t p = pt_off[t]; p < pt_off[t + 1]; p += RankLayout::POINTS) {
      const int n = (int)std::min<int64_t>(RankLayout::POINTS, pt_off[t + 1] - p);
      const int ch = (int)chunks.size();
      chunks.push_back(make_int4(t, (int)p, n, S > 1 ? slots : -1));
      if (S > 1) slots += S;
      if (S == 0) units.push_back({ch, -1, 0.0});   // no variants: the points get empty rankings
      for (int g = first_group[t]; g < first_group[t + 1]; g++) {
        double gw = 0;
        for (double x : gwork[g]) gw += x;
        // about ten operations per basis value and condition, once per point of the unit
        units.push_back({ch, g, (gw + 10.0 * gbasis[g]) * n});
        total_work += gw * n;
        evals += (int64_t)gwork[g].size() * n;
      }
    }
  }
  std::stable_sort(units.begin(), units.end(), [](const U &a, const U &b) { return a.cost > b.cost; });
  hp.units.resize(units.size());
  for (size_t i = 0; i < units.size(); i++) hp.units[i] = make_int2(units[i].chunk, units[i].group);
  return PM_OK;
}

static pm_status build_plan(pm_ctx *c, const int32_t *tables, const int32_t *var_off, int T, const int64_t *pt_off,
                            int slice_max, Plan **out) {
  HostPlan hp;
  pm_status hs = build_host_plan(c, tables, var_off, T, pt_off, slice_max, hp);
  if (hs) return hs;
  const std::vector<uint32_t> &img = hp.img;
  const std::vector<uint4> &targets = hp.targets, &contrib = hp.contrib;
  const std::vector<int4> &groups = hp.groups, &tmpl = hp.tmpl, &chunks = hp.chunks;
  const std::vector<int2> &hu = hp.units;
  Plan *p = new Plan();
  auto alloc = [&](const void *h, size_t bytes, void **d) -> pm_status {
    CU(cudaMalloc(d, std::max<size_t>(bytes, 16)));
    p->dev.push_back(*d);
    if (h && bytes) CU(cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice));
    return PM_OK;
  };
  auto fail = [&](pm_status s) {
    for (void *d : p->dev) cudaFree(d);
    delete p;
    return s;
  };
  void *d;
  pm_status s;
  if ((s = alloc(img.data(), img.size() * 4, &d))) return fail(s);
  p->d_img = (uint32_t *)d;
  if ((s = alloc(targets.data(), targets.size() * sizeof(uint4), &d))) return fail(s);
  p->d_targets = (const uint4 *)d;
  if ((s = alloc(contrib.data(), contrib.size() * sizeof(uint4), &d))) return fail(s);
  p->d_contrib = (const uint4 *)d;
  p->n_targets = (int)targets.size();
  if ((s = alloc(groups.data(), groups.size() * sizeof(int4), &d))) return fail(s);
  p->d_groups = (const int4 *)d;
  if ((s = alloc(tmpl.data(), tmpl.size() * sizeof(int4), &d))) return fail(s);
  p->d_tmpl = (const int4 *)d;
  if ((s = alloc(chunks.data(), chunks.size() * sizeof(int4), &d))) return fail(s);
  p->d_chunks = (const int4 *)d;
  if ((s = alloc(hu.data(), hu.size() * sizeof(int2), &d))) return fail(s);
  p->d_units = (const int2 *)d;
  if ((s = alloc(nullptr, sizeof(int) * (chunks.size() + 1), &d))) return fail(s);
  p->d_counter = (int *)d;  // [0] unit counter, [1..] per-chunk group counters
  if ((s = alloc(nullptr, (size_t)std::max(hp.slots, 1) * 16 * RankLayout::POINTS * 8, &d))) return fail(s);
  p->d_part_k = (int64_t *)d;
  p->n_chunks = (int)chunks.size();
  p->n_units = (int)hu.size();
  p->n_groups = (int)groups.size() / 2;
  p->n_templates = T;
  p->total_points = pt_off[T];
  p->total_evals = hp.evals;
  p->work_per_eval = hp.evals ? hp.total_work / (double)hp.evals : 0;
  p->img_words = hp.max_words;
  p->basis_cap = std::max(1, hp.max_basis);
  p->slice_max = slice_max;
  *out = p;
  return PM_OK;
}

// Test hook, not part of the C ABI in pm.h: the host arrays of the plan of an argument
// set of pm_eval_predict_topk (built with slice size `slice`, 0 = unlimited), before the
// upload: sizes[0..7] = image words, targets, contributions, groups, templates, chunks,
// units, partial slots; each array is copied when its buffer is large enough (NULL
// skips it).  Returns 0, or a pm_status error.
extern "C" int pmx_rank_plan(pm_ctx *c, const int32_t *tables, const int32_t *var_off, int32_t T,
                             const int64_t *pt_off, int32_t slice, int64_t *sizes, uint32_t *img, size_t img_cap,
                             uint4 *targets, size_t tg_cap, uint4 *contrib, size_t con_cap, int4 *groups,
                             size_t gr_cap, int4 *tmpl, size_t tm_cap, int4 *chunks, size_t ch_cap, int2 *units,
                             size_t un_cap) {
  if (!c || T <= 0 || !tables || !var_off || !pt_off || !sizes) return PM_ERR_INVALID_ARG;
  HostPlan hp;
  pm_status s = build_host_plan(c, tables, var_off, T, pt_off, slice > 0 ? slice : (1 << 30), hp);
  if (s) return s;
  sizes[0] = (int64_t)hp.img.size();
  sizes[1] = (int64_t)hp.targets.size();
  sizes[2] = (int64_t)hp.contrib.size();
  sizes[3] = (int64_t)hp.groups.size() / 2;
  sizes[4] = T;
  sizes[5] = (int64_t)hp.chunks.size();
  sizes[6] = (int64_t)hp.units.size();
  sizes[7] = hp.slots;
  auto put = [](void *dst, size_t cap, const void *src, size_t n, size_t el) {
    if (dst && n <= cap) std::memcpy(dst, src, n * el);
  };
  put(img, img_cap, hp.img.data(), hp.img.size(), 4);
  put(targets, tg_cap, hp.targets.data(), hp.targets.size(), 16);
  put(contrib, con_cap, hp.contrib.data(), hp.contrib.size(), 16);
  put(groups, gr_cap, hp.groups.data(), hp.groups.size(), 16);
  put(tmpl, tm_cap, hp.tmpl.data(), hp.tmpl.size(), 16);
  put(chunks, ch_cap, hp.chunks.data(), hp.chunks.size(), 16);
  put(units, un_cap, hp.units.data(), hp.units.size(), 8);
  return PM_OK;
}

// Launch shape of a plan: warps per CTA and CTAs per SM (autotuned when enabled).
static void default_shape(pm_ctx *c, Plan *p, int nw) {
  p->nw = nw;
  const int bps = pmd::rank_max_blocks_per_sm(nw, p->img_words, p->basis_cap);
  p->grid = std::max(1, c->n_sms * std::max(1, bps));
}

static constexpr int DEFAULT_SLICE = 1 << 30;   // one group per template unless a limit splits it
static constexpr int DEFAULT_NW = 8;

pm_status ctx_plan_k2(pm_ctx *c, const int32_t *tables, const int32_t *var_off, int T, const int64_t *pt_off,
                      Plan **out) {
  if (var_off[0] != 0 || pt_off[0] != 0) return pm_set_error(PM_ERR_INVALID_ARG, "offsets must start at 0");
  for (int t = 0; t < T; t++) {
    if (var_off[t + 1] < var_off[t] || pt_off[t + 1] < pt_off[t])
      return pm_set_error(PM_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (var_off[t + 1] - var_off[t] > 65536)
      return pm_set_error(PM_ERR_INVALID_ARG, "at most 65,536 variants per template");
  }
  if (pt_off[T] > (int64_t(1) << 31) - 64) return pm_set_error(PM_ERR_INVALID_ARG, "too many points");
  const std::string key = plan_key(tables, var_off, T, pt_off, 0);
  auto it = c->plans.find(key);
  if (it != c->plans.end()) { *out = it->second; return PM_OK; }
  Plan *p = nullptr;
  pm_status s = build_plan(c, tables, var_off, T, pt_off, DEFAULT_SLICE, &p);
  if (s) return s;
  default_shape(c, p, DEFAULT_NW);
  p->key = key;
  c->plans[key] = p;
  *out = p;
  return PM_OK;
}

static pm_status launch_plan(pm_ctx *c, Plan *p, const int64_t *pts, const double *w, int topk, int32_t *idx,
                             double *t, cudaStream_t st, int nw, int grid) {
  CU(cudaMemsetAsync(p->d_counter, 0, sizeof(int) * (p->n_chunks + 1), st));
  CU(pmd::launch_k2_weights(p->d_img, p->d_targets, p->d_contrib, p->n_targets, w, st));
  pmd::RankArgs a;
  a.img = p->d_img;
  a.groups = p->d_groups;
  a.tmpl = p->d_tmpl;
  a.chunks = p->d_chunks;
  a.units = p->d_units;
  a.n_units = p->n_units;
  a.unit_counter = p->d_counter;
  a.chunk_count = p->d_counter + 1;
  a.part_k = p->d_part_k;
  a.points = pts;
  a.w = w;
  a.topk = topk;
  a.top_idx = idx;
  a.top_t = t;
  a.status = c->d_status;
  a.img_words = p->img_words;
  a.basis_cap = p->basis_cap;
  CU(pmd::launch_rank(a, nw, grid, st));
  return PM_OK;
}

// ------------------------------------------------------------------ autotuner
//
// The tuner searches the schedule and the launch shape of the fused kernel on the
// caller's own inputs: the slice size (at most this many variants per ranking group,
// so large templates split into several units per point chunk: finer load balance
// against more partial lists), warps per CTA (more warps share one chunk's basis and
// thresholds but hold more shared memory) and CTAs per SM.  Every candidate is timed
// over two launches after a warm-up; the fastest is kept per plan and, when
// PM_TUNE_CACHE names a file, persisted by workload signature.
static std::string plan_signature(const Plan *p) {
  std::ostringstream o;
  o << "T" << p->n_templates << "_P" << p->total_points << "_E" << p->total_evals << "_W"
    << (int)(p->work_per_eval + 0.5) << "_G" << p->n_groups;
  return o.str();
}

static bool tune_lookup(const std::string &path, const std::string &sig, int *slice, int *nw, int *bps) {
  if (path.empty()) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    char s[256];
    int a, b, q;
    if (sscanf(line.c_str(), " \"%255[^\"]\": [%d, %d, %d]", s, &q, &a, &b) == 4 && sig == s) {
      *slice = q;
      *nw = a;
      *bps = b;
      return true;
    }
  }
  return false;
}

static void tune_store(const std::string &path, const std::string &sig, int slice, int nw, int bps) {
  if (path.empty()) return;
  std::vector<std::string> lines;
  {
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line))
      if (line.find("\": [") != std::string::npos && line.find("\"" + sig + "\"") == std::string::npos) {
        while (!line.empty() && (line.back() == ',' || line.back() == ' ')) line.pop_back();
        lines.push_back(line);
      }
  }
  std::ostringstream o;
  o << "  \"" << sig << "\": [" << slice << ", " << nw << ", " << bps << "]";
  lines.push_back(o.str());
  std::ofstream f(path);
  f << "{\n";
  for (size_t i = 0; i < lines.size(); i++) f << lines[i] << (i + 1 < lines.size() ? ",\n" : "\n");
  f << "}\n";
}

// Replace the plan's schedule by the one of another slice size (same arguments).
static pm_status replan(pm_ctx *c, Plan *p, const int32_t *tables, const int32_t *var_off, const int64_t *pt_off,
                        int slice) {
  if (slice == p->slice_max) return PM_OK;
  Plan *q = nullptr;
  pm_status s = build_plan(c, tables, var_off, p->n_templates, pt_off, slice, &q);
  if (s) return s;
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  for (void *d : p->dev) cudaFree(d);
  const std::string key = p->key;
  *p = *q;
  p->key = key;
  delete q;
  return PM_OK;
}

static pm_status tune_plan(pm_ctx *c, Plan *p, const int32_t *tables, const int32_t *var_off, const int64_t *pt_off,
                           const int64_t *pts, const double *w, int topk, int32_t *idx, double *t, cudaStream_t st) {
  const std::string sig = plan_signature(p);
  int slice, nw, bps;
  if (tune_lookup(c->tune_path, sig, &slice, &nw, &bps)) {
    pm_status s = replan(c, p, tables, var_off, pt_off, slice);
    if (s) return s;
    p->nw = nw;
    p->grid = c->n_sms * bps;
    p->tuned = true;
    return PM_OK;
  }
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int b_slice = p->slice_max, b_nw = p->nw, b_bps = std::max(1, p->grid / c->n_sms);
  std::vector<std::array<double, 4>> log;   // every candidate (replanning resets the plan's own log)
  for (int cand_slice : {DEFAULT_SLICE, 2048, 1024, 512}) {
    pm_status s = replan(c, p, tables, var_off, pt_off, cand_slice);
    if (s) return s;
    for (int cand_nw : {4, 8}) {
      const int mx = std::max(1, pmd::rank_max_blocks_per_sm(cand_nw, p->img_words, p->basis_cap));
      for (int cand_bps = std::max(1, mx - 2); cand_bps <= mx; cand_bps++) {
        const int grid = c->n_sms * cand_bps;
        s = launch_plan(c, p, pts, w, topk, idx, t, st, cand_nw, grid);  // warm-up
        if (s) return s;
        CU(cudaEventRecord(e0, st));
        for (int r = 0; r < 2; r++) {
          s = launch_plan(c, p, pts, w, topk, idx, t, st, cand_nw, grid);
          if (s) return s;
        }
        CU(cudaEventRecord(e1, st));
        CU(cudaEventSynchronize(e1));
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        ms *= 0.5f;
        log.push_back({(double)cand_slice, (double)cand_nw, (double)cand_bps, (double)ms});
        if (ms < best) { best = ms; b_slice = cand_slice; b_nw = cand_nw; b_bps = cand_bps; }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pm_status s = replan(c, p, tables, var_off, pt_off, b_slice);
  if (s) return s;
  p->tune_log = log;
  p->nw = b_nw;
  p->grid = c->n_sms * b_bps;
  p->tuned = true;
  tune_store(c->tune_path, sig, b_slice, b_nw, b_bps);
  return PM_OK;
}

pm_status ctx_run_k2(pm_ctx *c, Plan *p, const int32_t *tables, const int32_t *var_off, const int64_t *pt_off,
                     const int64_t *pts, const double *w, int topk, int32_t *idx, double *t, cudaStream_t st) {
  if (c->tune && !p->tuned) {
    pm_status s = tune_plan(c, p, tables, var_off, pt_off, pts, w, topk, idx, t, st);
    if (s) return s;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st) CU(cudaStreamIsCapturing(st, &cs));
  if (!st || cs != cudaStreamCaptureStatusNone) return launch_plan(c, p, pts, w, topk, idx, t, st, p->nw, p->grid);
  const void *key[6] = {pts, w, idx, t, p->d_img, st};
  bool same = p->graph_exec && p->g_topk == topk && p->g_nw == p->nw && p->g_grid == p->grid &&
              std::memcmp(key, p->g_key, sizeof key) == 0;
  if (!same) {
    if (p->graph_exec) { cudaGraphExecDestroy(p->graph_exec); p->graph_exec = nullptr; }
    cudaGraph_t g;
    CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    pm_status s = launch_plan(c, p, pts, w, topk, idx, t, st, p->nw, p->grid);
    cudaError_t ee = cudaStreamEndCapture(st, &g);
    if (s) return s;
    CU(ee);
    cudaError_t ie = cudaGraphInstantiate(&p->graph_exec, g, 0);
    cudaGraphDestroy(g);
    CU(ie);
    std::memcpy(p->g_key, key, sizeof key);
    p->g_topk = topk;
    p->g_nw = p->nw;
    p->g_grid = p->grid;
  }
  CU(cudaGraphLaunch(p->graph_exec, st));
  return PM_OK;
}

extern "C" pm_status pm_tune(pm_ctx *c, int32_t enable, const char *cache_path) {
  if (!c) return pm_set_error(PM_ERR_INVALID_ARG, "null context");
  c->tune = enable;
  c->tune_path = cache_path ? cache_path : "";
  return PM_OK;
}

extern "C" pm_status pm_plan_info(pm_ctx *c, const int32_t *tables, const int32_t *var_off, int32_t n_templates,
                                  const int64_t *pt_off, int64_t *out /*[8]*/) {
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (n_templates <= 0 || !tables || !var_off || !pt_off || !out) return pm_set_error(PM_ERR_INVALID_ARG, "null argument");
  Plan *p;
  pm_status s = ctx_plan_k2(c, tables, var_off, n_templates, pt_off, &p);
  if (s) return s;
  out[0] = p->n_units;
  out[1] = p->total_evals;
  out[2] = (int64_t)(p->work_per_eval * 1000);
  out[3] = p->nw;
  out[4] = p->grid;
  out[5] = p->tuned;
  out[6] = p->n_groups;
  out[7] = p->slice_max >= DEFAULT_SLICE ? 0 : p->slice_max;
  return PM_OK;
}

extern "C" int32_t pm_plan_tune_log(pm_ctx *c, const int32_t *tables, const int32_t *var_off, int32_t n_templates,
                                    const int64_t *pt_off, double *out, int32_t cap) {
  if (!c || n_templates <= 0 || !tables || !var_off || !pt_off) return -1;
  const std::string key = plan_key(tables, var_off, n_templates, pt_off, 0);
  auto it = c->plans.find(key);
  if (it == c->plans.end()) return 0;
  const auto &log = it->second->tune_log;
  const int n = (int)log.size();
  for (int i = 0; i < n && i < cap; i++)
    for (int q = 0; q < 4; q++) out[4 * i + q] = log[i][q];
  return n;
}
