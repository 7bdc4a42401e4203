// Schedules for the persistent fused launch (pm_eval_predict_topk): work units,
// longest-processing-time order, launch-shape tuning and CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
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

static constexpr int K2_WARPS = 4;                  // warps per CTA of the fused kernel
static constexpr int UNIT_POINTS = 32 * K2_WARPS;   // one point per lane
static constexpr int SLICE_VARIANTS = 128;

// Algorithmic lane operations of one evaluation of a table (average over its pieces):
//   atom floor((a.n + b)/c):  P multiply-adds, 1 add, 5 for the magic division   P + 6
//   condition with t terms:   2 per 64-bit multiply-add, 2 for sum and compare    2t + 2
//   monomial product:         one 64-bit multiply                                 3
//   coefficient entry:        64-bit multiply and add                             5
//   non-empty column:         its weighted term of the exact fixed-point dot        15
//   post-op min(loads, stores): compare-select 2 + its weighted term             17
//   box check, piece lookup, top-k compare                                        10
static double table_work(const std::vector<uint32_t> &w) {
  const int P = (int)w[pmt::H_NPARAMS], A = (int)w[pmt::H_NATOMS], NC = (int)w[pmt::H_NCONDS];
  double ops = 10.0 + (double)A * (P + 6) + 17.0 * w[pmt::H_NPOST];
  const uint32_t *cd = w.data() + w[pmt::H_OFF_CONDS];
  for (int c = 0; c < NC; c++) {
    ops += 2.0 * cd[0] + 2.0;
    cd += 3 + 2 * cd[0];
  }
  const int np = std::max(1u, w[pmt::H_NPIECES]);
  double per = 0;
  for (int p = 0; p < np; p++) {
    const uint32_t *pc = w.data() + w[pmt::H_OFF_PIECES] + 4 * p;
    per += 3.0 * pc[1];                                    // products: one 64-bit multiply each
    const uint32_t *en = w.data() + w[pmt::H_OFF_ENTRIES] + pmt::ENTRY_WORDS * pc[2];
    for (uint32_t e = 0; e < pc[3]; e++, en += pmt::ENTRY_WORDS) {
      per += 5.0;                                          // 64-bit multiply-add
      if (en[2] & pmt::ENTRY_LAST) per += 15.0;            // weighted term of the column
    }
  }
  return ops + per / np;
}

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
  for (int a = 0; a < A && P + a < pmt::MAX_SLOTS; a++, at += pmt::ATOM_WORDS) {
    i128 mn = (int32_t)at[4], mx = (int32_t)at[4];
    for (int p = 0; p < P; p++) {
      const i128 k = (int32_t)at[p];
      mn += k >= 0 ? k * lo[p] : k * hi[p];
      mx += k >= 0 ? k * hi[p] : k * lo[p];
    }
    const i128 c = at[5] ? (i128)at[5] : 1;
    r[P + a] = Range{floor_div_wide(mn, c), floor_div_wide(mx, c)};
  }
  r[pmt::CONST_SLOT] = Range{1, 1};
  const uint32_t *pr = T.data() + T[pmt::H_OFF_PRODS] + pc[0];
  for (uint32_t j = 0; j < pc[1] && P + A + (int)j < pmt::MAX_SLOTS; j++) {
    const Range x = r[std::min<uint32_t>(pr[j] & 0xFF, pmt::MAX_SLOTS - 1)];
    const Range y = r[std::min<uint32_t>((pr[j] >> 8) & 0xFF, pmt::MAX_SLOTS - 1)];
    const i128 q[4] = {clamp_wide(x.lo * y.lo), clamp_wide(x.lo * y.hi), clamp_wide(x.hi * y.lo),
                       clamp_wide(x.hi * y.hi)};
    r[P + A + j] = Range{*std::min_element(q, q + 4), *std::max_element(q, q + 4)};
  }
  return r;
}

// K2 program of one table: the table's words up to its entries, then a weight image
// that turns the per-column sums and the weight dot product into one dot product over
// the piece's evaluation slots (sum_col W_col sum_e coef_e slot_e = sum_slot Weff_slot
// slot).  Per piece the image holds the slots with their 128-bit weights Weff (filled
// on the device from the call's weights: `targets` name each weight's position and its
// (column, coefficient) contributions).  A post-op min(hold A, hold B) whose sign of
// A - B is fixed over the box (interval arithmetic on the piece's slots) is folded
// into the dot as the smaller column; the others stay as runtime post-ops with the
// entries of their held columns.
//   piece header p (8 words at I + 8 p, I = the table's entry offset rounded up to 4):
//     [dot_w, n_dot, dot_s, const-first, hold_off, n_hold, post_off, n_post]
//   dot_w: n_dot uint4 weights; dot_s: n_dot slot words; hold entries (4 words):
//   {slot | hold << 8, 0, coef_lo, coef_hi}; post entries (8 words): weight (4 words),
//   hold A | hold B << 8, 0, 0, 0.  Offsets are words from the program start.
static bool build_k2_program(const std::vector<uint32_t> &T, uint32_t base, std::vector<uint32_t> &out,
                             std::vector<uint4> &targets, std::vector<uint4> &contrib) {
  auto pad4 = [&]() { while (out.size() % 4) out.push_back(0); };
  out.assign(T.begin(), T.begin() + T[pmt::H_OFF_ENTRIES]);   // entries and post-ops are replaced by the image
  pad4();
  const uint32_t I = (uint32_t)out.size();
  const uint32_t npieces = T[pmt::H_NPIECES], npost = T[pmt::H_NPOST];
  out.resize(I + 8 * npieces, 0);
  using Contribs = std::vector<std::pair<uint32_t, uint64_t>>;
  auto add_target = [&](uint32_t word, const Contribs &cs) {
    targets.push_back(make_uint4(base + word, (uint32_t)contrib.size(), (uint32_t)cs.size(), 0));
    for (auto &cc : cs) contrib.push_back(make_uint4(cc.first, 0, (uint32_t)cc.second, (uint32_t)(cc.second >> 32)));
  };
  for (uint32_t p = 0; p < npieces; p++) {
    const uint32_t *pc = T.data() + T[pmt::H_OFF_PIECES] + 4 * p;
    const uint32_t *en = T.data() + T[pmt::H_OFF_ENTRIES] + pmt::ENTRY_WORDS * pc[2];
    std::map<uint32_t, Contribs> by_slot;
    std::vector<std::vector<std::pair<uint32_t, int64_t>>> held(pmt::MAX_HOLD);   // hold -> (slot, coef)
    std::vector<std::pair<uint32_t, int64_t>> col_entries;
    for (uint32_t e = 0; e < pc[3]; e++, en += pmt::ENTRY_WORDS) {
      const uint32_t col = en[2] & 0xFF, slot = (en[2] >> 8) & 0xFF;
      if (slot >= (uint32_t)pmt::MAX_SLOTS) return false;
      const uint64_t coef = (uint64_t)en[0] | ((uint64_t)en[1] << 32);
      if (col < 32) by_slot[slot].push_back({col, coef});
      col_entries.push_back({slot, (int64_t)coef});
      if (en[2] & pmt::ENTRY_LAST) {
        const uint32_t hold = (en[2] >> 16) & 0xF;
        if (hold) {
          if (hold > (uint32_t)pmt::MAX_HOLD) return false;
          held[hold - 1] = col_entries;
        }
        col_entries.clear();
      }
    }
    // post-ops: fold those whose smaller operand is fixed over the box
    const std::vector<Range> rg = slot_ranges(T, pc);
    std::vector<uint32_t> runtime_posts;
    bool hold_used[pmt::MAX_HOLD] = {false, false, false, false};
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
      } else {
        runtime_posts.push_back(w);
        hold_used[ha] = hold_used[hb] = true;
      }
    }
    // the constant slot, when present, goes first: its product is the weight itself
    std::vector<std::pair<uint32_t, Contribs>> dots(by_slot.begin(), by_slot.end());
    const bool has_const = !dots.empty() && dots.back().first == pmt::CONST_SLOT;
    if (has_const) std::rotate(dots.begin(), dots.end() - 1, dots.end());
    const uint32_t dot_w = (uint32_t)out.size();
    for (auto &kv : dots) {
      add_target((uint32_t)out.size(), kv.second);
      out.resize(out.size() + 4, 0);
    }
    const uint32_t dot_s = (uint32_t)out.size();
    for (auto &kv : dots) out.push_back(kv.first);
    pad4();
    const uint32_t hold_off = (uint32_t)out.size();
    uint32_t n_hold = 0;
    for (int h = 0; h < pmt::MAX_HOLD; h++) {
      if (!hold_used[h]) continue;
      for (auto &x : held[h]) {
        const uint64_t cf = (uint64_t)x.second;
        const uint32_t e[4] = {x.first | ((uint32_t)h << 8), 0, (uint32_t)cf, (uint32_t)(cf >> 32)};
        out.insert(out.end(), e, e + 4);
        n_hold++;
      }
    }
    const uint32_t post_off = (uint32_t)out.size();
    for (uint32_t w : runtime_posts) {
      add_target((uint32_t)out.size(), {{w & 0xFF, 1ull}});
      const uint32_t e[8] = {0, 0, 0, 0, ((w >> 8) & 3) | (((w >> 16) & 3) << 8), 0, 0, 0};
      out.insert(out.end(), e, e + 8);
    }
    uint32_t *ip = out.data() + I + 8 * p;
    ip[0] = dot_w;
    ip[1] = (uint32_t)dots.size();
    ip[2] = dot_s;
    ip[3] = has_const ? 1u : 0u;
    ip[4] = hold_off;
    ip[5] = n_hold;
    ip[6] = post_off;
    ip[7] = (uint32_t)runtime_posts.size();
  }
  return true;
}

// Test hook, not part of the C ABI in pm.h: the K2 program of one compiled table (at
// word offset 0) and its weight-fill recipe, for host-side checks of the program
// builder.  targets: 4 words each (program word, first contribution, count, 0);
// contrib: 4 words each (column, 0, coef_lo, coef_hi).  Returns 0, 1 if a buffer is
// too small (sizes are still reported), -1 for a malformed table.
extern "C" int pmx_k2_program(const uint32_t *table, size_t words, uint32_t *prog, size_t prog_cap,
                              size_t *prog_words, uint32_t *tgt, size_t tgt_cap, size_t *n_tgt, uint32_t *con,
                              size_t con_cap, size_t *n_con) {
  if (!table || words < (size_t)pmt::HEADER_WORDS || table[pmt::H_MAGIC] != pmt::MAGIC || table[pmt::H_WORDS] != words)
    return -1;
  std::vector<uint32_t> T(table, table + words), out;
  std::vector<uint4> targets, contrib;
  if (!build_k2_program(T, 0, out, targets, contrib)) return -1;
  *prog_words = out.size();
  *n_tgt = targets.size();
  *n_con = contrib.size();
  if (out.size() > prog_cap || targets.size() > tgt_cap || contrib.size() > con_cap) return 1;
  std::memcpy(prog, out.data(), out.size() * 4);
  std::memcpy(tgt, targets.data(), targets.size() * 16);
  std::memcpy(con, contrib.data(), contrib.size() * 16);
  return 0;
}

pm_status ctx_plan_k2(pm_ctx *c, const int32_t *tables, const int32_t *var_off, int T, const int64_t *pt_off,
                      Plan **out) {
  if (var_off[0] != 0 || pt_off[0] != 0) return pm_set_error(PM_ERR_INVALID_ARG, "offsets must start at 0");
  for (int t = 0; t < T; t++) {
    if (var_off[t + 1] < var_off[t] || pt_off[t + 1] < pt_off[t])
      return pm_set_error(PM_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (var_off[t + 1] - var_off[t] > 65536)
      return pm_set_error(PM_ERR_INVALID_ARG, "at most 65,536 variants per template");
  }
  const int nv = var_off[T];
  const int64_t np = pt_off[T];
  if (np > (int64_t(1) << 31) - 64) return pm_set_error(PM_ERR_INVALID_ARG, "too many points");
  std::string key;
  key.append((const char *)&T, sizeof T);
  key.append((const char *)tables, sizeof(int32_t) * nv);
  key.append((const char *)var_off, sizeof(int32_t) * (T + 1));
  key.append((const char *)pt_off, sizeof(int64_t) * (T + 1));
  auto it = c->plans.find(key);
  if (it != c->plans.end()) { *out = it->second; return PM_OK; }

  std::vector<int64_t> off(nv);
  std::vector<uint32_t> prog;                                   // K2 programs of the distinct tables
  std::vector<uint4> targets, contrib;                          // their weight-fill recipes
  std::map<int, std::pair<uint32_t, uint32_t>> prog_of;         // table id -> (word offset, words)
  std::vector<int32_t> nparams(T, 0);
  std::vector<double> tw(T, 0);
  std::vector<int4> box(2 * T, make_int4(0, 0, 0, 0));
  for (int t = 0; t < T; t++) {
    for (int v = var_off[t]; v < var_off[t + 1]; v++) {
      int id = tables[v];
      if (id < 0 || id >= (int)c->tables.size()) return pm_set_error(PM_ERR_NOT_FOUND, "unknown table id");
      const auto &w = c->tables[id];
      if ((int)w[pmt::H_K] != 32) return pm_set_error(PM_ERR_INVALID_ARG, "fused ranking needs PM_LAYOUT_32 tables");
      if (v == var_off[t]) nparams[t] = (int)w[pmt::H_NPARAMS];
      else if (nparams[t] != (int)w[pmt::H_NPARAMS])
        return pm_set_error(PM_ERR_INVALID_ARG, "variants of one template differ in parameter count");
      if ((int)w[pmt::H_WORDS] > pmd::k2_table_words())
        return pm_set_error(PM_ERR_UNSUPPORTED, "fused ranking needs tables of at most " +
                                                    std::to_string(pmd::k2_table_words() * 4) + " bytes");
      int4 lo = make_int4((int)w[pmt::H_BOX_LO], (int)w[pmt::H_BOX_LO + 1], (int)w[pmt::H_BOX_LO + 2],
                          (int)w[pmt::H_BOX_LO + 3]);
      int4 hi = make_int4((int)w[pmt::H_BOX_HI], (int)w[pmt::H_BOX_HI + 1], (int)w[pmt::H_BOX_HI + 2],
                          (int)w[pmt::H_BOX_HI + 3]);
      if (v == var_off[t]) { box[2 * t] = lo; box[2 * t + 1] = hi; }
      else if (std::memcmp(&box[2 * t], &lo, sizeof lo) || std::memcmp(&box[2 * t + 1], &hi, sizeof hi))
        return pm_set_error(PM_ERR_UNSUPPORTED, "variants of one template must share one parameter box");
      auto pit = prog_of.find(id);
      if (pit == prog_of.end()) {
        std::vector<uint32_t> pw;
        const uint32_t base = (uint32_t)prog.size();
        if (!build_k2_program(w, base, pw, targets, contrib))
          return pm_set_error(PM_ERR_INVALID_ARG, "malformed table");
        if ((int)pw.size() > pmd::k2_table_words())
          return pm_set_error(PM_ERR_UNSUPPORTED, "fused ranking needs tables whose program fits " +
                                                      std::to_string(pmd::k2_table_words() * 4) + " bytes");
        prog.insert(prog.end(), pw.begin(), pw.end());
        pit = prog_of.emplace(id, std::make_pair(base, (uint32_t)pw.size())).first;
      }
      off[v] = (int64_t)((uint64_t)pit->second.first | ((uint64_t)pit->second.second << 40));
      tw[t] += table_work(w);
    }
  }
  // Point chunks of 32 (one point per lane); each chunk's variants are cut into S slices
  // of about SLICE_VARIANTS so that work units stay small; units are ordered most
  // expensive first (longest processing time first).
  std::vector<int32_t> slices(T, 1);
  for (int t = 0; t < T; t++) {
    int nvt = var_off[t + 1] - var_off[t];
    slices[t] = std::max(1, std::min(pmd::K2_MAX_SLICES, (nvt + SLICE_VARIANTS - 1) / SLICE_VARIANTS));
  }
  struct U { int chunk, slice, vb, ve; double cost; };
  std::vector<int4> chunks;
  std::vector<U> units;
  double total_work = 0;
  int64_t evals = 0;
  int slots = 0;
  for (int t = 0; t < T; t++) {
    const int nvt = var_off[t + 1] - var_off[t];
    const int S = slices[t];
    const int L = std::max(1, (nvt + S - 1) / S);
    for (int64_t p = pt_off[t]; p < pt_off[t + 1]; p += UNIT_POINTS) {
      const int n = (int)std::min<int64_t>(UNIT_POINTS, pt_off[t + 1] - p);
      const int c = (int)chunks.size();
      chunks.push_back(make_int4(t, (int)p, n, slots));
      slots += S;
      for (int s = 0; s < S; s++) {
        int vb = var_off[t] + std::min(nvt, s * L), ve = var_off[t] + std::min(nvt, (s + 1) * L);
        double per = nvt ? tw[t] / nvt : 0;
        units.push_back({c, s, vb, ve, per * (ve - vb) * n});
      }
      total_work += tw[t] * n;
      evals += (int64_t)nvt * n;
    }
  }
  std::stable_sort(units.begin(), units.end(), [](const U &a, const U &b) { return a.cost > b.cost; });
  std::vector<int4> hu(units.size());
  for (size_t i = 0; i < units.size(); i++) hu[i] = make_int4(units[i].chunk, units[i].slice, units[i].vb, units[i].ve);

  Plan *p = new Plan();
  auto alloc = [&](const void *h, size_t bytes, void **d) -> pm_status {
    CU(cudaMalloc(d, std::max<size_t>(bytes, 16)));
    p->dev.push_back(*d);
    if (h) CU(cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice));
    return PM_OK;
  };
  void *d;
  pm_status s;
  if ((s = alloc(off.data(), off.size() * 8, &d))) return s;
  p->d_tab_off = (const uint64_t *)d;
  if ((s = alloc(prog.data(), prog.size() * 4, &d))) return s;
  p->d_prog = (uint32_t *)d;
  if ((s = alloc(targets.data(), targets.size() * sizeof(uint4), &d))) return s;
  p->d_targets = (const uint4 *)d;
  if ((s = alloc(contrib.data(), contrib.size() * sizeof(uint4), &d))) return s;
  p->d_contrib = (const uint4 *)d;
  p->n_targets = (int)targets.size();
  if ((s = alloc(var_off, sizeof(int32_t) * (T + 1), &d))) return s;
  p->d_var_off = (const int32_t *)d;
  if ((s = alloc(nparams.data(), sizeof(int32_t) * T, &d))) return s;
  p->d_nparams = (const int32_t *)d;
  if ((s = alloc(slices.data(), sizeof(int32_t) * T, &d))) return s;
  p->d_slices = (const int32_t *)d;
  if ((s = alloc(box.data(), sizeof(int4) * box.size(), &d))) return s;
  p->d_box = (const int4 *)d;
  if ((s = alloc(chunks.data(), sizeof(int4) * chunks.size(), &d))) return s;
  p->d_chunks = (const int4 *)d;
  if ((s = alloc(hu.data(), sizeof(int4) * hu.size(), &d))) return s;
  p->d_units = (const int4 *)d;
  if ((s = alloc(nullptr, sizeof(int) * (chunks.size() + 1), &d))) return s;
  p->d_counter = (int *)d;  // [0] unit counter, [1..] per-chunk slice counters
  const size_t part = (size_t)slots * 16 * UNIT_POINTS;
  if ((s = alloc(nullptr, part * 8, &d))) return s;
  p->d_part_k = (int64_t *)d;
  p->n_chunks = (int)chunks.size();
  p->n_units = (int)hu.size();
  p->n_templates = T;
  p->total_points = np;
  p->total_evals = evals;
  p->work_per_eval = evals ? total_work / (double)evals : 0;
  p->nw = K2_WARPS;
  int bps = pmd::k2_max_blocks_per_sm(p->nw);
  p->grid = std::max(1, c->n_sms * std::max(1, bps));
  c->plans[key] = p;
  *out = p;
  return PM_OK;
}

static pm_status launch_k2(pm_ctx *c, Plan *p, const int64_t *pts, const double *w, int topk, int32_t *idx,
                           double *t, cudaStream_t st, int nw, int grid) {
  CU(cudaMemsetAsync(p->d_counter, 0, sizeof(int) * (p->n_chunks + 1), st));
  CU(pmd::launch_k2_weights(p->d_prog, p->d_targets, p->d_contrib, p->n_targets, w, st));
  pmd::K2Args a;
  a.prog = p->d_prog;
  a.tab_off = p->d_tab_off;
  a.var_off = p->d_var_off;
  a.tmpl_nparams = p->d_nparams;
  a.tmpl_slices = p->d_slices;
  a.tmpl_box = p->d_box;
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
  CU(pmd::launch_eval_predict_topk(a, nw, grid, st));
  return PM_OK;
}

// Launch-shape tuning: time each candidate (warps per CTA x CTAs per SM) on the
// caller's own inputs and keep the fastest.  Results are cached per plan and,
// when PM_TUNE_CACHE names a file, persisted by workload signature.
static std::string plan_signature(const Plan *p) {
  std::ostringstream o;
  o << "T" << p->n_templates << "_P" << p->total_points << "_E" << p->total_evals << "_W"
    << (int)(p->work_per_eval + 0.5);
  return o.str();
}

static bool tune_lookup(const std::string &path, const std::string &sig, int *nw, int *bps) {
  if (path.empty()) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    char s[256];
    int a, b;
    if (sscanf(line.c_str(), " \"%255[^\"]\": [%d, %d]", s, &a, &b) == 3 && sig == s) {
      *nw = a;
      *bps = b;
      return true;
    }
  }
  return false;
}

static void tune_store(const std::string &path, const std::string &sig, int nw, int bps) {
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
  o << "  \"" << sig << "\": [" << nw << ", " << bps << "]";
  lines.push_back(o.str());
  std::ofstream f(path);
  f << "{\n";
  for (size_t i = 0; i < lines.size(); i++) f << lines[i] << (i + 1 < lines.size() ? ",\n" : "\n");
  f << "}\n";
}

static pm_status tune_k2(pm_ctx *c, Plan *p, const int64_t *pts, const double *w, int topk, int32_t *idx, double *t,
                         cudaStream_t st) {
  std::string sig = plan_signature(p);
  int nw, bps;
  if (tune_lookup(c->tune_path, sig, &nw, &bps)) {
    p->nw = nw;
    p->grid = c->n_sms * bps;
    p->tuned = true;
    return PM_OK;
  }
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int bnw = p->nw, bgrid = p->grid, bbps = 1;
  for (int cand_nw : {K2_WARPS}) {
    int mx = std::max(1, pmd::k2_max_blocks_per_sm(cand_nw));
    for (int cand_bps = 1; cand_bps <= mx; cand_bps++) {
      int grid = c->n_sms * cand_bps;
      pm_status s = launch_k2(c, p, pts, w, topk, idx, t, st, cand_nw, grid);  // warm-up
      if (s) return s;
      CU(cudaEventRecord(e0, st));
      for (int r = 0; r < 2; r++) {
        s = launch_k2(c, p, pts, w, topk, idx, t, st, cand_nw, grid);
        if (s) return s;
      }
      CU(cudaEventRecord(e1, st));
      CU(cudaEventSynchronize(e1));
      float ms = 0;
      CU(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; bnw = cand_nw; bgrid = grid; bbps = cand_bps; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->nw = bnw;
  p->grid = bgrid;
  p->tuned = true;
  tune_store(c->tune_path, sig, bnw, bbps);
  return PM_OK;
}

pm_status ctx_run_k2(pm_ctx *c, Plan *p, const int64_t *pts, const double *w, int topk, int32_t *idx, double *t,
                     cudaStream_t st) {
  if (c->tune && !p->tuned) {
    pm_status s = tune_k2(c, p, pts, w, topk, idx, t, st);
    if (s) return s;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st) CU(cudaStreamIsCapturing(st, &cs));
  if (!st || cs != cudaStreamCaptureStatusNone) return launch_k2(c, p, pts, w, topk, idx, t, st, p->nw, p->grid);
  const void *key[6] = {pts, w, idx, t, p->d_prog, st};
  bool same = p->graph_exec && p->g_topk == topk && p->g_nw == p->nw && p->g_grid == p->grid &&
              std::memcmp(key, p->g_key, sizeof key) == 0;
  if (!same) {
    if (p->graph_exec) { cudaGraphExecDestroy(p->graph_exec); p->graph_exec = nullptr; }
    cudaGraph_t g;
    CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    pm_status s = launch_k2(c, p, pts, w, topk, idx, t, st, p->nw, p->grid);
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
                                  const int64_t *pt_off, int64_t *out /*[6]*/) {
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  Plan *p;
  pm_status s = ctx_plan_k2(c, tables, var_off, n_templates, pt_off, &p);
  if (s) return s;
  out[0] = p->n_units;
  out[1] = p->total_evals;
  out[2] = (int64_t)(p->work_per_eval * 1000);
  out[3] = p->nw;
  out[4] = p->grid;
  out[5] = p->tuned;
  return PM_OK;
}
