// Host side of the C ABI: context, resident tables, argument checks, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "pm.h"
#include "pm_internal.h"
#include "pm_table.h"
#include "trace.h"

int pm_compile_table(const char *ir, size_t len, int layout, const int64_t *plo, const int64_t *phi,
                     std::vector<uint32_t> &words, int info[8], std::string &msg);

// Last error of the calling thread, in a fixed buffer (reporting an error allocates nothing).
static thread_local char g_err[512];

pm_status pm_set_error_c(pm_status code, const char *m) {
  size_t n = 0;
  while (m[n] && n < sizeof(g_err) - 1) { g_err[n] = m[n]; n++; }
  g_err[n] = 0;
  return code;
}

pm_status pm_set_error(pm_status code, const std::string &m) { return pm_set_error_c(code, m.c_str()); }

extern "C" const char *pm_last_error(void) { return g_err; }

#define CU(x)                                                                                          \
  do {                                                                                                 \
    cudaError_t e__ = (x);                                                                             \
    if (e__ != cudaSuccess) return pm_set_error(PM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e__)); \
  } while (0)

// ------------------------------------------------------------------------------------- context

pm_status ctx_device_guard(pm_ctx *c) {
  if (!c) return pm_set_error(PM_ERR_INVALID_ARG, "null context");
  if (c->device < 0) return pm_set_error(PM_ERR_INVALID_ARG, "host-only context has no device");
  CU(cudaSetDevice(c->device));
  return PM_OK;
}

extern "C" pm_status pm_create(pm_ctx **out, int device, size_t mem_budget_bytes) {
  if (!out) return pm_set_error(PM_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  std::unique_ptr<pm_ctx> c(new pm_ctx());
  c->device = device;
  c->budget = mem_budget_bytes ? mem_budget_bytes : (size_t(16) << 30);
  if (device >= 0) {
    int n = 0;
    CU(cudaGetDeviceCount(&n));
    if (device >= n) return pm_set_error(PM_ERR_INVALID_ARG, "no such device");
    CU(cudaSetDevice(device));
    CU(cudaMalloc(&c->d_status, sizeof(int)));
    CU(cudaMemset(c->d_status, 0, sizeof(int)));
    CU(cudaMallocHost(&c->h_status, sizeof(int)));
    CU(cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device));
  }
  *out = c.release();
  return PM_OK;
}

extern "C" void pm_destroy(pm_ctx *c) {
  if (!c) return;
  serve_destroy(c);
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &kv : c->dcache) cudaFree(kv.second);
    for (auto &kv : c->plans) {
      if (kv.second->graph_exec) cudaGraphExecDestroy(kv.second->graph_exec);
      for (void *p : kv.second->dev) cudaFree(p);
      delete kv.second;
    }
    cudaFree(c->arena);
    cudaFree(c->d_status);
    cudaFree(c->scratch);
    cudaFreeHost(c->h_status);
    if (c->fit_host) cudaFreeHost(c->fit_host);
  }
  delete c;
}

extern "C" pm_status pm_sync_status(pm_ctx *c, void *stream) {
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  cudaStream_t st = (cudaStream_t)stream;
  CU(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
  CU(cudaStreamSynchronize(st));
  int s = *c->h_status;
  if (s & pmd::ST_OUT_OF_BOX) return pm_set_error(PM_ERR_OUT_OF_BOX, "a parameter point lies outside its table's box");
  if (s & pmd::ST_BAD_TABLE) return pm_set_error(PM_ERR_INVALID_ARG, "malformed table reached the device");
  if (s & pmd::ST_TIMEOUT) return pm_set_error(PM_ERR_TIMEOUT, "a device wait ran out");
  if (s & pmd::ST_BAD_INPUT) return pm_set_error(PM_ERR_INVALID_ARG, "a timing is not positive and finite");
  if (s & pmd::ST_BAD_ROW) return pm_set_error(PM_ERR_INVALID_ARG, "a listed row lies outside [0, R)");
  return PM_OK;
}

// Device copy of a small host array, cached by content (schedules, offsets).
pm_status ctx_dcopy(pm_ctx *c, const void *h, size_t bytes, void **d) {
  std::string key((const char *)h, bytes);
  auto it = c->dcache.find(key);
  if (it != c->dcache.end()) { *d = it->second; return PM_OK; }
  if (c->dcache.size() > 4096) {
    CU(cudaDeviceSynchronize());
    for (auto &kv : c->dcache) cudaFree(kv.second);
    c->dcache.clear();
  }
  void *p = nullptr;
  CU(cudaMalloc(&p, std::max<size_t>(bytes, 16)));
  CU(cudaMemcpy(p, h, bytes, cudaMemcpyHostToDevice));
  c->dcache[key] = p;
  *d = p;
  return PM_OK;
}

pm_status ctx_scratch(pm_ctx *c, size_t bytes, void **d) {
  if (bytes > c->scratch_cap) {
    CU(cudaDeviceSynchronize());
    cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_cap = 0;
    CU(cudaMalloc(&c->scratch, bytes));
    c->scratch_cap = bytes;
  }
  *d = c->scratch;
  return PM_OK;
}

static pm_status upload_table(pm_ctx *c, int id) {
  const auto &w = c->tables[id];
  size_t need = c->arena_used + w.size();
  if (need > c->arena_cap) {
    size_t cap = std::max<size_t>(need * 2, size_t(1) << 20);
    uint32_t *na = nullptr;
    CU(cudaMalloc(&na, cap * 4));
    if (c->arena_used) CU(cudaMemcpy(na, c->arena, c->arena_used * 4, cudaMemcpyDeviceToDevice));
    CU(cudaDeviceSynchronize());
    cudaFree(c->arena);
    c->arena = na;
    c->arena_cap = cap;
  }
  CU(cudaMemcpy(c->arena + c->arena_used, w.data(), w.size() * 4, cudaMemcpyHostToDevice));
  c->dev_off[id] = (int64_t)c->arena_used;
  c->arena_used += w.size();
  return PM_OK;
}

// ------------------------------------------------------------------------------------- counting

// Upload the newly added table id (the last one) to the device arena; on failure the
// table is taken back out, so that no id refers to a table without device words.
static pm_status register_on_device(pm_ctx *c, int id) {
  if (c->device < 0) return PM_OK;
  pm_status s = ctx_device_guard(c);
  if (!s) s = upload_table(c, id);
  if (s) {
    c->tables.pop_back();
    c->dev_off.pop_back();
  }
  return s;
}

extern "C" pm_status pm_compile_counts(pm_ctx *c, const char *ir, size_t len, int32_t layout, const int64_t *lo,
                                       const int64_t *hi, int32_t *out_id, pm_table_info *info) {
  PM_TRACE("pm_compile_counts");
  if (!c || !ir || !lo || !hi || !out_id) return pm_set_error(PM_ERR_INVALID_ARG, "null argument");
  if (layout != PM_LAYOUT_12 && layout != PM_LAYOUT_32) return pm_set_error(PM_ERR_INVALID_ARG, "layout must be 12 or 32");
  std::vector<uint32_t> words;
  int inf[8];
  std::string msg;
  int rc = pm_compile_table(ir, len, layout, lo, hi, words, inf, msg);
  if (rc) return pm_set_error(rc, msg);
  std::lock_guard<std::mutex> lk(c->mu);
  int id = (int)c->tables.size();
  c->tables.push_back(std::move(words));
  c->dev_off.push_back(-1);
  if (pm_status u = register_on_device(c, id)) return u;
  *out_id = id;
  if (info) {
    info->n_params = inf[0]; info->n_atoms = inf[1]; info->n_conds = inf[2]; info->n_pieces = inf[3];
    info->n_monomials = inf[4]; info->n_columns = inf[5]; info->n_words = inf[6]; info->degree = inf[7];
  }
  return PM_OK;
}

bool pm_table_valid(const uint32_t *w, size_t n, std::string &why);   // table_check.cpp

extern "C" pm_status pm_table_load(pm_ctx *c, const uint32_t *words, size_t n_words, int32_t *out_id) {
  PM_TRACE("pm_table_load");
  if (!c || !words || !out_id) return pm_set_error(PM_ERR_INVALID_ARG, "null argument");
  std::string why;
  if (!pm_table_valid(words, n_words, why)) return pm_set_error(PM_ERR_INVALID_ARG, "table image rejected: " + why);
  std::lock_guard<std::mutex> lk(c->mu);
  int id = (int)c->tables.size();
  c->tables.emplace_back(words, words + n_words);
  c->dev_off.push_back(-1);
  if (pm_status u = register_on_device(c, id)) return u;
  *out_id = id;
  return PM_OK;
}

extern "C" pm_status pm_table_image(pm_ctx *c, int32_t id, uint32_t *buf, size_t cap, size_t *out_words) {
  if (!c || id < 0 || id >= (int)c->tables.size()) return pm_set_error(PM_ERR_NOT_FOUND, "no such table");
  const auto &w = c->tables[id];
  if (out_words) *out_words = w.size();
  if (buf) {
    if (cap < w.size()) return pm_set_error(PM_ERR_INVALID_ARG, "buffer too small");
    std::memcpy(buf, w.data(), w.size() * 4);
  }
  return PM_OK;
}

pm_status ctx_table_offsets(pm_ctx *c, const int32_t *ids, int n, int *P, int *K, const int64_t **d_off) {
  std::vector<int64_t> off(n);
  *P = -1;
  *K = -1;
  for (int i = 0; i < n; i++) {
    int id = ids[i];
    if (id < 0 || id >= (int)c->tables.size()) return pm_set_error(PM_ERR_NOT_FOUND, "unknown table id");
    const auto &w = c->tables[id];
    int p = (int)w[pmt::H_NPARAMS], k = (int)w[pmt::H_K];
    if (*P < 0) { *P = p; *K = k; }
    if (P && *P != p) return pm_set_error(PM_ERR_INVALID_ARG, "tables differ in parameter count");
    if (*K != k) return pm_set_error(PM_ERR_INVALID_ARG, "tables differ in layout");
    if (c->device >= 0 && c->dev_off[id] < 0) return pm_set_error(PM_ERR_INVALID_ARG, "table not on the device");
    off[i] = c->dev_off[id];
  }
  void *d = nullptr;
  pm_status s = ctx_dcopy(c, off.data(), off.size() * 8, &d);
  *d_off = (const int64_t *)d;
  return s;
}

extern "C" pm_status pm_eval_counts(pm_ctx *c, const int32_t *ids, int32_t n_tables, const int64_t *d_points,
                                    int64_t n_points, int64_t *d_counts, void *stream) {
  PM_TRACE("pm_eval_counts");
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (n_tables < 0 || n_points < 0 || (n_tables && !ids)) return pm_set_error(PM_ERR_INVALID_ARG, "bad sizes");
  if (n_tables == 0 || n_points == 0) return PM_OK;
  if (!d_points || !d_counts) return pm_set_error(PM_ERR_INVALID_ARG, "null device buffer");
  // the launch puts points on grid x (128 per block) and tables on grid y (at most 65,535)
  if (n_points > (int64_t(1) << 37)) return pm_set_error(PM_ERR_INVALID_ARG, "too many points");
  int P, K;
  const int64_t *d_off;
  pm_status s = ctx_table_offsets(c, ids, n_tables, &P, &K, &d_off);
  if (s) return s;
  constexpr int64_t MAX_GRID_Y = 65535;
  for (int64_t t0 = 0; t0 < n_tables; t0 += MAX_GRID_Y) {
    const int nt = (int)std::min<int64_t>(MAX_GRID_Y, n_tables - t0);
    CU(pmd::launch_eval_counts(c->arena, d_off + t0, nt, d_points, n_points, P, K,
                               d_counts + (int64_t)t0 * n_points * K, c->d_status, (cudaStream_t)stream));
  }
  return PM_OK;
}

// ------------------------------------------------------------------------------------- prediction

extern "C" pm_status pm_predict(pm_ctx *c, const int64_t *F, int64_t R, int32_t k, const double *W, int32_t M,
                                int32_t precision, double *T, void *stream) {
  PM_TRACE("pm_predict");
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (R < 0 || k <= 0 || M <= 0) return pm_set_error(PM_ERR_INVALID_ARG, "bad sizes");
  if (R == 0) return PM_OK;
  if (!F || !W || !T) return pm_set_error(PM_ERR_INVALID_ARG, "null device buffer");
  if (precision == PM_PREC_BF16X3) return pm_predict_bf16x3(c, F, R, k, W, M, T, nullptr, nullptr, stream);
  if (precision != PM_PREC_FP64 && precision != PM_PREC_NATIVE_FP64)
    return pm_set_error(PM_ERR_INVALID_ARG, "unknown precision");
  if (precision == PM_PREC_FP64 && (k > 40 || M > 64)) return pm_set_error(PM_ERR_INVALID_ARG, "k <= 40 and M <= 64");
  CU(pmd::launch_predict(F, R, k, W, M, precision, T, (cudaStream_t)stream));
  return PM_OK;
}

extern "C" pm_status pm_predict_argmin(pm_ctx *c, const int64_t *F, int64_t R, int32_t k, const double *W,
                                       int32_t M, int32_t precision, int64_t *arg, double *mn, void *stream) {
  PM_TRACE("pm_predict_argmin");
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (R < 0 || k <= 0 || k > 40 || M <= 0 || M > 64) return pm_set_error(PM_ERR_INVALID_ARG, "bad sizes");
  if ((!F && R > 0) || !W || !arg || !mn) return pm_set_error(PM_ERR_INVALID_ARG, "null device buffer");
  if (precision == PM_PREC_BF16X3) return pm_predict_bf16x3(c, F, R, k, W, M, nullptr, arg, mn, stream);
  if (precision != PM_PREC_FP64) return pm_set_error(PM_ERR_INVALID_ARG, "argmin supports PM_PREC_FP64 and PM_PREC_BF16X3");
  void *scr = nullptr;
  pm_status s = ctx_scratch(c, pmd::argmin_scratch_bytes(M, pmd::argmin_parts()), &scr);
  if (s) return s;
  CU(pmd::launch_predict_argmin(F, R, k, W, M, precision, scr, arg, mn, (cudaStream_t)stream));
  return PM_OK;
}

extern "C" pm_status pm_predict_topk(pm_ctx *c, const int64_t *F, int64_t R, int32_t k, const double *W, int32_t M,
                                     int32_t precision, const int64_t *h_seg_off, int32_t G, const int64_t *d_rows,
                                     int32_t topk, int64_t *d_top_idx, double *d_top_t, void *stream) {
  PM_TRACE("pm_predict_topk");
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (R < 0 || k <= 0 || k > 40 || M <= 0 || M > 64 || G < 0 || topk < 1 || topk > pmd::TOPK_MAX)
    return pm_set_error(PM_ERR_INVALID_ARG, "bad sizes (need 0 < k <= 40, 0 < M <= 64, G >= 0, 1 <= topk <= 16)");
  if (precision != PM_PREC_FP64) return pm_set_error(PM_ERR_INVALID_ARG, "pm_predict_topk supports PM_PREC_FP64");
  if (G == 0) return PM_OK;
  if (!h_seg_off || !W || !d_top_idx || !d_top_t || (!F && R > 0)) return pm_set_error(PM_ERR_INVALID_ARG, "null buffer");
  if (h_seg_off[0] < 0) return pm_set_error(PM_ERR_INVALID_ARG, "group offsets must start at 0 or above");
  for (int32_t i = 0; i < G; i++)
    if (h_seg_off[i + 1] < h_seg_off[i]) return pm_set_error(PM_ERR_INVALID_ARG, "group offsets must be non-decreasing");
  if (!d_rows && h_seg_off[G] > R) return pm_set_error(PM_ERR_INVALID_ARG, "without a row list the groups must lie in [0, R)");
  // work units: groups cut into chunks of TOPK_CHUNK positions; a one-chunk group
  // (an empty one too) is written directly, the others through partial lists
  std::vector<pmd::TopkUnit> units;
  std::vector<pmd::TopkMerge> merges;
  int64_t parts = 0;
  for (int32_t i = 0; i < G; i++) {
    const int64_t p0 = h_seg_off[i], p1 = h_seg_off[i + 1];
    const int64_t nch = std::max<int64_t>(1, (p1 - p0 + pmd::TOPK_CHUNK - 1) / pmd::TOPK_CHUNK);
    if (nch == 1) {
      units.push_back(pmd::TopkUnit{p0, p1, i, -1});
      continue;
    }
    if (parts + nch > INT32_MAX) return pm_set_error(PM_ERR_INVALID_ARG, "too many rows");
    merges.push_back(pmd::TopkMerge{i, (int32_t)parts, (int32_t)nch, 0});
    for (int64_t q = 0; q < nch; q++)
      units.push_back(pmd::TopkUnit{p0 + q * pmd::TOPK_CHUNK, std::min(p1, p0 + (q + 1) * pmd::TOPK_CHUNK), i,
                                    (int32_t)(parts + q)});
    parts += nch;
  }
  if (units.size() > (size_t)INT32_MAX) return pm_set_error(PM_ERR_INVALID_ARG, "too many groups");
  const size_t ub = units.size() * sizeof(pmd::TopkUnit), mb = merges.size() * sizeof(pmd::TopkMerge);
  std::vector<uint8_t> meta(ub + mb);
  std::memcpy(meta.data(), units.data(), ub);
  if (mb) std::memcpy(meta.data() + ub, merges.data(), mb);
  void *d_meta = nullptr, *scr = nullptr;
  pm_status s = ctx_dcopy(c, meta.data(), meta.size(), &d_meta);
  if (s) return s;
  const size_t pb = (size_t)parts * M * topk * sizeof(double);
  if (parts) {
    s = ctx_scratch(c, 2 * pb, &scr);
    if (s) return s;
  }
  CU(pmd::launch_predict_topk(F, R, k, W, M, d_rows, (const pmd::TopkUnit *)d_meta, (int)units.size(),
                              (const pmd::TopkMerge *)((uint8_t *)d_meta + ub), (int)merges.size(), topk,
                              (double *)scr, (int64_t *)((uint8_t *)scr + pb), d_top_idx, d_top_t, c->d_status,
                              (cudaStream_t)stream));
  return PM_OK;
}

// Tensor-core path (three-term bf16 split, FP32 accumulation): T, or per-model argmin.
pm_status pm_predict_bf16x3(pm_ctx *c, const int64_t *F, int64_t R, int k, const double *W, int M, double *T,
                            int64_t *arg, double *mn, void *stream) {
  if (k != 32 || M > 64) return pm_set_error(PM_ERR_INVALID_ARG, "PM_PREC_BF16X3 needs k == 32 and M <= 64");
  if ((uintptr_t)F % 16 != 0) return pm_set_error(PM_ERR_INVALID_ARG, "PM_PREC_BF16X3 needs F 16-byte aligned");
  void *scr = nullptr;
  if (arg) {
    pm_status s = ctx_scratch(c, pmd::tc_argmin_scratch_bytes(M, c->n_sms), &scr);
    if (s) return s;
  }
  CU(pmd::launch_predict_tc(F, R, k, W, M, T, arg, mn, scr, c->n_sms, c->d_status, (cudaStream_t)stream));
  return PM_OK;
}

// ------------------------------------------------------------------------------------- batched eval+predict+top-k

extern "C" pm_status pm_eval_predict_topk(pm_ctx *c, const int32_t *tables, const int32_t *var_off,
                                          int32_t n_templates, const int64_t *d_points, const int64_t *pt_off,
                                          const double *d_w, int32_t topk, int32_t *d_top_idx, double *d_top_t,
                                          void *stream) {
  PM_TRACE("pm_eval_predict_topk");
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (n_templates <= 0 || !tables || !var_off || !pt_off || !d_points || !d_w || !d_top_idx || !d_top_t)
    return pm_set_error(PM_ERR_INVALID_ARG, "null argument");
  if (topk < 1 || topk > PM_MAX_TOPK) return pm_set_error(PM_ERR_INVALID_ARG, "topk must be 1..16");
  Plan *plan = nullptr;
  pm_status s = ctx_plan_k2(c, tables, var_off, n_templates, pt_off, &plan);
  if (s) return s;
  return ctx_run_k2(c, plan, tables, var_off, pt_off, d_points, d_w, topk, d_top_idx, d_top_t, (cudaStream_t)stream);
}

// ------------------------------------------------------------------------------------- fit (Sec. 4.3)

extern "C" pm_status pm_fit_weights(pm_ctx *c, const int64_t *F, int64_t R, int32_t k, const double *T, int32_t M,
                                    int32_t objective, int32_t precision, int32_t refine_steps, double *W_out,
                                    pm_fit_report *rep, void *stream) {
  PM_TRACE("pm_fit_weights");
  pm_status g = ctx_device_guard(c);
  if (g) return g;
  if (R <= 0 || k <= 0 || k > 32 || M <= 0 || M > 64 || refine_steps < 0 || refine_steps > 50)
    return pm_set_error(PM_ERR_INVALID_ARG, "need R > 0, 0 < k <= 32, 0 < M <= 64, 0 <= refine_steps <= 50");
  if (!F || !T || !W_out || !rep) return pm_set_error(PM_ERR_INVALID_ARG, "null argument");
  if (objective != PM_FIT_RELATIVE && objective != PM_FIT_ABSOLUTE) return pm_set_error(PM_ERR_INVALID_ARG, "objective");
  if (precision != PM_PREC_FP64 && precision != PM_PREC_BF16X3) return pm_set_error(PM_ERR_INVALID_ARG, "precision");
  void *scr = nullptr;
  pm_status s = ctx_scratch(c, pmd::fit_scratch_bytes(R, k, M), &scr);
  if (s) return s;
  if (!c->fit_host) {
    CU(cudaMallocHost(&c->fit_host, 64 * (16 + 8 * 4)));
  }
  pmd::FitHost h;
  h.info = (int *)c->fit_host;
  h.ratio = (double *)((char *)c->fit_host + 64 * 16);
  h.upd = h.ratio + 64;
  h.rr = h.upd + 64;
  h.bb = h.rr + 64;
  cudaStream_t st = (cudaStream_t)stream;
  // PM_PREC_BF16X3: the Gram from three bf16 terms first; refinement with exact residuals
  // makes it accurate when cond(G) 2^-24 is well below one.  If some model's last
  // correction is still large (or its factor reports a rank drop the exact Gram may not
  // have), the fit is repeated with the exact digit Gram.
  int gram = precision == PM_PREC_BF16X3 ? 1 : 0;
  for (;;) {
    CU(pmd::launch_fit(F, R, k, T, M, objective, gram, refine_steps, scr, W_out, &h, c->d_status, st));
    CU(cudaStreamSynchronize(st));
    s = pm_sync_status(c, stream);
    if (s) return s;
    if (gram != 1 || refine_steps == 0) break;
    bool converged = true;
    for (int m = 0; m < M; m++) converged &= h.upd[m] < 1e-10 && h.info[m * 4 + 2] == 0;
    if (converged) break;
    gram = 2;
  }
  bool deficient = false;
  for (int m = 0; m < M; m++) {
    pm_fit_report &r = rep[m];
    r.rank = h.info[m * 4 + 0];
    r.n_dropped = h.info[m * 4 + 1];
    r.iters = refine_steps;
    r.cond_est = h.ratio[m];
    r.rel_resid = h.bb[m] > 0 ? std::sqrt(h.rr[m] / h.bb[m]) : 0.0;
    r.last_update = h.upd[m];
    r.status = h.info[m * 4 + 2] ? 1 : (refine_steps > 0 && !(r.last_update < 1e-6) ? 2 : 0);
    deficient |= h.info[m * 4 + 2] != 0;
  }
  return deficient ? PM_WARN_RANK_DEFICIENT : PM_OK;
}
