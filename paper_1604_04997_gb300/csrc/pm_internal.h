// Internal host-side state shared by the API translation units.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pm.h"

struct ServeState;

// Cached schedule of one pm_eval_predict_topk argument set.
struct Plan {
  std::vector<void *> dev;          // device allocations owned by the plan
  uint32_t *d_img = nullptr;        // ranking-group images (weights filled per call)
  const uint4 *d_targets = nullptr; // weight-fill recipe: (word, first contribution, count)
  const uint4 *d_contrib = nullptr; // contributions (column, -, coef lo, coef hi)
  int n_targets = 0;
  const int4 *d_groups = nullptr;
  const int4 *d_tmpl = nullptr;
  const int4 *d_chunks = nullptr;
  const int2 *d_units = nullptr;
  int *d_counter = nullptr;
  int64_t *d_part_k = nullptr;
  int n_units = 0, n_templates = 0, n_chunks = 0, n_groups = 0;
  int img_words = 0, basis_cap = 1;  // the largest group image and basis (shared-memory layout)
  int slice_max = 0;                 // at most this many variants per group
  int64_t total_points = 0, total_evals = 0;
  double work_per_eval = 0;          // algorithmic integer operations per evaluation
  int nw = 8, grid = 0;              // launch shape (autotuned when enabled)
  bool tuned = false;
  std::string key;
  std::vector<std::array<double, 4>> tune_log;   // (slice, warps, CTAs per SM, ms) per candidate
  // CUDA graph of the last argument set
  cudaGraphExec_t graph_exec = nullptr;
  const void *g_key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int g_topk = 0, g_nw = 0, g_grid = 0;
};

struct pm_ctx {
  int device = -1;
  int n_sms = 0;
  size_t budget = 0;
  std::mutex mu;
  std::vector<std::vector<uint32_t>> tables;  // host images
  std::vector<int64_t> dev_off;               // word offset of each table in the arena
  uint32_t *arena = nullptr;
  size_t arena_cap = 0, arena_used = 0;       // in words
  int *d_status = nullptr;
  int *h_status = nullptr;
  std::map<std::string, void *> dcache;
  std::map<std::string, Plan *> plans;
  void *scratch = nullptr;
  size_t scratch_cap = 0;
  int tune = 0;
  std::string tune_path;
  ServeState *serve = nullptr;
  double *d_models = nullptr;                 // resident weights [n_models][32]
  void *fit_host = nullptr;                   // pinned report buffers of the fit
  int n_models = 0;
};

pm_status pm_set_error(pm_status code, const std::string &m);
void serve_destroy(pm_ctx *c);   // stops the serve loop and frees its state and resident weights
pm_status pm_set_error_c(pm_status code, const char *m);
pm_status ctx_device_guard(pm_ctx *c);
pm_status ctx_dcopy(pm_ctx *c, const void *h, size_t bytes, void **d);
pm_status ctx_scratch(pm_ctx *c, size_t bytes, void **d);
pm_status ctx_table_offsets(pm_ctx *c, const int32_t *ids, int n, int *P, int *K, const int64_t **d_off);
pm_status ctx_plan_k2(pm_ctx *c, const int32_t *tables, const int32_t *var_off, int n_templates,
                      const int64_t *pt_off, Plan **out);
pm_status ctx_run_k2(pm_ctx *c, Plan *p, const int32_t *tables, const int32_t *var_off, const int64_t *pt_off,
                     const int64_t *d_points, const double *d_w, int topk, int32_t *d_idx, double *d_t,
                     cudaStream_t st);
pm_status pm_predict_bf16x3(pm_ctx *c, const int64_t *F, int64_t R, int k, const double *W, int M, double *T,
                            int64_t *arg, double *mn, void *stream);
