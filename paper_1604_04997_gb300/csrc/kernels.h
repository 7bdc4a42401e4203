// Launch interfaces between the host API layer and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pmd {

// bits of the device status word
enum StatusBits { ST_OUT_OF_BOX = 1, ST_BAD_TABLE = 2, ST_TIMEOUT = 4, ST_BAD_INPUT = 8, ST_BAD_ROW = 16 };

// K1 (eval.cu)
cudaError_t launch_eval_counts(const uint32_t *arena, const int64_t *d_tab_off, int n_tables, const int64_t *points,
                               int64_t n_points, int P, int K, int64_t *out, int *status, cudaStream_t st);

// K2 (eval.cu)
constexpr int K2_MAX_SLICES = 16;
struct K2Args {
  const uint32_t *prog;        // K2 programs: table words followed by the weight image
  const uint64_t *tab_off;     // [n_variants] word offset into prog | program words << 40
  const int32_t *var_off;      // [n_templates+1] CSR into tab_off
  const int32_t *tmpl_nparams; // [n_templates]
  const int32_t *tmpl_slices;  // [n_templates] variant slices S per point chunk (<= K2_MAX_SLICES)
  const int4 *tmpl_box;        // [n_templates][2] parameter box (lo, hi) shared by the template's tables
  const int4 *chunks;          // [n_chunks] (template, first point, point count <= 256, first partial slot)
  const int4 *units;           // [n_units] (chunk, slice, first variant, end variant), schedule order
  int n_units;
  int *unit_counter;           // reset to 0 before each launch
  int *chunk_count;            // [n_chunks] slices finished, reset to 0 before each launch
  int64_t *part_k;             // [slots][16][points per chunk] partial lists (packed entries) of chunks with S > 1
  const int64_t *points;       // [total][4]
  const double *w;             // [32]
  int topk;
  int32_t *top_idx;            // [total][topk]
  double *top_t;               // [total][topk]
  int *status;
};
cudaError_t launch_eval_predict_topk(const K2Args &args, int nw, int grid, cudaStream_t st);
// fill the 128-bit weights of the K2 programs from w (fp64 [32])
cudaError_t launch_k2_weights(uint32_t *prog, const uint4 *targets, const uint4 *contrib, int n_targets,
                              const double *w, cudaStream_t st);
int k2_max_blocks_per_sm(int nw);
int k2_table_words();
int k2_points_per_cta(int nw);

// predict.cu
struct ArgPart { double t; int64_t r; };   // a partial per-model minimum: time and row
// per-model minimum over n_part partials part[p][M] (smaller time, then smaller row);
// n_part == 0 gives -1 and +inf
cudaError_t launch_argmin_reduce(const ArgPart *part, int n_part, int M, int64_t *arg, double *mn, cudaStream_t st);
cudaError_t launch_predict(const int64_t *F, int64_t R, int k, const double *W, int M, int precision, double *T,
                           cudaStream_t st);
// argmin: per-model partial results go to scratch (n_part [M] (double, int64) pairs), then reduced.
size_t argmin_scratch_bytes(int M, int n_part);
int argmin_parts();
cudaError_t launch_predict_argmin(const int64_t *F, int64_t R, int k, const double *W, int M, int precision,
                                  void *scratch, int64_t *arg, double *mn, cudaStream_t st);

// top-k rows per (group, model): work units of at most TOPK_CHUNK positions of one
// group; a group of one unit is written directly (part < 0), the partial lists of the
// others ([part][M][topk]) are merged per group (TopkMerge)
constexpr int TOPK_MAX = 16;
constexpr int64_t TOPK_CHUNK = 1024;
struct TopkUnit { int64_t p0, p1; int32_t g, part; };
struct TopkMerge { int32_t g, part0, n_parts, pad; };
cudaError_t launch_predict_topk(const int64_t *F, int64_t R, int k, const double *W, int M, const int64_t *rows,
                                const TopkUnit *units, int n_units, const TopkMerge *merges, int n_merges, int topk,
                                double *part_t, int64_t *part_r, int64_t *top_idx, double *top_t, int *status,
                                cudaStream_t st);

// predict_tc.cu (tensor cores, three-term bf16 split)
int tc_parts(int sms);
size_t tc_argmin_scratch_bytes(int M, int sms);
cudaError_t launch_predict_tc(const int64_t *F, int64_t R, int k, const double *W, int M, double *T, int64_t *arg,
                              double *mn, void *scratch, int sms, int *status, cudaStream_t st);

// serve.cu: one batch of queries, all arrays inside one device region
constexpr int SV_MAX_TOPK = 16;
struct SQuery {               // 24 bytes
  int64_t begin;              // first candidate of the query in the batch
  int32_t n;                  // candidates
  int32_t model;              // row of models
  int32_t topk;               // 1..16
  int32_t pad;
};
struct ServeArgs {
  const uint32_t *arena;      // compiled tables
  const SQuery *queries;
  int n_queries;
  const int2 *blocks;         // per k_serve_eval CTA: (query, chunk of 128 candidates)
  const uint32_t *cand_off;   // [N] arena word offset of each candidate's table
  const int64_t *points;      // [N][4]
  const double *models;       // [n_models][32]
  int64_t *keys;              // [N] scratch
  int32_t *q_status;          // [n_queries] status bits
  int32_t *out_idx;           // [n_queries][16]
  double *out_t;              // [n_queries][16]
};
cudaError_t launch_serve(const ServeArgs &a, int n_blocks, cudaStream_t st);

// fit.cu
struct FitHost {            // pinned host buffers filled by the fit (per model)
  int *info;                // [M][4] rank, zero columns, rank deficient, dropped-direction mask
  double *ratio, *upd, *rr, *bb;
};
size_t fit_scratch_bytes(int64_t R, int k, int M);
cudaError_t launch_fit(const int64_t *F, int64_t R, int k, const double *T, int M, int objective, int precision,
                       int steps, void *scratch, double *W_out, FitHost *host, int *status, cudaStream_t st);
// exact tensor-core Gram matrices of the fit (adds into G, upper triangle, [M][32][32])
cudaError_t launch_gram_tc(const float *Uh, const float *Ul, const float2 *rf, int64_t R, int k, int M,
                           const unsigned *amax, double *G, int *status, cudaStream_t st);

}  // namespace pmd
