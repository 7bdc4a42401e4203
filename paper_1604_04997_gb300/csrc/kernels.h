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

// Fused ranking (rank.cu).  A ranking group's image (32-bit words, 16-byte aligned
// sections; built by plan.cpp):
//   header [HDR_WORDS]: basis entries B, dependency levels, conditions, image words,
//     the end of each level (entries are ordered by level), section offsets;
//   basis definitions, 8 words each: [a0 a1 a2 a3 | b c magic kind] for an atom
//     floor((a . n + b) / c) (kind = 2 | shift << 8 | numerator-may-be-negative << 16),
//     [i j . . | . . . kind] for a parameter (kind 0, i = its index), the constant
//     (kind 1) or a product of entries i and j (kind 3);
//   conditions (at most 64): [n_terms, const_lo, const_hi, (entry, coef_lo, coef_hi) *
//     n_terms], bit q of a point's two mask words when const + sum coef * value >= 0:
//     the tables' piece conditions and the signs of undecided post-op differences A - B;
//   programs (one per distinct table), as records of four words:
//     condition node [1 | n << 8 | piece records << 16, condition ids 0-4 (6 bits each),
//       ids 5-9, LUT offset]: the LUT byte of the n condition bits names a piece record;
//     sub node [2 | n << 8, condition ids, children, 0]: child record = children + 4 * bits;
//     leaf [n64 << 8 | n32 << 16 | nwide << 24, term records, denominator block or 0,
//       constant present]: term records are the constant's 128-bit weight (if present),
//       then [w0 w1 w2 entry] per term with a 96-bit weight (n64 terms whose basis value
//       may leave [0, 2^32), then n32 terms), then [w0 w1 w2 w3][entry 0 0 0] per term
//       with a 128-bit weight; the denominator block is [shift, 0, 0, 0, d^-1 mod 2^128];
//   the walk order: variants sorted by program shape (every leaf of a program is padded
//     to one count of 64-bit- and of 32-bit-class terms): per position its program's
//     root record offset and its variant index in the group (16 bits each), and runs
//     [shape = n64 | n32 << 8 (0xFFFF: 128-bit weights), first position, count, 0].
struct RankLayout {
  static constexpr int POINTS = 32;   // points per work unit: one per lane
  enum { H_B = 0, H_NLEV = 1, H_NCOND = 2, H_WORDS = 3, H_LEVEL_END = 4, H_OFF_BASIS = 12, H_OFF_COND = 13,
         H_OFF_VARMAP = 14, H_OFF_VIDMAP = 15, H_OFF_RUNS = 16, H_NRUNS = 17, HDR_WORDS = 20 };
};
struct RankArgs {
  const uint32_t *img;         // every group's image (weights filled per call)
  const int4 *groups;          // [n_groups][2]: (image word offset, image words, first variant
                               //   (template-relative), variants), (template, group index in template, 0, 0)
  const int4 *tmpl;            // [T][3]: (parameters, groups, 0, 0), box lo, box hi
  const int4 *chunks;          // [n_chunks] (template, first point, point count <= 32, first partial slot or -1)
  const int2 *units;           // [n_units] (chunk, group or -1 for a template without variants), schedule order
  int n_units;
  int *unit_counter;           // reset to 0 before each launch
  int *chunk_count;            // [n_chunks] groups finished, reset to 0 before each launch
  int64_t *part_k;             // [slots][16][32] partial lists of chunks with several groups
  const int64_t *points;       // [total][4]
  const double *w;             // [32]
  int topk;
  int32_t *top_idx;            // [total][topk]
  double *top_t;               // [total][topk]
  int *status;
  int img_words, basis_cap;    // shared-memory layout: the largest image and basis of the plan
};
cudaError_t launch_rank(const RankArgs &args, int nw, int grid, cudaStream_t st);
int rank_max_blocks_per_sm(int nw, int img_words, int basis_cap);
// fill the 128-bit term weights of the ranking programs from w (fp64 [32])
cudaError_t launch_k2_weights(uint32_t *prog, const uint4 *targets, const uint4 *contrib, int n_targets,
                              const double *w, cudaStream_t st);

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
cudaError_t launch_fit(const int64_t *F, int64_t R, int k, const double *T, int M, int objective, int gram,
                       int steps, void *scratch, double *W_out, FitHost *host, int *status, cudaStream_t st);
// exact tensor-core Gram matrices of the fit (adds into G, upper triangle, [M][32][32])
// gram: 0 float-float (k_gram), 1 three bf16 terms on the tensor cores, 2 exact bf16 digits
cudaError_t launch_gram_tc(const float *Uh, const float *Ul, const float2 *rf, int64_t R, int k, int M,
                           const unsigned *amax, double *G, int exact, int *status, cudaStream_t st);

}  // namespace pmd
