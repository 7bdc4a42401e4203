/* pm.h -- C ABI of the GB300 implementation of the linear kernel run-time model
 * of Stevens & Kloeckner, "A Unified, Hardware-Fitted, Cross-GPU Performance
 * Model" (arXiv:1604.04997).
 *
 *   T_wall(n) ~= sum_i alpha_i p_i(n)                                  (Sec. 2)
 *
 * p_i(n) are kernel properties (operation counts by category), piecewise
 * quasi-polynomials in the size parameters n, compiled once from a kernel
 * description and then re-evaluated cheaply for many n (Sec. 2, Sec. 3.2,
 * Alg. 1-2).  alpha_i are per-device weights fitted from measurement-kernel
 * timings by least squares on relative error (Sec. 4.3).
 *
 * Conventions for every entry point:
 *   - Return value: PM_OK (0) on success, a negative PM_ERR_* code on error,
 *     or a positive code for warnings / pending work.  Nothing aborts or exits.
 *     pm_last_error() describes the last failure of the calling thread.
 *   - Arguments named d_* are DEVICE pointers (cudaMalloc'd or torch tensors on
 *     the context's device), h_* are HOST pointers.  The caller owns all of them;
 *     the library never frees or retains them after the call's stream work ends.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work is enqueued on it; calls return without synchronising
 *     unless stated otherwise.  Argument checks run on the host before launch.
 *   - Device-side errors (e.g. a parameter point outside the declared box) are
 *     recorded in a context status word; pm_sync_status() reads and clears it.
 *   - A context is used by one host thread at a time, except pm_serve_submit,
 *     pm_serve_poll and pm_serve_stats, which any number of threads may call while
 *     the serve loop runs (and pm_compile_counts, which may run beside them).
 */
#ifndef PM_H
#define PM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pm_ctx pm_ctx;
typedef int32_t pm_status;

#define PM_OK 0
#define PM_ERR_INVALID_ARG -1
#define PM_ERR_PARSE -2           /* malformed kernel description */
#define PM_ERR_UNSUPPORTED -3     /* a form the counter does not cover (coupled guards without a
                                      unit-coefficient index, degree > 4, > 10 piece conditions ...) */
#define PM_ERR_OVERFLOW_RANGE -4  /* a count or atom could leave int64/int32 inside the declared box */
#define PM_ERR_NOMEM -5
#define PM_ERR_BUSY -6            /* serve: request can never fit the memory budget */
#define PM_ERR_TIMEOUT -7
#define PM_ERR_CUDA -8
#define PM_ERR_OUT_OF_BOX -9      /* device: a parameter point lies outside its table's box */
#define PM_ERR_NOT_FOUND -10
#define PM_WARN_RANK_DEFICIENT 1  /* fit: some model had a rank-deficient system */
#define PM_PENDING 2              /* serve: request not finished yet */

#define PM_LAYOUT_12 12           /* 12 aggregated feature columns */
#define PM_LAYOUT_32 32           /* 32 feature columns */

#define PM_PREC_FP64 0            /* FP64-accurate (exact fixed-point products, 128-bit sums) */
#define PM_PREC_BF16X3 1          /* three-term bf16 split on tensor cores, FP32 accumulate */
#define PM_PREC_NATIVE_FP64 2     /* plain double FMA (cross-check path) */

#define PM_FIT_RELATIVE 0         /* minimise sum_j (1 - F_j w / t_j)^2 (Sec. 4.3) */
#define PM_FIT_ABSOLUTE 1         /* minimise sum_j (t_j - F_j w)^2 */

#define PM_MAX_PARAMS 4
#define PM_MAX_TOPK 16

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  mem_budget_bytes bounds the device
 * memory the serve loop may hold for queries (0 = 16 GiB). */
pm_status pm_create(pm_ctx **out, int device, size_t mem_budget_bytes);
void pm_destroy(pm_ctx *ctx);
/* Thread-local description of the calling thread's last error; valid until its next call. */
const char *pm_last_error(void);
/* Wait for `stream`, then read and clear the device status word (PM_OK or a PM_ERR_*). */
pm_status pm_sync_status(pm_ctx *ctx, void *stream);

/* ------------------------------------------------------------------ counting (Sec. 3.2) */

typedef struct {
  int32_t n_params;     /* size parameters of the kernel (<= 4) */
  int32_t n_atoms;      /* floor((a.n + b)/c) atoms beyond the parameters */
  int32_t n_conds;      /* piece-selecting conditions */
  int32_t n_pieces;     /* distinct quasi-polynomial pieces */
  int32_t n_monomials;  /* monomials over all pieces */
  int32_t n_columns;    /* feature columns (12 or 32) */
  int32_t n_words;      /* table size in 32-bit words */
  int32_t degree;       /* largest monomial degree */
} pm_table_info;

/* Compile the operation counts of one kernel, written in the affine loop-nest
 * IR (`ir`, `len` bytes, not necessarily NUL-terminated), into a table of
 * piecewise quasi-polynomials valid on the parameter box
 * param_lo[i] <= n_i <= param_hi[i] (host arrays of n_params entries).
 * Implements Alg. 1 (n_ops = sum_i |pi_i(D_i)| n_ops,i) with exact point counting
 * (per-axis intervals; coupled domains such as j <= i or bands by index elimination
 * with closed-form power sums, giving a table denominator), the access
 * categorisation of Sec. 2.1 (size, direction, amortized stride fraction via the
 * footprint of Alg. 2) and the min(loads, stores) property.  The table stays
 * resident in the context (host and device).
 * Errors: PM_ERR_PARSE, PM_ERR_UNSUPPORTED, PM_ERR_OVERFLOW_RANGE, PM_ERR_INVALID_ARG. */
pm_status pm_compile_counts(pm_ctx *ctx, const char *ir, size_t len, int32_t layout,
                            const int64_t *h_param_lo, const int64_t *h_param_hi,
                            int32_t *out_table_id, pm_table_info *out_info);

/* Register a table from its image (h_words, n_words 32-bit words, as pm_table_image
 * wrote it), e.g. one saved earlier, without compiling the IR again; *out_table_id
 * receives its id in this context.  The image is checked on the host before anything
 * reaches the device: header limits, every section offset inside the image, condition
 * terms, the piece table, product operands, entry slots and columns, post-op holds,
 * the atoms' divisors and magic numbers and their int32 numerator range over the
 * declared box, and the denominator's inverse.  PM_ERR_INVALID_ARG (with the failed
 * check in pm_last_error) for an image that fails.  The counts are those of the
 * compiled table the image came from. */
pm_status pm_table_load(pm_ctx *ctx, const uint32_t *h_words, size_t n_words, int32_t *out_table_id);

/* Copy the host image of a compiled table (n_words 32-bit words) into h_buf. */
pm_status pm_table_image(pm_ctx *ctx, int32_t table_id, uint32_t *h_buf, size_t cap_words,
                         size_t *out_words);

/* Evaluate the counts of n_tables tables (h_table_ids, host) at n_points
 * parameter points: d_points int64 [n_points][P] (P = the tables' common
 * parameter count), d_counts int64 [n_tables][n_points][k] (k = the tables'
 * common layout).  Exact int64 (Sec. 2: p_i re-evaluated for changed n).
 * n_points <= 2^37; any number of tables (launched 65,535 at a time).
 * A point outside a table's box yields zeros and sets PM_ERR_OUT_OF_BOX. */
pm_status pm_eval_counts(pm_ctx *ctx, const int32_t *h_table_ids, int32_t n_tables,
                         const int64_t *d_points, int64_t n_points, int64_t *d_counts, void *stream);

/* ------------------------------------------------------------------ prediction (Sec. 2) */

/* d_T[r][m] = sum_i d_F[r][i] * d_W[m][i]   (F int64 [R][k], W fp64 [M][k], T fp64 [R][M]).
 * precision PM_PREC_FP64: weights rounded to fixed point per model (W = round(w 2^E),
 *   E the largest with sum_i |W_i| <= 2^62), products and sums exact in 128 bits for
 *   any int64 F: error <= 2^-62 (sum_i|W_mi| / min_i|W_mi|) sum_i |F_ri W_mi| plus
 *   2^-56 |T|, e.g. 4e-11 of sum_i |F_ri W_mi| for weights spread like Table 2's;
 * PM_PREC_BF16X3: <= ~1e-6 of the same (tensor cores, power-of-two column scaling);
 *   needs k == 32, M <= 64 and d_F 16-byte aligned (else PM_ERR_INVALID_ARG);
 * PM_PREC_NATIVE_FP64: double FMA. */
pm_status pm_predict(pm_ctx *ctx, const int64_t *d_F, int64_t R, int32_t k, const double *d_W,
                     int32_t M, int32_t precision, double *d_T, void *stream);

/* Per-model argmin over rows (configuration selection, Sec. 6.1): d_arg int64 [M],
 * d_min fp64 [M]; ties broken by the smaller row index; R == 0 gives -1 and +inf.
 * Does not materialise T. */
pm_status pm_predict_argmin(pm_ctx *ctx, const int64_t *d_F, int64_t R, int32_t k,
                            const double *d_W, int32_t M, int32_t precision, int64_t *d_arg,
                            double *d_min, void *stream);

/* Top-k rows per (group, model) over materialised features (configuration selection,
 * Sec. 6.1: for each problem size, the variants with the smallest predicted time).
 * Group g consists of the positions [h_seg_off[g], h_seg_off[g+1]) (h_seg_off: host,
 * int64 [G+1], non-decreasing, h_seg_off[0] >= 0).  Position p names row d_rows[p]
 * (a device int64 list of at least h_seg_off[G] entries, owned by the caller; e.g.
 * the rows t * n_points + p of one point p of a [tables][points][k] counts array),
 * or row p itself when d_rows is NULL (then h_seg_off[G] <= R).
 * Out: d_top_idx int64 [G][M][topk] row indices and d_top_t fp64
 * [G][M][topk] times, ascending by (time, row); a group with fewer than topk rows
 * fills the rest with -1 and +inf.  The times are bit for bit those pm_predict writes
 * at PM_PREC_FP64 (the only precision accepted here); 1 <= topk <= 16, k <= 40,
 * M <= 64.  A listed row outside [0, R) is skipped and makes pm_sync_status return
 * PM_ERR_INVALID_ARG.  A row listed twice in a group may be returned twice.
 * Groups of more than 1,024 positions use context scratch memory (16 bytes per
 * (1,024 positions, model, k-entry)). */
pm_status pm_predict_topk(pm_ctx *ctx, const int64_t *d_F, int64_t R, int32_t k, const double *d_W,
                          int32_t M, int32_t precision, const int64_t *h_seg_off, int32_t G,
                          const int64_t *d_rows, int32_t topk, int64_t *d_top_idx, double *d_top_t,
                          void *stream);

/* Allocation-free variant of pm_predict_argmin (PM_PREC_FP64), for callers that
 * cannot allocate device memory: code running while another allocator owns the
 * GPU's memory, latency-critical loops that must not trigger cudaMalloc's implicit
 * synchronisation, or callers that have no pm_ctx (creating one allocates).  The
 * paper has no counterpart; this is a deployment convenience.
 * Its partial results live in a fixed 1 MiB device array inside the library, held
 * by every GPU that loads the library until the process exits; it needs no context
 * and calls no allocating routine.  d_F, d_W, d_arg, d_min as in pm_predict_argmin
 * (device pointers of the current device); k <= 40, M <= 64 (larger M is rejected
 * with PM_ERR_INVALID_ARG).  The first call on each device looks up the array's
 * device address with that device current, so make that first call before any
 * stream capture.  All calls share the one array: calls whose work overlaps on the
 * GPU (different streams, or different host threads) race and must be serialised by
 * the caller.  Each launch writes every partial entry before reading it, so no
 * clearing is needed between calls. */
pm_status pm_predict_argmin_static(const int64_t *d_F, int64_t R, int32_t k, const double *d_W, int32_t M,
                                   int64_t *d_arg, double *d_min, void *stream);

/* Batched tuning evaluation: for each template t (0..n_templates-1), its
 * variants are the tables h_tables[h_var_off[t] .. h_var_off[t+1]) and its
 * points are rows h_pt_off[t] .. h_pt_off[t+1] of d_points (int64 [total][4],
 * unused parameter slots ignored).  Every (variant, point) pair is evaluated,
 * predicted with the weights d_w (fp64 [32], PM_LAYOUT_32 tables) to FP64
 * accuracy, and the topk (<= 16) smallest predicted times per point are
 * returned, ordered by (time, variant index within the template).  The ranking is
 * on the exact fixed-point sums (weights as in pm_predict); a returned time keeps
 * 40 bits of its sum's mantissa (rounded toward -infinity), so its error is at most 2^-40 |t|
 * plus pm_predict's weight-rounding bound:
 * d_top_idx int32 [total][topk] (-1 if fewer variants), d_top_t fp64 [total][topk].
 * One persistent launch; the host-side schedule is built once per distinct
 * argument set and cached. */
pm_status pm_eval_predict_topk(pm_ctx *ctx, const int32_t *h_tables, const int32_t *h_var_off,
                               int32_t n_templates, const int64_t *d_points,
                               const int64_t *h_pt_off, const double *d_w, int32_t topk,
                               int32_t *d_top_idx, double *d_top_t, void *stream);

/* Launch-shape tuning of pm_eval_predict_topk.  When enabled, the first call of
 * each new argument set times the candidate shapes (warps per CTA x CTAs per SM)
 * on the caller's own buffers (the outputs are rewritten by the final run) and
 * keeps the fastest; with cache_path (host string or NULL) the choice is stored
 * in / read from that JSON file, keyed by the workload's size signature. */
pm_status pm_tune(pm_ctx *ctx, int32_t enable, const char *cache_path);

/* Schedule of a pm_eval_predict_topk argument set (built and cached if new):
 * h_out[0] work units, [1] (variant, point) evaluations, [2] algorithmic integer
 * operations per evaluation x 1000, [3] warps per CTA, [4] CTAs, [5] tuned,
 * [6] ranking groups (variants of one template sharing one basis of values),
 * [7] the tuned slice size (at most this many variants per group; 0 = unlimited).
 * h_out: host int64 [8]. */
pm_status pm_plan_info(pm_ctx *ctx, const int32_t *h_tables, const int32_t *h_var_off, int32_t n_templates,
                       const int64_t *h_pt_off, int64_t *h_out);
/* The autotuner's measurements for an argument set already planned and tuned:
 * rows (slice size, warps per CTA, CTAs per SM, ms per launch), h_out fp64 [cap][4].
 * Returns the number of rows (which may exceed cap), 0 if not tuned, -1 on bad args. */
int32_t pm_plan_tune_log(pm_ctx *ctx, const int32_t *h_tables, const int32_t *h_var_off, int32_t n_templates,
                         const int64_t *h_pt_off, double *h_out, int32_t cap);

/* ------------------------------------------------------------------ fit (Sec. 4.3) */

typedef struct {
  int32_t rank;          /* numerical rank of the column-scaled system */
  int32_t iters;         /* refinement steps taken */
  int32_t status;        /* 0 ok, 1 rank deficient, 2 refinement did not converge */
  int32_t n_dropped;     /* all-zero columns (weight 0) */
  double cond_est;       /* condition estimate of the scaled Gram matrix (diag ratio of its Cholesky factor, squared) */
  double rel_resid;      /* ||b - A w|| / ||b|| of the scaled system */
  double last_update;    /* relative size of the last refinement correction */
} pm_fit_report;

/* Fit M weight vectors at once: d_F int64 [R][k], d_T fp64 [R][M] (measured
 * times > 0), d_W_out fp64 [M][k], h_report [M] (host).  Each column of F is
 * scaled by a power of two; the Gram matrices A^T A are formed on the tensor cores
 * from three bf16 terms of every entry (24 significant bits) with FP32 accumulation
 * (precision PM_PREC_BF16X3), or with float-float products and compensated FP32 sums
 * (PM_PREC_FP64; about 2^-44 relative); the k x k systems are solved by FP64
 * Cholesky and refined with residuals from exact products (refine_steps, e.g. 3),
 * which recovers the accuracy of the three-term Gram when cond(A)^2 2^-24 is well
 * below one.  If after the steps some model's last correction is still above 1e-10
 * of its weights, or its factor lost rank, the PM_PREC_BF16X3 fit is repeated with a
 * Gram formed exactly on the tensor cores (a 47-bit fixed-point image of A in seven
 * bf16 digits).  Synchronises `stream` to fill h_report.
 * Returns PM_OK or PM_WARN_RANK_DEFICIENT. */
pm_status pm_fit_weights(pm_ctx *ctx, const int64_t *d_F, int64_t R, int32_t k, const double *d_T,
                         int32_t M, int32_t objective, int32_t precision, int32_t refine_steps,
                         double *d_W_out, pm_fit_report *h_report, void *stream);

/* ------------------------------------------------------------------ serving */

typedef struct {
  int32_t batch_interval_us;   /* longest a query waits for batch mates while the GPU is busy (e.g. 200) */
  int32_t n_streams;           /* compute streams that overlap batches (>= 1) */
  int32_t max_batch_queries;   /* queries per batch (<= 1024) */
  int32_t reserved;
} pm_serve_config;

/* One autotuner query: evaluate and rank n_cand (variant, point) candidates of
 * one template with the resident weights of model `model`.  h_tables[c] and
 * h_points[c][4] give candidate c.  Results go to the caller's host buffers
 * h_top_idx / h_top_t (topk entries, candidate index and time, ordered by
 * (time, candidate index)), which must stay valid until pm_serve_poll returns
 * something other than PM_PENDING. */
typedef struct {
  int32_t model;
  int32_t topk;
  int64_t n_cand;
  const int32_t *h_tables;
  const int64_t *h_points;
  int32_t *h_top_idx;
  double *h_top_t;
} pm_query;

/* Latency and volume of the queries completed since the last reset.  Latency runs
 * from pm_serve_submit to the moment the results are in the caller's buffers. */
typedef struct {
  int64_t n_queries;
  int64_t n_batches;
  int64_t n_candidates;
  double p50_us, p99_us, max_us, mean_us;
  int64_t n_rejected;   /* submissions refused with PM_ERR_BUSY (can never fit the budget) */
  int64_t h2d_bytes;    /* bytes copied host -> device by the launched batches */
  int64_t d2h_bytes;    /* bytes copied device -> host by the launched batches */
} pm_serve_stats_t;

/* Make the weights of n_models device models resident (h_W fp64 [n_models][32], finite).
 * PM_ERR_BUSY while the serve loop runs. */
pm_status pm_serve_set_weights(pm_ctx *ctx, const double *h_W, int32_t n_models);
/* Start the serve loop (a batching thread and a completion thread).  It holds
 * min(mem_budget, 1 GiB) of device memory and as much pinned host memory for the
 * queries in flight.  Queries are batched while the GPU is busy: a batch is launched
 * at once when no batch is in flight, otherwise when its oldest query has waited
 * batch_interval_us, max_batch_queries are queued or the batches in flight finish.
 * Queries are admitted in arrival order while they fit the free memory, so a small
 * budget queues them. */
pm_status pm_serve_start(pm_ctx *ctx, const pm_serve_config *cfg);
/* Queue a query (thread-safe).  Its tables must be PM_LAYOUT_32 tables of this
 * context; h_tables and h_points are read when its batch is formed, so they too stay
 * valid until pm_serve_poll returns something other than PM_PENDING.  n_cand == 0
 * completes at once with idx -1 and time +inf.  PM_ERR_BUSY if the query can never
 * fit the memory budget. */
pm_status pm_serve_submit(pm_ctx *ctx, const pm_query *q, uint64_t *ticket);
/* PM_PENDING, PM_OK (results written) or an error (PM_ERR_OUT_OF_BOX: some candidate
 * point lies outside its table's box; the others are still ranked and written);
 * waits at most timeout_us (0 = no wait).  A ticket is forgotten once it has
 * returned something other than PM_PENDING (then PM_ERR_NOT_FOUND). */
pm_status pm_serve_poll(pm_ctx *ctx, uint64_t ticket, int32_t timeout_us);
/* Counters and submit-to-completion latencies since the last reset (reset != 0 clears
 * them after reading).  max_us and mean_us are exact over every query since the reset.
 * The percentiles are exact over the first 4,194,304 queries since the reset and then
 * taken over a uniform random sample of that many of them, so a long-running server
 * holds at most 16 MB of latencies.  The percentiles are computed after the serve
 * lock is released, so a stats call does not stall admission. */
pm_status pm_serve_stats(pm_ctx *ctx, int32_t reset, pm_serve_stats_t *out);
/* Finish every queued and running query, then stop the threads and free the serve
 * memory.  Unpolled tickets stay pollable until the next pm_serve_start. */
pm_status pm_serve_stop(pm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
