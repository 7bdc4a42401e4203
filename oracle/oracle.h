/* Oracle for the linear kernel run-time model of Stevens & Kloeckner,
 * "A Unified, Hardware-Fitted, Cross-GPU Performance Model" (arXiv:1604.04997).
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, slow CPU implementation exists to check
 * the CUDA library against the paper.  Only the tests, the smoke check and the
 * bench's CPU-baseline leg may load it; the product path never does.  It shares
 * no code with the library (its own parser, counters, layouts, arithmetic).
 *
 * What it computes:
 *   - per-kernel operation counts (Sec. 2, Alg. 1), by brute-force enumeration
 *     of every iteration-domain point (orc_count_brute) and by a numeric per-axis
 *     evaluator (orc_count_struct), which is pinned to the brute force;
 *   - the amortized stride fraction class of each global access (Sec. 2.1, Alg. 2);
 *   - the 12- and 32-column feature layouts incl. min(loads, stores) (Sec. 2.1);
 *   - predicted times T = sum_i alpha_i p_i (Sec. 2) with a compensated dot
 *     product (Ogita, Rump, Oishi, "Accurate sum and dot product", SISC 2005);
 *   - top-k ranking by (time, index);
 *   - the weight fit minimising sum_j (1 - sum_i alpha_i p_ij / T_j)^2 (Sec. 4.3)
 *     by Householder QR with column pivoting (Golub & Van Loan, Alg. 5.4.1).
 */
#ifndef PM_ORACLE_H
#define PM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_kernel orc_kernel;

/* Full key space of the paper's properties. */
enum {
  ORC_K_CONST = 0, ORC_K_GROUPS = 1, ORC_K_BARRIERS = 2,
  ORC_K_FLOP = 3,                       /* + dtype*5 + kind  (dtype 0=f32 1=f64; kind add,mul,div,pow,spec) */
  ORC_K_LLOAD = 13,                     /* + dtype */
  ORC_K_LSTORE = 15,                    /* + dtype */
  ORC_K_GLOBAL = 17,                    /* + (dir*3 + size)*15 + class ; dir 0 load 1 store; size 0:32 1:64 2:128 */
  ORC_NKEYS = 17 + 2 * 3 * 15
};
/* stride classes: 0 "0", 1 "1", 2 "1/2", 3 "2/2", 4 "1/3", 5 "2/3", 6 "3/3",
   7..10 "1/4".."4/4", 11..14 "1/>4".."4/>4" */
#define ORC_NCLASS 15

orc_kernel *orc_parse(const char *text, char *err, int errlen);
void orc_free(orc_kernel *k);
int orc_n_params(const orc_kernel *k);
int orc_n_stmts(const orc_kernel *k);
int orc_n_access(const orc_kernel *k, int stmt);

/* Access classification at the classification instance (every parameter = 128).
   out[stmt][access] class code (-1 for local accesses).  Returns 0 or <0 on error. */
int orc_classify(orc_kernel *k, int32_t *out, int cap);

/* Counts of every key at one parameter point.  0 = ok, <0 error
   (-2 too many points for brute force, -3 unsupported form, -4 count exceeds int64). */
int orc_count_brute(orc_kernel *k, const int64_t *params, int64_t max_points, int64_t *keys);
int orc_count_struct(orc_kernel *k, const int64_t *params, int64_t *keys);

/* Key vector -> feature columns; layout 12 or 32.  Returns k or <0. */
int orc_layout(const int64_t *keys, int layout, int64_t *cols);

/* Features for many points: out[p][k].  method 0 brute, 1 struct. */
int orc_eval(orc_kernel *k, int layout, int method, const int64_t *points, int64_t n_points,
             int64_t max_points, int64_t *out);

/* Compensated prediction: T[r][m] = sum_i F[r][i] W[m][i]. */
void orc_predict(const int64_t *F, int64_t R, int k, const double *W, int M, double *T);
/* Plain magnitude sum_i |F[r][i] W[m][i]| (for cancellation-aware tolerances). */
void orc_predict_abs(const int64_t *F, int64_t R, int k, const double *W, int M, double *A);

/* Top-k smallest by (t, index) within each of n_groups consecutive segments of length seg. */
void orc_topk(const double *t, int64_t n_groups, int64_t seg, int topk, int32_t *idx, double *val);

/* Least squares fit of one model.  objective 0 relative (Sec. 4.3), 1 absolute.
   w_out[k]; report[0]=rank report[1]=cond estimate report[2]=relative residual.
   Columns that are identically zero are dropped (weight 0). Returns 0 ok, 1 rank deficient. */
int orc_fit(const int64_t *F, int64_t R, int k, const double *t, int objective,
            double *w_out, double *report);

/* Batched CPU baseline of the tuning workload: for every point of a template,
   evaluate all its variants (struct counts, layout 32), predict with w, keep top-k.
   kernels[v]; points [n_points][P]; out idx/val [n_points][topk].  Uses OpenMP. */
int orc_eval_predict_topk(orc_kernel **kernels, int n_variants, const int64_t *points,
                          int64_t n_points, const double *w, int topk, int32_t *idx,
                          double *val, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
