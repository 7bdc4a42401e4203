/* Measurement kernels: timed CUDA kernels whose operation counts the IR describes
 * exactly, for fitting and checking the linear run-time model on this GPU.
 *
 * The weights of T = sum_i alpha_i p_i(n) are fitted per device from timings of
 * "measurement kernels" chosen to exercise the counted properties (Sec. 4.1), timed
 * as in Sec. 4.2 (repeated runs, the first few dropped, the minimum kept), and the
 * model is then evaluated on held-out "test kernels" (Sec. 5).  Each configuration
 * here has an IR description (paper_1604_04997_gb300.workloads.probe_ir) whose
 * loads, stores, flops, barriers and work-group counts are exactly what the CUDA
 * kernel performs per work-item.
 *
 * Kinds (pmm_config.kind) and their variant / k / group fields:
 *   PMM_EMPTY        2-D grid over an n x n index space, no work      group gx x gy
 *   PMM_COPY         b[i] = a[i]                                       group gx
 *   PMM_SUM4         c[i] = a0[i] + a1[i] + a2[i] + a3[i]              group gx
 *   PMM_INDEX        a[i] = i                                          group gx
 *   PMM_VSA          c[s i] = alpha a[s i] + beta b[s i], s = variant  group gx
 *   PMM_FILLED       o[i] = sum_{k' < k, j < s} a[k'][s i + j]         group gx, s = variant
 *   PMM_ARITH        o[y][x] = k iterations of 8 operations of type variant
 *                    (0 add/sub, 1 mul, 2 div, 3 exp, 4 rsqrt)         group gx x gy
 *   PMM_TRANSPOSE_P  out = in^T through a local (T x T+1) tile         tile T = gx
 *   PMM_TRANSPOSE_R  out[x][y] = in[y][x] (reads unit stride)          tile T = gx
 *   PMM_TRANSPOSE_W  out[y][x] = in[x][y] (writes unit stride)         tile T = gx
 *   PMM_MATMUL       C = A B, A n x m, B m x l, local T x T tiles      tile T = gx
 *   PMM_MATMUL_NAIVE C = A B, one element per work-item                tile T = gx
 *   PMM_STENCIL      5-point stencil on the interior of an n x n grid  tile T = gx
 *   PMM_MATVEC       y_b = A_b x_b, n batches of 32 x 32 (fp64)        256 items
 *   PMM_REDUCTION    one sum per group of variant^2 elements           group gx
 *   PMM_AXPY         y = alpha x + y (fp64), variant^2 elements/group  group gx
 *   PMM_VECADD       c = a + b, variant^2 elements per group           group gx
 *   PMM_NBODY        all-pairs gravitation on n bodies (f32)           group gx
 *   PMM_CONV5        5 x 5 convolution, valid region of n x n (f32)    group gx x gy
 * Sizes: n (and m, l for the matmuls) as in the IR's parameters.
 *
 * pmm_time runs the configuration `runs` times on `stream` (each run timed by
 * CUDA events), drops the first `skip` runs and reports the minimum and the mean
 * of the rest in milliseconds.  Device buffers are allocated (and initialised) by
 * the call and freed before it returns; the call synchronises the stream.
 * Returns PM_OK, PM_ERR_INVALID_ARG (unknown kind, bad sizes or group, runs <=
 * skip), PM_ERR_NOMEM or PM_ERR_CUDA; pm_last_error() describes the failure.
 */
#ifndef PM_MEASURE_H
#define PM_MEASURE_H
#include <stdint.h>

#include "pm.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PMM_EMPTY = 0, PMM_COPY, PMM_SUM4, PMM_INDEX, PMM_VSA, PMM_FILLED, PMM_ARITH, PMM_TRANSPOSE_P,
  PMM_TRANSPOSE_R, PMM_TRANSPOSE_W, PMM_MATMUL, PMM_MATMUL_NAIVE, PMM_STENCIL, PMM_MATVEC,
  PMM_REDUCTION, PMM_AXPY, PMM_VECADD, PMM_NBODY, PMM_CONV5, PMM_NKINDS
};

typedef struct {
  int32_t kind;
  int32_t variant;
  int32_t k;
  int32_t gx, gy;
  int32_t f64;         /* 1: fp64 data (and arithmetic) for PMM_COPY, PMM_SUM4, PMM_INDEX, PMM_VSA,
                          PMM_ARITH types 0-2 */
  int64_t n, m, l;
} pmm_config;

pm_status pmm_time(const pmm_config *cfg, int32_t runs, int32_t skip, double *h_min_ms, double *h_mean_ms,
                   void *stream);

/* Integer issue rate of this GPU, the denominator's counterpart for integer-bound
 * kernels: every lane of a fully occupied grid advances independent chains of 32-bit
 * multiply-add, xor and add (the instruction mix of the counting and ranking kernels);
 * the best of five CUDA-event timings gives lane operations (PTX instructions) per
 * second in *h_lane_ops_per_s.  Synchronises `stream`.  PM_OK, PM_ERR_INVALID_ARG,
 * PM_ERR_NOMEM or PM_ERR_CUDA. */
pm_status pmm_int_issue_rate(double *h_lane_ops_per_s, void *stream);

#ifdef __cplusplus
}
#endif
#endif
