// Prediction T = F W^T: the "small inner product" of Sec. 2,
// T_wall(n) ~= sum_i alpha_i p_i(n), for many feature rows and device models.
//
// FP64-accurate path: exact fixed-point arithmetic on the integer pipes.  Each
// model's weights become integers W = round(w * 2^E_m) with sum_i |W_i| <= 2^62 (so
// any int64 counts keep the sum below 2^126); every product F_ri W_mi is formed
// exactly and summed in 128 bits, then converted once.  Error <= 2^-(E_m+1)
// sum_i |F_ri| + 2^-56 |T|, i.e. at most 2^-62 (sum_i |w_i| / min_i |w_i|) + 2^-56 of
// sum_i |F_ri w_mi|: 4e-11 for weights spread like the paper's Table 2.  (64-bit integer <-> float conversions, which would be
// needed per term by a float-float scheme, run on the FP64 pipe of this GPU.)
// The same products feed a per-model argmin over rows and a top-k per (group, model)
// (configuration selection, Sec. 6.1) without writing T.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "eval_common.cuh"
#include "kernels.h"
#include "pm.h"
#include "pm_internal.h"
#include "trace.h"

namespace pmd {

constexpr int PR_ROWS = 32;     // rows per tile
constexpr int PR_WARPS = 8;     // each warp: 4 rows of the tile
constexpr int PR_MAXK = 40;
constexpr int PR_MAXM = 64;

struct PredictSmem {
  int64_t f[PR_ROWS][PR_MAXK + 1];
  int64_t w[PR_MAXK][PR_MAXM];
  int E[PR_MAXM];
};

__device__ void load_weights(PredictSmem &S, const double *W, int M, int k) {
  for (int m = threadIdx.x; m < PR_MAXM; m += blockDim.x) {
    const int E = m < M ? weight_exponent(W + (int64_t)m * k, k) : 0;
    for (int i = 0; i < PR_MAXK; i++) S.w[i][m] = (m < M && i < k) ? llrint(ldexp(W[(int64_t)m * k + i], E)) : 0;
    S.E[m] = E;
  }
}

__device__ void load_rows(PredictSmem &S, const int64_t *F, int64_t r0, int64_t R, int k) {
  for (int i = threadIdx.x; i < PR_ROWS * k; i += blockDim.x) {
    int r = i / k, c = i - r * k;
    S.f[r][c] = (r0 + r < R) ? F[(r0 + r) * k + c] : 0;
  }
}

// A += v W (mod 2^128), v and W signed 64-bit, A four 32-bit limbs: the unsigned
// product from three carry chains of 32-bit multiply-adds (limb products v0 W0, v0 W1,
// v1 W0, v1 W1), then the corrections of the signed operands (v = v_u - 2^64 when
// negative, likewise W), which subtract the other operand from the upper 64 bits.
__device__ __forceinline__ void acc_mad(uint32_t (&A)[4], int64_t v, int64_t W) {
  const uint32_t v0 = (uint32_t)v, v1 = (uint32_t)((uint64_t)v >> 32);
  const uint32_t w0 = (uint32_t)W, w1 = (uint32_t)((uint64_t)W >> 32);
  asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
      "madc.lo.cc.u32 %1, %4, %7, %1;\n\t"
      "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
      "madc.hi.u32    %3, %5, %7, %3;\n\t"
      "mad.hi.cc.u32  %1, %4, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
      "addc.u32       %3, %3, 0;\n\t"
      "mad.lo.cc.u32  %1, %5, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
      "addc.u32       %3, %3, 0;\n\t"
      : "+r"(A[0]), "+r"(A[1]), "+r"(A[2]), "+r"(A[3])
      : "r"(v0), "r"(v1), "r"(w0), "r"(w1));
  if (v < 0) asm("sub.cc.u32 %0, %0, %2;\n\tsubc.u32 %1, %1, %3;\n\t" : "+r"(A[2]), "+r"(A[3]) : "r"(w0), "r"(w1));
  if (W < 0) asm("sub.cc.u32 %0, %0, %2;\n\tsubc.u32 %1, %1, %3;\n\t" : "+r"(A[2]), "+r"(A[3]) : "r"(v0), "r"(v1));
}

// Each thread: rows warp + 8 q (q < 4), models lane + 32 j (j < 2).
__device__ __forceinline__ void tile_fixed(const PredictSmem &S, int k, Acc128 acc[4][2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t a[4][2][4];
#pragma unroll
  for (int q = 0; q < 4; q++)
#pragma unroll
    for (int j = 0; j < 2; j++)
#pragma unroll
      for (int l = 0; l < 4; l++) a[q][j][l] = 0;
  for (int i = 0; i < k; i++) {
    const int64_t w0 = S.w[i][lane], w1 = S.w[i][lane + 32];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int64_t v = S.f[warp + 8 * q][i];
      acc_mad(a[q][0], v, w0);
      acc_mad(a[q][1], v, w1);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; q++)
#pragma unroll
    for (int j = 0; j < 2; j++) {
      acc[q][j].lo = (uint64_t)a[q][j][0] | ((uint64_t)a[q][j][1] << 32);
      acc[q][j].hi = (uint64_t)a[q][j][2] | ((uint64_t)a[q][j][3] << 32);
    }
}

__global__ void __launch_bounds__(PR_WARPS * 32) k_predict_ff(const int64_t *__restrict__ F, int64_t R, int k,
                                                              const double *__restrict__ W, int M,
                                                              double *__restrict__ T) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  PredictSmem &S = *(PredictSmem *)smem_raw;
  load_weights(S, W, M, k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ntiles = (R + PR_ROWS - 1) / PR_ROWS;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * PR_ROWS;
    __syncthreads();
    load_rows(S, F, r0, R, k);
    __syncthreads();
    Acc128 acc[4][2];
    tile_fixed(S, k, acc);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int64_t r = r0 + warp + 8 * q;
      if (r >= R) continue;
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int m = lane + 32 * j;
        if (m < M) T[r * M + m] = key_value(acc_key(acc[q][j]), S.E[m]);
      }
    }
  }
}

// Plain double FMA (cross-check path).
__global__ void k_predict_f64(const int64_t *__restrict__ F, int64_t R, int k, const double *__restrict__ W, int M,
                              double *__restrict__ T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R * M) return;
  const int64_t r = i / M;
  const int m = (int)(i - r * M);
  double acc = 0;
  for (int c = 0; c < k; c++) acc = fma((double)F[r * k + c], W[(int64_t)m * k + c], acc);
  T[i] = acc;
}

static int g_num_sms = 0;
static int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

cudaError_t launch_predict(const int64_t *F, int64_t R, int k, const double *W, int M, int precision, double *T,
                           cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  if (precision == PM_PREC_NATIVE_FP64) {
    int64_t n = R * M;
    k_predict_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F, R, k, W, M, T);
    return cudaGetLastError();
  }
  if (k > PR_MAXK || M > PR_MAXM) return cudaErrorInvalidValue;
  size_t sm = sizeof(PredictSmem);
  cudaFuncSetAttribute(k_predict_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int64_t ntiles = (R + PR_ROWS - 1) / PR_ROWS;
  int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms() * 8);
  k_predict_ff<<<grid, PR_WARPS * 32, sm, st>>>(F, R, k, W, M, T);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- argmin over rows per model

// The order of the times as 64-bit integers: a double's bit pattern, with the magnitude
// bits of negative values flipped, orders like the double itself for everything these
// kernels produce (no NaN, no -0.0).  Comparing integers keeps the comparisons off this
// GPU's narrow FP64 pipe.
__device__ __forceinline__ int64_t time_order(double t) {
  const int64_t b = __double_as_longlong(t);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

__device__ __forceinline__ bool arg_less(double a, int64_t ra, double b, int64_t rb) {
  const int64_t ka = time_order(a), kb = time_order(b);
  return ka < kb || (ka == kb && ra < rb);
}

__global__ void __launch_bounds__(PR_WARPS * 32) k_predict_argmin_part(const int64_t *__restrict__ F, int64_t R,
                                                                       int k, const double *__restrict__ W, int M,
                                                                       ArgPart *__restrict__ part) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  PredictSmem &S = *(PredictSmem *)smem_raw;
  __shared__ ArgPart red[PR_WARPS][PR_MAXM];
  load_weights(S, W, M, k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double bt[2] = {__longlong_as_double(0x7ff0000000000000ll), __longlong_as_double(0x7ff0000000000000ll)};
  int64_t br[2] = {INT64_MAX, INT64_MAX};
  const int64_t ntiles = (R + PR_ROWS - 1) / PR_ROWS;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * PR_ROWS;
    __syncthreads();
    load_rows(S, F, r0, R, k);
    __syncthreads();
    Acc128 acc[4][2];
    tile_fixed(S, k, acc);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int64_t r = r0 + warp + 8 * q;
      if (r >= R) continue;
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int m = lane + 32 * j;
        const double tv = key_value(acc_key(acc[q][j]), S.E[m]);
        if (arg_less(tv, r, bt[j], br[j])) { bt[j] = tv; br[j] = r; }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 2; j++) red[warp][lane + 32 * j] = ArgPart{bt[j], br[j]};
  __syncthreads();
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    ArgPart b = red[0][m];
    for (int w = 1; w < PR_WARPS; w++)
      if (arg_less(red[w][m].t, red[w][m].r, b.t, b.r)) b = red[w][m];
    part[(int64_t)blockIdx.x * M + m] = b;
  }
}

// One CTA per model: strided scan of the partials, then a warp and a CTA reduction.
__global__ void __launch_bounds__(128) k_argmin_reduce(const ArgPart *__restrict__ part, int n_part, int M,
                                                       int64_t *arg, double *mn) {
  __shared__ double s_t[4];
  __shared__ int64_t s_r[4];
  const int m = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double bt = __longlong_as_double(0x7ff0000000000000ll);
  int64_t br = INT64_MAX;
  for (int p = threadIdx.x; p < n_part; p += blockDim.x) {
    const ArgPart x = part[(int64_t)p * M + m];
    if (arg_less(x.t, x.r, bt, br)) { bt = x.t; br = x.r; }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double ot = __shfl_xor_sync(0xffffffffu, bt, o);
    const int64_t orr = __shfl_xor_sync(0xffffffffu, br, o);
    if (arg_less(ot, orr, bt, br)) { bt = ot; br = orr; }
  }
  if (lane == 0) { s_t[warp] = bt; s_r[warp] = br; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 4; w++)
      if (arg_less(s_t[w], s_r[w], bt, br)) { bt = s_t[w]; br = s_r[w]; }
    arg[m] = br == INT64_MAX ? -1 : br;
    mn[m] = bt;
  }
}

cudaError_t launch_argmin_reduce(const ArgPart *part, int n_part, int M, int64_t *arg, double *mn, cudaStream_t st) {
  k_argmin_reduce<<<M, 128, 0, st>>>(part, n_part, M, arg, mn);
  return cudaGetLastError();
}

int argmin_parts() { return num_sms() * 4; }
size_t argmin_scratch_bytes(int M, int n_part) { return (size_t)M * n_part * sizeof(ArgPart); }

static cudaError_t launch_argmin_parts(const int64_t *F, int64_t R, int k, const double *W, int M, void *scratch,
                                       int np, int64_t *arg, double *mn, cudaStream_t st) {
  size_t sm = sizeof(PredictSmem);
  cudaFuncSetAttribute(k_predict_argmin_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_predict_argmin_part<<<np, PR_WARPS * 32, sm, st>>>(F, R, k, W, M, (ArgPart *)scratch);
  return launch_argmin_reduce((const ArgPart *)scratch, np, M, arg, mn, st);
}

cudaError_t launch_predict_argmin(const int64_t *F, int64_t R, int k, const double *W, int M, int precision,
                                  void *scratch, int64_t *arg, double *mn, cudaStream_t st) {
  if (k > PR_MAXK || M > PR_MAXM || precision != PM_PREC_FP64) return cudaErrorInvalidValue;
  return launch_argmin_parts(F, R, k, W, M, scratch, argmin_parts(), arg, mn, st);
}

// ---------------------------------------------------------------- top-k rows per (group, model)

// Configuration selection over materialised features (Sec. 6.1): for every group of
// rows and every model, the topk rows with the smallest predicted time, ordered by
// (time, row).  The times are those k_predict_ff writes, bit for bit.  A warp keeps one
// sorted list per model it owns, entry i in lane i; a tile's 32 candidates are tested
// against the list's last entry and only the passing ones are inserted, smallest first.

constexpr double TK_INF = __builtin_huge_val();

// One compare-exchange stage across lanes lane and lane ^ j: this lane keeps the
// smaller (take_min) or the larger (t, r) pair of the two.
__device__ __forceinline__ void lane_cmp_swap(double &t, int64_t &r, int j, bool take_min) {
  const double ot = __shfl_xor_sync(0xffffffffu, t, j);
  const int64_t orr = __shfl_xor_sync(0xffffffffu, r, j);
  if (arg_less(ot, orr, t, r) == take_min) { t = ot; r = orr; }
}

// Merge this lane's candidate (t, r), if ok, into the warp's sorted list (lt, lr):
// entry i in lane i for i < topk, (+inf, INT64_MAX) in the other lanes.  Warp-uniform
// call; every shuffle and ballot is executed by all 32 lanes (none sits behind a
// short-circuit or a lane-dependent branch).  Candidates not below the list's last
// entry are dropped; one or two survivors are inserted one at a time (warp argmin,
// then a shift), more are sorted by a bitonic network and merged in one pass (the
// elementwise minimum of the list and the reversed candidates holds the 32 smallest
// as a bitonic sequence, which a 5-stage bitonic merge sorts).
__device__ __forceinline__ void warp_list_merge(double &lt, int64_t &lr, double t, int64_t r, bool ok, int topk,
                                                int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  double kt = __shfl_sync(FULL, lt, topk - 1);     // the list's last entry: the threshold
  int64_t kr = __shfl_sync(FULL, lr, topk - 1);
  bool pass = ok && arg_less(t, r, kt, kr);
  unsigned mask = __ballot_sync(FULL, pass);
  if (__popc(mask) > 2) {
    double ct = pass ? t : TK_INF;
    int64_t cr = pass ? r : INT64_MAX;
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1)
#pragma unroll
      for (int j = kk >> 1; j > 0; j >>= 1) lane_cmp_swap(ct, cr, j, ((lane & j) == 0) == ((lane & kk) == 0));
    const double rt = __shfl_sync(FULL, ct, 31 - lane);
    const int64_t rr = __shfl_sync(FULL, cr, 31 - lane);
    if (arg_less(rt, rr, lt, lr)) { lt = rt; lr = rr; }
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) lane_cmp_swap(lt, lr, j, (lane & j) == 0);
    mask = 0;
  }
  for (int round = 0; mask && round < 32; round++) {   // one insertion per round; the winning lane drops out
    double bt = pass ? t : TK_INF;
    int64_t br = pass ? r : INT64_MAX;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double ot = __shfl_xor_sync(FULL, bt, o);
      const int64_t orr = __shfl_xor_sync(FULL, br, o);
      if (arg_less(ot, orr, bt, br)) { bt = ot; br = orr; }
    }
    const int win = __ffs(__ballot_sync(FULL, pass && __double_as_longlong(t) == __double_as_longlong(bt) && r == br)) - 1;
    const int pos = __popc(__ballot_sync(FULL, lane < topk && arg_less(lt, lr, bt, br)));   // <= topk - 1
    const double ut = __shfl_up_sync(FULL, lt, 1);
    const int64_t ur = __shfl_up_sync(FULL, lr, 1);
    if (lane > pos) { lt = ut; lr = ur; }
    else if (lane == pos) { lt = bt; lr = br; }
    if (lane == win) pass = false;
    kt = __shfl_sync(FULL, lt, topk - 1);
    kr = __shfl_sync(FULL, lr, topk - 1);
    pass = pass && arg_less(t, r, kt, kr);
    mask = __ballot_sync(FULL, pass);
  }
  if (lane >= topk) { lt = TK_INF; lr = INT64_MAX; }
}

constexpr int TK_MODELS_PER_WARP = PR_MAXM / PR_WARPS;   // 8

// the tile's times, [row][model] with one pad column, so that a warp reading one
// model's 32 rows hits 32 different banks
constexpr int TK_TSTRIDE = PR_MAXM + 1;
size_t predict_topk_smem() { return sizeof(PredictSmem) + sizeof(double) * PR_ROWS * TK_TSTRIDE + sizeof(int64_t) * PR_ROWS; }

__global__ void __launch_bounds__(PR_WARPS * 32) k_predict_topk(const int64_t *__restrict__ F, int64_t R, int k,
                                                                const double *__restrict__ W, int M,
                                                                const int64_t *__restrict__ rows,
                                                                const TopkUnit *__restrict__ units, int n_units,
                                                                int topk, double *__restrict__ part_t,
                                                                int64_t *__restrict__ part_r,
                                                                int64_t *__restrict__ top_idx,
                                                                double *__restrict__ top_t, int *status) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  PredictSmem &S = *(PredictSmem *)smem_raw;
  double(*tT)[TK_TSTRIDE] = (double(*)[TK_TSTRIDE])(smem_raw + sizeof(PredictSmem));
  int64_t *tR = (int64_t *)(smem_raw + sizeof(PredictSmem) + sizeof(double) * PR_ROWS * TK_TSTRIDE);
  load_weights(S, W, M, k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
    const TopkUnit U = units[u];
    double lt[TK_MODELS_PER_WARP];
    int64_t lr[TK_MODELS_PER_WARP];
#pragma unroll
    for (int j = 0; j < TK_MODELS_PER_WARP; j++) { lt[j] = TK_INF; lr[j] = INT64_MAX; }
    for (int64_t t0 = U.p0; t0 < U.p1; t0 += PR_ROWS) {
      __syncthreads();
      // rows of this tile: positions t0 .. t0+31 of the unit, through the row list if any
      for (int i = threadIdx.x; i < PR_ROWS * k; i += blockDim.x) {
        const int r = i / k, c = i - r * k;
        const int64_t pos = t0 + r;
        int64_t row = -1;
        if (pos < U.p1) {
          row = rows ? rows[pos] : pos;
          if (row < 0 || row >= R) {
            if (c == 0) atomicOr(status, ST_BAD_ROW);
            row = -1;
          }
        }
        S.f[r][c] = row >= 0 ? F[row * k + c] : 0;
        if (c == 0) tR[r] = row;
      }
      __syncthreads();
      Acc128 acc[4][2];
      tile_fixed(S, k, acc);
#pragma unroll
      for (int q = 0; q < 4; q++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
          const int m = lane + 32 * j;
          tT[warp + 8 * q][m] = m < M ? key_value(acc_key(acc[q][j]), S.E[m]) : 0.0;
        }
      __syncthreads();
      const int64_t row = tR[lane];
#pragma unroll
      for (int j = 0; j < TK_MODELS_PER_WARP; j++) {
        const int m = warp + PR_WARPS * j;
        if (m < M) warp_list_merge(lt[j], lr[j], tT[lane][m], row, row >= 0, topk, lane);
      }
    }
#pragma unroll
    for (int j = 0; j < TK_MODELS_PER_WARP; j++) {
      const int m = warp + PR_WARPS * j;
      if (m >= M || lane >= topk) continue;
      if (U.part < 0) {
        const int64_t o = ((int64_t)U.g * M + m) * topk + lane;
        top_idx[o] = lr[j] == INT64_MAX ? -1 : lr[j];
        top_t[o] = lt[j];
      } else {
        const int64_t o = ((int64_t)U.part * M + m) * topk + lane;
        part_t[o] = lt[j];
        part_r[o] = lr[j];
      }
    }
  }
}

// The same top-k for few models (M <= 8): the 64-model tile above would leave most of
// its products and warps idle, so here each lane owns one row (a warp takes 32
// consecutive positions of the unit, the CTA 256) and computes its M exact sums; each
// warp keeps its own sorted lists per model, and at the end of the unit warp m merges
// the eight warps' lists of model m.  Same products, same keys, same (time, row) order.
template <int MN>
__global__ void __launch_bounds__(PR_WARPS * 32) k_predict_topk_rows(const int64_t *__restrict__ F, int64_t R, int k,
                                                                     const double *__restrict__ W, int M,
                                                                     const int64_t *__restrict__ rows,
                                                                     const TopkUnit *__restrict__ units, int n_units,
                                                                     int topk, double *__restrict__ part_t,
                                                                     int64_t *__restrict__ part_r,
                                                                     int64_t *__restrict__ top_idx,
                                                                     double *__restrict__ top_t, int *status) {
  __shared__ int64_t sw[PR_MAXK][MN];
  __shared__ int sE[MN];
  __shared__ double st[PR_WARPS][MN][32];
  __shared__ int64_t sr[PR_WARPS][MN][32];
  for (int m = threadIdx.x; m < MN; m += blockDim.x) {
    const int E = m < M ? weight_exponent(W + (int64_t)m * k, k) : 0;
    for (int i = 0; i < PR_MAXK; i++) sw[i][m] = (m < M && i < k) ? llrint(ldexp(W[(int64_t)m * k + i], E)) : 0;
    sE[m] = E;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
    const TopkUnit U = units[u];
    double lt[MN];
    int64_t lr[MN];
#pragma unroll
    for (int m = 0; m < MN; m++) { lt[m] = TK_INF; lr[m] = INT64_MAX; }
    for (int64_t t0 = U.p0 + 32 * warp; t0 < U.p1; t0 += 32 * PR_WARPS) {   // warp-uniform
      const int64_t pos = t0 + lane;
      int64_t row = -1;
      if (pos < U.p1) {
        row = rows ? rows[pos] : pos;
        if (row < 0 || row >= R) {
          atomicOr(status, ST_BAD_ROW);
          row = -1;
        }
      }
      uint32_t a[MN][4];
#pragma unroll
      for (int m = 0; m < MN; m++) a[m][0] = a[m][1] = a[m][2] = a[m][3] = 0;
      if (row >= 0) {
        const int64_t *f = F + row * k;
        for (int i = 0; i < k; i++) {
          const int64_t v = __ldg(f + i);
#pragma unroll
          for (int m = 0; m < MN; m++) acc_mad(a[m], v, sw[i][m]);
        }
      }
#pragma unroll
      for (int m = 0; m < MN; m++) {
        if (m < M) {   // warp-uniform
          Acc128 A;
          A.lo = (uint64_t)a[m][0] | ((uint64_t)a[m][1] << 32);
          A.hi = (uint64_t)a[m][2] | ((uint64_t)a[m][3] << 32);
          warp_list_merge(lt[m], lr[m], key_value(acc_key(A), sE[m]), row, row >= 0, topk, lane);
        }
      }
    }
    __syncthreads();   // the previous unit's merge has read st / sr
#pragma unroll
    for (int m = 0; m < MN; m++) {
      st[warp][m][lane] = lt[m];
      sr[warp][m][lane] = lr[m];
    }
    __syncthreads();
    if (warp < M && warp < MN) {
      const int m = warp;
      double ft = TK_INF;
      int64_t fr = INT64_MAX;
      for (int w = 0; w < PR_WARPS; w++) {
        const double t = st[w][m][lane];
        const int64_t r = sr[w][m][lane];
        warp_list_merge(ft, fr, t, r, lane < topk && r != INT64_MAX, topk, lane);
      }
      if (lane < topk) {
        if (U.part < 0) {
          const int64_t o = ((int64_t)U.g * M + m) * topk + lane;
          top_idx[o] = fr == INT64_MAX ? -1 : fr;
          top_t[o] = ft;
        } else {
          const int64_t o = ((int64_t)U.part * M + m) * topk + lane;
          part_t[o] = ft;
          part_r[o] = fr;
        }
      }
    }
  }
}

template <int MN>
static void launch_topk_rows(const int64_t *F, int64_t R, int k, const double *W, int M, const int64_t *rows,
                             const TopkUnit *units, int n_units, int topk, double *part_t, int64_t *part_r,
                             int64_t *top_idx, double *top_t, int *status, cudaStream_t st) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_predict_topk_rows<MN>, PR_WARPS * 32, 0);
  const int grid = std::min(n_units, num_sms() * std::max(1, per_sm));
  k_predict_topk_rows<MN><<<grid, PR_WARPS * 32, 0, st>>>(F, R, k, W, M, rows, units, n_units, topk, part_t, part_r,
                                                          top_idx, top_t, status);
}

// Groups split over several units: one CTA per (group, model) merges the units' sorted
// lists of that model; its warps take every eighth block of 32 candidates, then warp 0
// merges the eight warp lists.
__global__ void __launch_bounds__(PR_WARPS * 32) k_topk_merge(const TopkMerge *__restrict__ merges, int M, int topk,
                                                              const double *__restrict__ part_t,
                                                              const int64_t *__restrict__ part_r,
                                                              int64_t *__restrict__ top_idx,
                                                              double *__restrict__ top_t) {
  __shared__ double st[PR_WARPS][32];
  __shared__ int64_t sr[PR_WARPS][32];
  const TopkMerge G = merges[blockIdx.x];
  const int m = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = (int64_t)G.n_parts * topk;
  double lt = TK_INF;
  int64_t lr = INT64_MAX;
  for (int64_t c0 = 32 * warp; c0 < n; c0 += 32 * PR_WARPS) {   // warp-uniform
    const int64_t c = c0 + lane;
    double t = TK_INF;
    int64_t r = INT64_MAX;
    if (c < n) {
      const int64_t o = (((int64_t)G.part0 + c / topk) * M + m) * topk + c % topk;
      t = part_t[o];
      r = part_r[o];
    }
    warp_list_merge(lt, lr, t, r, r != INT64_MAX, topk, lane);
  }
  st[warp][lane] = lt;
  sr[warp][lane] = lr;
  __syncthreads();
  if (warp == 0) {
    double ft = TK_INF;
    int64_t fr = INT64_MAX;
    for (int w = 0; w < PR_WARPS; w++) {
      const int64_t r = sr[w][lane];
      warp_list_merge(ft, fr, st[w][lane], r, lane < topk && r != INT64_MAX, topk, lane);
    }
    if (lane < topk) {
      const int64_t o = ((int64_t)G.g * M + m) * topk + lane;
      top_idx[o] = fr == INT64_MAX ? -1 : fr;
      top_t[o] = ft;
    }
  }
}

cudaError_t launch_predict_topk(const int64_t *F, int64_t R, int k, const double *W, int M, const int64_t *rows,
                                const TopkUnit *units, int n_units, const TopkMerge *merges, int n_merges, int topk,
                                double *part_t, int64_t *part_r, int64_t *top_idx, double *top_t, int *status,
                                cudaStream_t st) {
  if (k > PR_MAXK || M > PR_MAXM || topk < 1 || topk > TOPK_MAX) return cudaErrorInvalidValue;
  if (n_units <= 0) return cudaSuccess;
  if (M <= 8) {   // few models: one row per lane
    if (M == 1) launch_topk_rows<1>(F, R, k, W, M, rows, units, n_units, topk, part_t, part_r, top_idx, top_t, status, st);
    else if (M == 2) launch_topk_rows<2>(F, R, k, W, M, rows, units, n_units, topk, part_t, part_r, top_idx, top_t, status, st);
    else if (M <= 4) launch_topk_rows<4>(F, R, k, W, M, rows, units, n_units, topk, part_t, part_r, top_idx, top_t, status, st);
    else launch_topk_rows<8>(F, R, k, W, M, rows, units, n_units, topk, part_t, part_r, top_idx, top_t, status, st);
  } else {
    const size_t sm = predict_topk_smem();
    cudaFuncSetAttribute(k_predict_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int grid = std::min(n_units, num_sms() * 2);
    k_predict_topk<<<grid, PR_WARPS * 32, sm, st>>>(F, R, k, W, M, rows, units, n_units, topk, part_t, part_r,
                                                    top_idx, top_t, status);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_merges == 0) return e;
  k_topk_merge<<<dim3((unsigned)n_merges, (unsigned)M), PR_WARPS * 32, 0, st>>>(merges, M, topk, part_t, part_r,
                                                                              top_idx, top_t);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- allocation-free argmin

// Partial results of pm_predict_argmin_static live in this fixed device array instead
// of memory from cudaMalloc.  Every GPU that loads the library holds it until exit.
constexpr size_t STATIC_ARGMIN_BYTES = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_argmin_scratch[STATIC_ARGMIN_BYTES];

// Device address of g_argmin_scratch per device, looked up on the first call made
// with that device current (host code may not use the symbol itself as a pointer).
constexpr int STATIC_MAX_DEVICES = 64;
static std::atomic<void *> g_argmin_addr[STATIC_MAX_DEVICES];

}  // namespace pmd

extern "C" pm_status pm_predict_argmin_static(const int64_t *d_F, int64_t R, int32_t k, const double *d_W,
                                              int32_t M, int64_t *d_arg, double *d_min, void *stream) {
  PM_TRACE("pm_predict_argmin_static");
  using namespace pmd;
  if (R < 0 || k <= 0 || k > PR_MAXK || M <= 0 || M > PR_MAXM)
    return pm_set_error_c(PM_ERR_INVALID_ARG, "pm_predict_argmin_static: need R >= 0, 0 < k <= 40, 0 < M <= 64");
  if ((!d_F && R > 0) || !d_W || !d_arg || !d_min) return pm_set_error_c(PM_ERR_INVALID_ARG, "pm_predict_argmin_static: null pointer");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= STATIC_MAX_DEVICES)
    return pm_set_error_c(PM_ERR_CUDA, "pm_predict_argmin_static: no usable current device");
  void *scratch = g_argmin_addr[dev].load();
  if (!scratch) {
    if (cudaGetSymbolAddress(&scratch, g_argmin_scratch) != cudaSuccess || !scratch)
      return pm_set_error_c(PM_ERR_CUDA, "pm_predict_argmin_static: cudaGetSymbolAddress of the scratch array failed");
    g_argmin_addr[dev].store(scratch);
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return pm_set_error_c(PM_ERR_CUDA, "pm_predict_argmin_static: cannot read the SM count");
  // one partial result per (CTA, model); fewer CTAs if the fixed array would overflow
  const int cap = (int)(STATIC_ARGMIN_BYTES / ((size_t)M * sizeof(ArgPart)));
  const int np = std::min(4 * sms, cap);
  if (np < 1) return pm_set_error_c(PM_ERR_INVALID_ARG, "pm_predict_argmin_static: M too large for the scratch array");
  if (launch_argmin_parts(d_F, R, k, d_W, M, scratch, np, d_arg, d_min, (cudaStream_t)stream) != cudaSuccess)
    return pm_set_error_c(PM_ERR_CUDA, "pm_predict_argmin_static: kernel launch failed");
  return PM_OK;
}
