// Weight fit (Sec. 4.3): for every device model m, find w_m minimising
//   relative objective  sum_j (1 - F_j w_m / t_jm)^2     (the paper's)
//   absolute objective  sum_j (t_jm - F_j w_m)^2
// The least-squares matrix of model m is A_m = diag(1/t_m) F (relative) or F
// (absolute); its columns are scaled by powers of two so that max_r |A_rc| lies in
// [1/2, 1).  The normal equations A^T A x = A^T b (b = 1, or b = t_m) are formed
// in float-float arithmetic on the FP32 pipes (entries split exactly into hi + lo
// pairs, error-free products by FMA, compensated sums; about 2^-44 relative) per row
// chunk, chunks summed in FP64 (precision PM_PREC_FP64), or on the tensor cores from
// three bf16 terms of A with FP32 accumulation (PM_PREC_BF16X3), or exactly from bf16
// digits of a 47-bit fixed-point image of A when refinement on the three-term Gram
// does not converge (gram_tc.cu);
// the k x k systems are factored by FP64 Cholesky.  Iterative refinement then
// recovers the accuracy: r = b - A x is formed from the exact fixed-point product
// F w (the prediction kernel's arithmetic), t - F w in FP64 and float-float products
// with 1/t (about 2^-45), the correction solves G d = A^T r with the same factor, and
// x += d.  FP64 is kept to the Cholesky factors, the substitutions and the sums: this
// GPU's FP64 pipe is narrow.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "eval_common.cuh"
#include "kernels.h"
#include "pm.h"

namespace pmd {

constexpr int FIT_MAXK = 32;
constexpr int FIT_ROWS = 64;      // rows staged per batch
constexpr int FIT_THREADS = 256;

// ---- column maxima of |F| (as unsigned bit patterns, for atomicMax)
__global__ void k_colmax(const int64_t *__restrict__ F, int64_t R, int k, unsigned long long *cmax) {
  __shared__ unsigned long long s[FIT_MAXK];
  if (threadIdx.x < FIT_MAXK) s[threadIdx.x] = 0;
  __syncthreads();
  const int c = threadIdx.x % k;
  const int rstep = blockDim.x / k;
  unsigned long long m = 0;
  if (threadIdx.x < rstep * k) {
    for (int64_t r = (int64_t)blockIdx.x * rstep + threadIdx.x / k; r < R; r += (int64_t)gridDim.x * rstep) {
      const int64_t v = F[r * k + c];
      const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
      m = a > m ? a : m;
    }
    atomicMax(&s[c], m);
  }
  __syncthreads();
  if (threadIdx.x < k) atomicMax(&cmax[threadIdx.x], s[threadIdx.x]);
}

// exponent e_c with max |F_c| in [2^(e-1), 2^e) (0 for an all-zero column)
__device__ __forceinline__ int col_exp(unsigned long long mx) { return mx ? 64 - __clzll((long long)mx) : 0; }

// ---- U = F diag(2^-e) as float-float pairs: Uh = rn(F), Ul = rn(F - Uh), scaled exactly
__global__ void k_scale(const int64_t *__restrict__ F, int64_t R, int k, const unsigned long long *cmax,
                        float *__restrict__ Uh, float *__restrict__ Ul) {
  const int64_t n = R * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % k);
    const int64_t v = F[i];
    const float h = __ll2float_rn(v);
    const float l = __ll2float_rn(v - (int64_t)h);
    const int e = col_exp(cmax[c]);
    Uh[i] = ldexpf(h, -e);
    Ul[i] = ldexpf(l, -e);
  }
}

// A double as a float-float pair (hi + lo within 2^-47 of x) with integer operations
// when its exponent is in [-70, 120] (this GPU's FP64 pipe is narrow; timings,
// predictions and residuals are well inside that range), else by FP64 conversions.
__device__ __forceinline__ float2 ff_of_double(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -70 || e > 120) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
  }
  const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;                      // 52 fraction bits
  // hi: the leading one and the next 23 bits (truncated); lo: the 29 bits below, rounded
  const float h = __uint_as_float(sgn | ((uint32_t)(e + 127) << 23) | (uint32_t)(m >> 29));
  const float l = __uint2float_rn((uint32_t)(m & 0x1FFFFFFFu)) * __uint_as_float((uint32_t)(e - 52 + 127) << 23);
  return make_float2(h, sgn ? -l : l);
}

// 1/t for t > 0 as float-float (within ~2^-46): FP32 reciprocal, one Newton step with
// the residual formed by FMA; FP64 division outside [2^-100, 2^100].
__device__ __forceinline__ float2 ff_recip(double t) {
  const uint64_t b = (uint64_t)__double_as_longlong(t);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -100 || e > 100) {
    const double r = 1.0 / t;
    const float h = __double2float_rn(r);
    return make_float2(h, __double2float_rn(r - (double)h));
  }
  const float2 tt = ff_of_double(t);
  const float y = __frcp_rn(tt.x);
  float res = __fmaf_rn(-tt.x, y, 1.0f);       // 1 - th y, exact: th y is within 2^-23 of 1
  res = __fmaf_rn(-tt.y, y, res);              // - tl y
  const float lo = __fmul_rn(y, res);
  const float hi = __fadd_rn(y, lo);           // renormalise (Fast2Sum: |y| >= |lo|)
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, y)));
}

// ---- row factors as float-float: 1/t (relative) or 1 (absolute); beta = 1 or t.  The
// residual kernel reuses the relative row factor as 1/t.
__global__ void k_rowfac(const double *__restrict__ T, int64_t n, int objective, float2 *__restrict__ rf,
                         float2 *__restrict__ beta, int *status) {
  const int64_t big = __double_as_longlong(1e300);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = T[i];
    const int64_t tb = __double_as_longlong(t);   // 0 < t <= 1e300 (NaN excluded) by its bits
    if (tb <= 0 || tb > big) {
      atomicOr(status, ST_BAD_INPUT);
      rf[i] = beta[i] = make_float2(0.f, 0.f);
      continue;
    }
    if (objective == PM_FIT_RELATIVE) {
      rf[i] = ff_recip(t);
      beta[i] = make_float2(1.f, 0.f);
    } else {
      rf[i] = make_float2(1.f, 0.f);
      beta[i] = ff_of_double(t);
    }
  }
}

// float-float helpers: error-free product by FMA, compensated accumulation
__device__ __forceinline__ float2 ff_mul(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  return make_float2(p, e);
}
__device__ __forceinline__ void ff_acc(float &s, float &c, float2 p) {
  const float t = __fadd_rn(s, p.x);
  const float z = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p.x, z)), p.y));
  s = t;
}

// ---- per (model, column) maxima of |A_rc| = |U_rc| * rowfactor_rm (float bits, atomicMax)
__global__ void k_acolmax(const float *__restrict__ U, const float2 *__restrict__ rf, int64_t R, int k, int M,
                          int64_t rows_per_chunk, unsigned *__restrict__ amax) {
  const int m = blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t r1 = min(R, r0 + rows_per_chunk);
  const int c = threadIdx.x % 32, lr = threadIdx.x / 32;
  float mx = 0.f;
  if (c < k)
    for (int64_t r = r0 + lr; r < r1; r += FIT_THREADS / 32) {
      mx = fmaxf(mx, fabsf(__fmul_rn(U[r * k + c], rf[r * M + m].x)));
    }
  __shared__ float red[FIT_THREADS];
  red[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x < 32 && c < k) {
    float t = 0.f;
    for (int q = 0; q < FIT_THREADS / 32; q++) t = fmaxf(t, red[q * 32 + threadIdx.x]);
    atomicMax(&amax[m * FIT_MAXK + c], __float_as_uint(t));   // non-negative floats order as integers
  }
}

// power-of-two exponent f with max |A_c| * 2^-f in [1/2, 1) (0 for an all-zero column)
__device__ __forceinline__ int acol_exp(unsigned bits) {
  if (!bits) return 0;
  int e;
  frexpf(__uint_as_float(bits), &e);
  return e;
}

// ---- Gram matrices and right-hand sides.
// Grid (row chunks, models).  Each CTA accumulates, for its model, the upper triangle
// of sum_r v_r v_r^T and sum_r v_r * beta_r over its rows, where
// relative: v = u / t, beta = 1;   absolute: v = u, beta = t.
// The row [v | beta] (k + 1 <= 33 values, padded to 36) is staged in shared memory as
// float-float pairs; the 36 x 36 upper triangle is cut into the 45 4x4 blocks (bi <=
// bj) of a 9 x 9 block grid, and each of 5 row groups of 45 threads takes every
// block once: a thread reads two 4-column slices per row and forms 16 error-free
// products, accumulated with TwoSum compensation.  Chunk results are added to the
// FP64 totals with atomics.
constexpr int GB_COLS = 36, GB_BLOCKS = 9, GB_TASKS = 45, GB_GROUPS = 5;
__global__ void __launch_bounds__(FIT_THREADS) k_gram(const float *__restrict__ Uh, const float *__restrict__ Ul,
                                                      const float2 *__restrict__ rf, const float2 *__restrict__ bt,
                                                      int64_t R, int k, int M, int64_t rows_per_chunk,
                                                      const unsigned *__restrict__ amax, double *__restrict__ G,
                                                      double *__restrict__ rhs) {
  __shared__ __align__(16) float vh[FIT_ROWS][GB_COLS], vl[FIT_ROWS][GB_COLS];
  __shared__ int f[FIT_MAXK];
  const int m = blockIdx.y;
  if (threadIdx.x < FIT_MAXK) f[threadIdx.x] = threadIdx.x < k ? acol_exp(amax[m * FIT_MAXK + threadIdx.x]) : 0;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t r1 = min(R, r0 + rows_per_chunk);
  // this thread's block (bi, bj) and row group
  const int task = threadIdx.x % GB_TASKS, grp = threadIdx.x / GB_TASKS;
  int bi = 0, rest = task;
  while (rest >= GB_BLOCKS - bi) { rest -= GB_BLOCKS - bi; bi++; }
  const int bj = bi + rest;
  const bool active = grp < GB_GROUPS && 4 * bi <= k && 4 * bj <= k;   // column k is beta
  constexpr int RPG = (FIT_ROWS + GB_GROUPS - 1) / GB_GROUPS;
  float s[16], c[16];
#pragma unroll
  for (int q = 0; q < 16; q++) s[q] = c[q] = 0.f;
  for (int64_t rb = r0; rb < r1; rb += FIT_ROWS) {
    __syncthreads();
    const int nr = (int)min((int64_t)FIT_ROWS, r1 - rb);
    for (int i = threadIdx.x; i < FIT_ROWS * GB_COLS; i += FIT_THREADS) {
      const int rr = i / GB_COLS, cc = i - rr * GB_COLS;
      float2 v = make_float2(0.f, 0.f);
      if (rr < nr) {
        if (cc < k) {
          const int64_t o = (rb + rr) * k + cc;
          const float2 r = rf[(rb + rr) * M + m];
          v = ff_mul(Uh[o], Ul[o], r.x, r.y);
          v.x = ldexpf(v.x, -f[cc]);
          v.y = ldexpf(v.y, -f[cc]);
        } else if (cc == k) {
          v = bt[(rb + rr) * M + m];
        }
      }
      vh[rr][cc] = v.x;
      vl[rr][cc] = v.y;
    }
    __syncthreads();
    if (active) {
      const int rend = min(nr, (grp + 1) * RPG);
      for (int rr = grp * RPG; rr < rend; rr++) {
        const float4 ah = *(const float4 *)&vh[rr][4 * bi], al = *(const float4 *)&vl[rr][4 * bi];
        const float4 bh = *(const float4 *)&vh[rr][4 * bj], bl = *(const float4 *)&vl[rr][4 * bj];
        const float xa[4] = {ah.x, ah.y, ah.z, ah.w}, ya[4] = {al.x, al.y, al.z, al.w};
        const float xb[4] = {bh.x, bh.y, bh.z, bh.w}, yb[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
          for (int j = 0; j < 4; j++) ff_acc(s[4 * i + j], c[4 * i + j], ff_mul(xa[i], ya[i], xb[j], yb[j]));
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int i = 0; i < 4; i++) {
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int a = 4 * bi + i, b = 4 * bj + j;
      if (a > b || a >= k || b > k) continue;
      const double val = (double)s[4 * i + j] + (double)c[4 * i + j];
      if (b < k) atomicAdd(&G[((int64_t)m * FIT_MAXK + a) * FIT_MAXK + b], val);
      else atomicAdd(&rhs[(int64_t)m * FIT_MAXK + a], val);
    }
  }
}

// ---- Cholesky of each model's Gram (one warp per model), FP64.
// Columns whose scale exponent marks them all-zero are replaced by identity rows
// (weight 0).  A pivot below tol * (largest diagonal) marks the model rank deficient
// and its direction is dropped likewise.  Writes L (lower) and the first solution.
__global__ void k_chol_solve(double *__restrict__ G, const double *__restrict__ rhs, int k, int M,
                             const unsigned long long *cmax, double *__restrict__ x, int *__restrict__ info,
                             double *__restrict__ diag_ratio) {
  const int m = blockIdx.x;
  if (m >= M) return;
  __shared__ double L[FIT_MAXK][FIT_MAXK + 1];
  __shared__ double y[FIT_MAXK];
  __shared__ int dead[FIT_MAXK];
  const int lane = threadIdx.x;
  double *Gm = G + (int64_t)m * FIT_MAXK * FIT_MAXK;
  for (int i = lane; i < k * k; i += 32) {
    const int a = i / k, b = i - a * k;
    L[a][b] = a <= b ? Gm[a * FIT_MAXK + b] : Gm[b * FIT_MAXK + a];   // symmetric from the upper triangle
  }
  if (lane < k) dead[lane] = cmax[lane] == 0;
  __syncwarp();
  double dmax = 0;
  for (int a = 0; a < k; a++) if (!dead[a]) dmax = fmax(dmax, L[a][a]);
  const double tol = dmax * 1e-13;
  int rank = 0;
  double pmin = 1e300, pmax = 0;
  for (int j = 0; j < k; j++) {
    // L[j][j] = sqrt(G[j][j] - sum_{p<j} L[j][p]^2)
    double d = L[j][j];
    for (int p = 0; p < j; p++) d -= L[j][p] * L[j][p];
    const bool drop = dead[j] || !(d > tol);
    __syncwarp();
    if (drop) {
      if (lane == 0) { dead[j] = 1; L[j][j] = 1.0; }
      if (lane < k && lane > j) L[lane][j] = 0.0;
      if (lane < j) L[j][lane] = 0.0;
      __syncwarp();
      continue;
    }
    const double ljj = sqrt(d);
    rank++;
    pmin = fmin(pmin, ljj);
    pmax = fmax(pmax, ljj);
    if (lane > j && lane < k) {
      double s = L[lane][j];
      for (int p = 0; p < j; p++) s -= L[lane][p] * L[j][p];
      L[lane][j] = s / ljj;
    }
    __syncwarp();
    if (lane == 0) L[j][j] = ljj;
    __syncwarp();
  }
  // forward and back substitution (one lane), dead directions get 0
  if (lane == 0) {
    for (int a = 0; a < k; a++) {
      double s = dead[a] ? 0.0 : rhs[(int64_t)m * FIT_MAXK + a];
      for (int p = 0; p < a; p++) s -= L[a][p] * y[p];
      y[a] = dead[a] ? 0.0 : s / L[a][a];
    }
    for (int a = k - 1; a >= 0; a--) {
      double s = y[a];
      for (int p = a + 1; p < k; p++) s -= L[p][a] * x[(int64_t)m * FIT_MAXK + p];
      x[(int64_t)m * FIT_MAXK + a] = dead[a] ? 0.0 : s / L[a][a];
    }
    int nz = 0;
    for (int a = 0; a < k; a++) nz += cmax[a] == 0;
    unsigned mask = 0;
    for (int a = 0; a < k; a++) mask |= (unsigned)dead[a] << a;
    info[m * 4 + 0] = rank;
    info[m * 4 + 1] = nz;
    info[m * 4 + 2] = rank < k - nz ? 1 : 0;
    info[m * 4 + 3] = (int)mask;
    diag_ratio[m] = pmin > 0 ? (pmax / pmin) * (pmax / pmin) : 1e300;
  }
  __syncwarp();
  for (int i = lane; i < k * k; i += 32) {
    const int a = i / k, b = i - a * k;
    Gm[a * FIT_MAXK + b] = b <= a ? L[a][b] : 0.0;   // keep L for the refinement solves
  }
  if (lane < k) Gm[lane * FIT_MAXK + lane] = L[lane][lane];
}

// ---- weights from scaled coordinates: w_c = x_c * 2^-e_c
__global__ void k_unscale(const double *__restrict__ x, int k, int M, const unsigned long long *cmax,
                          const unsigned *__restrict__ amax, double *__restrict__ W) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k * M) return;
  const int m = i / k, c = i - m * k;
  W[i] = cmax[c] ? ldexp(x[(int64_t)m * FIT_MAXK + c], -col_exp(cmax[c]) - acol_exp(amax[m * FIT_MAXK + c])) : 0.0;
}

// ---- residual q = (b - A x) scaled for A^T q, from the exact product p = F w:
// relative: r = 1 - p / t = (t - p) (1/t), q = r / t;   absolute: r = t - p, q = r.
// Also sums r^2 and b^2 (b = 1, or t).  Relative objective: t - p in FP64 (exact while
// p is within a factor 2 of t), then float-float products with the row factor 1/t and
// a float-float sum of r^2, so that one FP64 operation per element remains.
__global__ void k_residual(const double *__restrict__ P, const double *__restrict__ T, const float2 *__restrict__ rf,
                           int64_t R, int M, int objective, float2 *__restrict__ Q, double *__restrict__ rr,
                           double *__restrict__ bb) {
  __shared__ double s_r[64], s_b[64];
  if (threadIdx.x < 64) { s_r[threadIdx.x] = 0; s_b[threadIdx.x] = 0; }
  __syncthreads();
  const int64_t n = R * M, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool fixed_m = stride % M == 0;   // then every element of this thread has model i0 % M
  float sr = 0.f, cr = 0.f;               // float-float sum of r^2 (relative)
  double ar = 0, ab = 0;
  int64_t cnt = 0;
  for (int64_t i = i0; i < n; i += stride) {
    const double t = T[i], p = P[i];
    if (objective == PM_FIT_RELATIVE) {
      const float2 d = ff_of_double(t - p), it = rf[i];
      const float2 r = ff_mul(d.x, d.y, it.x, it.y);
      Q[i] = ff_mul(r.x, r.y, it.x, it.y);
      const float2 r2 = ff_mul(r.x, r.y, r.x, r.y);
      if (fixed_m) {
        ff_acc(sr, cr, r2);
        cnt++;
      } else {
        const int m = (int)(i % M);
        atomicAdd(&s_r[m], (double)r2.x + (double)r2.y);
        atomicAdd(&s_b[m], 1.0);
      }
    } else {
      const double r = t - p;
      Q[i] = ff_of_double(r);
      if (fixed_m) { ar += r * r; ab += t * t; }
      else { const int m = (int)(i % M); atomicAdd(&s_r[m], r * r); atomicAdd(&s_b[m], t * t); }
    }
  }
  if (fixed_m && i0 < n) {
    if (objective == PM_FIT_RELATIVE) { ar = (double)sr + (double)cr; ab = (double)cnt; }
    atomicAdd(&s_r[i0 % M], ar);
    atomicAdd(&s_b[i0 % M], ab);
  }
  __syncthreads();
  if (threadIdx.x < M && threadIdx.x < 64) {
    atomicAdd(&rr[threadIdx.x], s_r[threadIdx.x]);
    atomicAdd(&bb[threadIdx.x], s_b[threadIdx.x]);
  }
}

// ---- g_m = U^T q_m  (float-float products and sums per chunk, FP64 totals).
// Grid (row chunks, groups of 8 models): each feature value is read once for the 8
// models of its CTA; thread (column c, row lane) keeps 8 compensated sums.
constexpr int ATQ_MODELS = 8;
__global__ void __launch_bounds__(FIT_THREADS) k_atq(const float *__restrict__ Uh, const float *__restrict__ Ul,
                                                     const float2 *__restrict__ Q, int64_t R, int k, int M,
                                                     int64_t rows_per_chunk, const unsigned *__restrict__ amax,
                                                     double *__restrict__ g) {
  const int m0 = blockIdx.y * ATQ_MODELS;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t r1 = min(R, r0 + rows_per_chunk);
  const int c = threadIdx.x % 32, lane_r = threadIdx.x / 32;   // 8 row lanes x 32 columns
  const int nm = min(ATQ_MODELS, M - m0);
  float s[ATQ_MODELS], cc[ATQ_MODELS];
#pragma unroll
  for (int j = 0; j < ATQ_MODELS; j++) s[j] = cc[j] = 0.f;
  if (c < k) {
    for (int64_t r = r0 + lane_r; r < r1; r += FIT_THREADS / 32) {
      const float uh = Uh[r * k + c], ul = Ul[r * k + c];
      const float2 *q = Q + r * M + m0;
#pragma unroll
      for (int j = 0; j < ATQ_MODELS; j++) {
        if (j < nm) {
          const float2 qj = q[j];
          ff_acc(s[j], cc[j], ff_mul(uh, ul, qj.x, qj.y));
        }
      }
    }
  }
  __shared__ double red[FIT_THREADS / 32][ATQ_MODELS][32];
#pragma unroll
  for (int j = 0; j < ATQ_MODELS; j++) red[lane_r][j][c] = (double)s[j] + (double)cc[j];
  __syncthreads();
  for (int o = threadIdx.x; o < ATQ_MODELS * 32; o += FIT_THREADS) {
    const int j = o / 32, col = o % 32;
    if (j < nm && col < k) {
      double tot = 0;
      for (int q = 0; q < FIT_THREADS / 32; q++) tot += red[q][j][col];
      atomicAdd(&g[(int64_t)(m0 + j) * FIT_MAXK + col], ldexp(tot, -acol_exp(amax[(m0 + j) * FIT_MAXK + col])));
    }
  }
}

// ---- x += L^-T L^-1 g per model; records |d| / |x|.  One warp per model, lane a owns
// row a: the forward and backward substitutions run column by column, each step one
// division by lane a and one multiply-add in every lane below (or above) it, so the
// FP64 latency of a step is paid once per column, not once per term.
__global__ void __launch_bounds__(32) k_refine_update(const double *__restrict__ Lall, const double *__restrict__ g,
                                                      int k, int M, const int *__restrict__ info,
                                                      double *__restrict__ x, double *__restrict__ upd) {
  const int m = blockIdx.x, a = threadIdx.x;
  if (m >= M) return;
  const unsigned dead = (unsigned)info[m * 4 + 3];
  const double *L = Lall + (int64_t)m * FIT_MAXK * FIT_MAXK;
  const bool live = a < k;
  const double diag = live ? L[a * FIT_MAXK + a] : 1.0;
  // L y = g: s_a = g_a - sum_{p<a} L[a][p] y_p, subtracted in the order p = 0, 1, ...
  double s = (live && !((dead >> a) & 1)) ? g[(int64_t)m * FIT_MAXK + a] : 0.0;
  double y = 0.0;
  for (int c = 0; c < k; c++) {
    if (a == c) y = s / diag;
    const double yc = __shfl_sync(0xffffffffu, y, c);
    if (live && a > c) s -= L[a * FIT_MAXK + c] * yc;
  }
  // L^T d = y: t_a = y_a - sum_{p>a} L[p][a] d_p
  double t = y, d = 0.0;
  for (int c = k - 1; c >= 0; c--) {
    if (a == c) d = t / diag;
    const double dc = __shfl_sync(0xffffffffu, d, c);
    if (live && a < c) t -= L[c * FIT_MAXK + a] * dc;
  }
  if (!live || ((dead >> a) & 1)) d = 0.0;
  double xa = 0.0;
  if (live) {
    xa = x[(int64_t)m * FIT_MAXK + a] + d;
    x[(int64_t)m * FIT_MAXK + a] = xa;
  }
  double dn = d * d, xn = xa * xa;
  for (int o = 16; o; o >>= 1) {
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
    xn += __shfl_xor_sync(0xffffffffu, xn, o);
  }
  if (a == 0) upd[m] = xn > 0 ? sqrt(dn / xn) : 0.0;
}

// ------------------------------------------------------------------------------------ host side

size_t fit_scratch_bytes(int64_t R, int k, int M) {
  size_t b = 0;
  b += 256;                                        // cmax
  b += (size_t)M * FIT_MAXK * 4;                   // amax
  b += (size_t)R * k * 8;                          // Uh, Ul
  b += (size_t)R * M * 16;                         // row factors, beta
  b += (size_t)R * M * 8;                          // Q
  b += (size_t)R * M * 8;                          // P
  b += (size_t)M * FIT_MAXK * FIT_MAXK * 8;        // G / L
  b += (size_t)M * FIT_MAXK * 8 * 3;               // rhs, x, g
  b += (size_t)M * (4 * 4 + 8 * 4);                // info, ratio, upd, rr, bb
  return b + 32 * 256;                             // every carve rounds up to 256 bytes
}

static char *carve(char *&p, size_t bytes) {
  char *r = p;
  p += (bytes + 255) & ~(size_t)255;
  return r;
}

cudaError_t launch_fit(const int64_t *F, int64_t R, int k, const double *T, int M, int objective, int gram,
                       int steps, void *scratch, double *W_out, FitHost *host, int *status, cudaStream_t st) {
  char *p = (char *)scratch;
  unsigned long long *cmax = (unsigned long long *)carve(p, 256);
  unsigned *amax = (unsigned *)carve(p, (size_t)M * FIT_MAXK * 4);
  float *U = (float *)carve(p, (size_t)R * k * 4);
  float *Ul = (float *)carve(p, (size_t)R * k * 4);
  float2 *rf = (float2 *)carve(p, (size_t)R * M * 8);
  float2 *bt = (float2 *)carve(p, (size_t)R * M * 8);
  float2 *Q = (float2 *)carve(p, (size_t)R * M * 8);
  double *P = (double *)carve(p, (size_t)R * M * 8);
  double *G = (double *)carve(p, (size_t)M * FIT_MAXK * FIT_MAXK * 8);
  double *rhs = (double *)carve(p, (size_t)M * FIT_MAXK * 8);
  double *x = (double *)carve(p, (size_t)M * FIT_MAXK * 8);
  double *g = (double *)carve(p, (size_t)M * FIT_MAXK * 8);
  int *info = (int *)carve(p, (size_t)M * 16);
  double *ratio = (double *)carve(p, (size_t)M * 8);
  double *upd = (double *)carve(p, (size_t)M * 8);
  double *rr = (double *)carve(p, (size_t)M * 8);
  double *bb = (double *)carve(p, (size_t)M * 8);
  cudaError_t e;
  cudaMemsetAsync(cmax, 0, 256, st);
  cudaMemsetAsync(amax, 0, (size_t)M * FIT_MAXK * 4, st);
  cudaMemsetAsync(G, 0, (size_t)M * FIT_MAXK * FIT_MAXK * 8, st);
  cudaMemsetAsync(rhs, 0, (size_t)M * FIT_MAXK * 8, st);
  cudaMemsetAsync(upd, 0, (size_t)M * 8, st);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_colmax<<<sms * 2, 256, 0, st>>>(F, R, k, cmax);
  k_scale<<<sms * 8, 256, 0, st>>>(F, R, k, cmax, U, Ul);
  k_rowfac<<<sms * 8, 256, 0, st>>>(T, R * M, objective, rf, bt, status);
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(4 * sms / std::max(1, M) + 1, (R + 255) / 256));
  const int64_t rpc = (R + chunks - 1) / chunks;
  const int mchunks = (int)std::max<int64_t>(1, std::min<int64_t>(16 * sms / std::max(1, M) + 1, (R + 255) / 256));
  k_acolmax<<<dim3(mchunks, M), FIT_THREADS, 0, st>>>(U, rf, R, k, M, (R + mchunks - 1) / mchunks, amax);
  const int groups = (M + ATQ_MODELS - 1) / ATQ_MODELS;
  // enough row chunks for several CTAs per SM: the float-float sums are load-latency bound
  const int achunks = (int)std::max<int64_t>(1, std::min<int64_t>(16 * sms / groups + 1, (R + 255) / 256));
  const int64_t arpc = (R + achunks - 1) / achunks;
  if (gram != 0) {
    // Gram on the tensor cores (three bf16 terms of A, or the exact digits of its 47-bit
    // fixed-point image); right-hand side A^T b = U^T (rowfactor b) with the
    // float-float product kernel
    if ((e = launch_gram_tc(U, Ul, rf, R, k, M, amax, G, gram == 2, status, st)) != cudaSuccess) return e;
    k_atq<<<dim3(achunks, groups), FIT_THREADS, 0, st>>>(U, Ul, objective == PM_FIT_RELATIVE ? rf : bt, R, k, M,
                                                         arpc, amax, rhs);
  } else {
    k_gram<<<dim3(chunks, M), FIT_THREADS, 0, st>>>(U, Ul, rf, bt, R, k, M, rpc, amax, G, rhs);
  }
  k_chol_solve<<<M, 32, 0, st>>>(G, rhs, k, M, cmax, x, info, ratio);
  for (int it = 0; it < steps; it++) {
    k_unscale<<<(k * M + 255) / 256, 256, 0, st>>>(x, k, M, cmax, amax, W_out);
    if ((e = launch_predict(F, R, k, W_out, M, PM_PREC_FP64, P, st)) != cudaSuccess) return e;
    cudaMemsetAsync(rr, 0, (size_t)M * 8, st);
    cudaMemsetAsync(bb, 0, (size_t)M * 8, st);
    cudaMemsetAsync(g, 0, (size_t)M * FIT_MAXK * 8, st);
    k_residual<<<sms * 4, 256, 0, st>>>(P, T, rf, R, M, objective, Q, rr, bb);
    k_atq<<<dim3(achunks, groups), FIT_THREADS, 0, st>>>(U, Ul, Q, R, k, M, arpc, amax, g);
    k_refine_update<<<M, 32, 0, st>>>(G, g, k, M, info, x, upd);
  }
  k_unscale<<<(k * M + 255) / 256, 256, 0, st>>>(x, k, M, cmax, amax, W_out);
  // final residual for the report
  if ((e = launch_predict(F, R, k, W_out, M, PM_PREC_FP64, P, st)) != cudaSuccess) return e;
  cudaMemsetAsync(rr, 0, (size_t)M * 8, st);
  cudaMemsetAsync(bb, 0, (size_t)M * 8, st);
  k_residual<<<sms * 4, 256, 0, st>>>(P, T, rf, R, M, objective, Q, rr, bb);
  cudaMemcpyAsync(host->info, info, (size_t)M * 16, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(host->ratio, ratio, (size_t)M * 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(host->upd, upd, (size_t)M * 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(host->rr, rr, (size_t)M * 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(host->bb, bb, (size_t)M * 8, cudaMemcpyDeviceToHost, st);
  return cudaGetLastError();
}

}  // namespace pmd
