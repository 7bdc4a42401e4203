// Gram matrices of the weight fit (Sec. 4.3) on the fifth-generation tensor cores,
// exactly in integer arithmetic:
//   G_m = A_m^T A_m,   A_m = diag(rowfactor_m) U diag(2^-f_mc)   (|A| < 1 per column)
//
// Every entry is rounded once to a 47-bit fixed-point integer a = round(A 2^47) and
// written as seven balanced base-128 digits, a = sum_q d_q 128^q with d_q in [-64, 63].
// A digit is exact in bf16 and a digit product is at most 2^12 in magnitude, so a
// tcgen05.mma (kind::f16, FP32 accumulation) sums 4096 rows of digit products without
// rounding: every partial sum is an integer below 2^24.  With the digits of column c
// at operand row 32 q + c, one 128-row stage X (224 digit rows, padded to 256) feeds
// two MMAs (M = 128 rows each, N = 224, K = 16 per instruction):
//   D1 = X[0:128]^T X[0:224],   D2 = X[128:256]^T X[0:224]
// so D holds P[q,c][q',c'] = sum_rows d_q(c) d_q'(c') for every digit pair.  After each
// 4096-row chunk the epilogue combines sum_{q,q'} 128^(q+q') P exactly in integers
// (two 64-bit parts), converts to FP64, scales by 2^-94 and adds the chunk into G.
// The only error is the rounding of A to 47 bits (relative 2^-47 of the column's
// largest entry), below the 2^-44 of the float-float path.
//
// Three-term mode (precision PM_PREC_BF16X3): every entry of A is instead split into
// three bf16 terms, A ~ h + m + l (h = bf16(A), m = bf16(A - h), l = bf16(A - h - m):
// 24 significant bits), at operand rows 32 q + c (q = 0, 1, 2; rows 96..127 zero); one
// MMA (M = 128, N = 96) per K-step gives the nine term-pair sums in FP32, whose sum is
// G to about 2^-24 relative per 4096-row chunk.  The fit's iterative refinement, with
// exact residuals, recovers full accuracy as long as cond(G) 2^-24 is well below 1.
//
// One CTA per SM (the two accumulators take 448 of the 512 TMEM columns), persistent
// over (model, chunk) work items, 16 warps; 128-row stages are double-buffered so the
// digits of stage s + 1 are written while the MMAs of stage s run, and each thread's
// inputs are loaded one stage ahead.  Every mbarrier wait is bounded; on timeout the
// kernel records ST_TIMEOUT and stops.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include <algorithm>

#include "eval_common.cuh"
#include "kernels.h"
#include "mbar_wait.cuh"

namespace pmd {

namespace {

constexpr int GT_THREADS = 512;
constexpr int GT_COLS = 32;               // feature columns (padded)
constexpr int GT_KS = 128;                // rows per stage (8 per warp): 8 MMA K-steps of 16
constexpr int GT_CHUNK = 4096;            // rows per accumulation in TMEM
constexpr uint32_t GT_SBO = (GT_KS / 8) * 128;          // 2048 B between 8-row operand groups

// the two modes: DIG terms per entry (7 exact digits, or 3 bf16 terms); operand rows
// DIG * 32 (padded to MN); MMA N = DIG * 32; stage and TMEM sizes
template <int DIG> struct GtMode {
  static constexpr int N = DIG * GT_COLS;                            // 224 or 96
  static constexpr int MN = DIG == 7 ? 256 : 128;                    // operand rows with padding
  static constexpr uint32_t STAGE = MN / 8 * GT_SBO;                 // 64 KB or 32 KB per stage
  static constexpr uint32_t CONTRIB = DIG * GT_COLS * GT_COLS * 8;   // per-chunk partial sums
  static constexpr uint32_t TMEM_COLS = DIG == 7 ? 512 : 128;
  // instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major, N, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                                    ((uint32_t)(128 >> 4) << 24);
};

__device__ __forceinline__ uint32_t gt_saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: K-groups 128 B apart, 8-row groups GT_SBO apart
__device__ __forceinline__ uint64_t gt_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((GT_SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void gt_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// 8 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void gt_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// round(x 2^s) for |x 2^s| < 2^48, with integer operations only (ties away from zero)
__device__ __forceinline__ int64_t gt_fix(float x, int s) {
  const uint32_t u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xFF);
  if (e == 0) return 0;                                    // zero or subnormal: below 2^-126
  const int64_t mant = (int64_t)((u & 0x7FFFFFu) | 0x800000u);
  const int sh = e - 150 + s;
  int64_t r;
  if (sh >= 0) r = mant << min(sh, 40);
  else if (sh > -26) r = (mant + ((int64_t)1 << (-sh - 1))) >> (-sh);
  else r = 0;
  return (u >> 31) ? -r : r;
}

// the same for the low part of a float-float (|x 2^s| < 2^24): 32-bit shifts suffice
__device__ __forceinline__ int32_t gt_fix_lo(float x, int s) {
  const uint32_t u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xFF);
  const uint32_t mant = (u & 0x7FFFFFu) | 0x800000u;
  const int k = 150 - s - e;                               // right shift
  uint32_t r;
  if (k > 0) r = k < 25 ? (mant + (1u << (k - 1))) >> k : 0u;
  else r = mant << min(-k, 7);
  if (e == 0) r = 0;
  return (u >> 31) ? -(int32_t)r : (int32_t)r;
}

// float-float product (error-free by FMA)
__device__ __forceinline__ float2 gt_ffmul(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  return make_float2(p, e);
}

// exponent f with max |A_c| 2^-f in [1/2, 1) (0 for an all-zero column)
__device__ __forceinline__ int gt_colexp(unsigned bits) {
  if (!bits) return 0;
  int e;
  frexpf(__uint_as_float(bits), &e);
  return e;
}

// float of a small integer without a conversion instruction: (1.5 2^23 + d) - 1.5 2^23
__device__ __forceinline__ float gt_flt(int d) { return __fsub_rn(__int_as_float(0x4B400000 + d), 12582912.0f); }

// two small integers (|d| <= 64, exact in bf16) -> packed bf16 pair, d0 in the low half
__device__ __forceinline__ uint32_t gt_bf2(int d0, int d1) {
  return __byte_perm(__float_as_uint(gt_flt(d0)), __float_as_uint(gt_flt(d1)), 0x7632);
}

// the seven balanced base-128 digits of a (|a| < 2^47), in 32-bit arithmetic: four
// from the low 28 bits (their carry moves into the high part), three from the rest
__device__ __forceinline__ void gt_digits(int64_t a, int (&d)[7]) {
  uint32_t x = (uint32_t)a & 0x0FFFFFFFu;
  int32_t y = (int32_t)(a >> 28);
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int t = (int)((x & 127u) ^ 64u) - 64;   // in [-64, 63], = x mod 128
    d[q] = t;
    x = (uint32_t)((int32_t)x - t) >> 7;
  }
  y += (int32_t)x;                                  // carry 0 or 1
#pragma unroll
  for (int q = 4; q < 7; q++) {
    const int t = (int)(((uint32_t)y & 127u) ^ 64u) - 64;
    d[q] = t;
    y = (y - t) >> 7;
  }
}

// the three bf16 terms of a float-float value x + y: h = bf16(x), m = bf16((x - h) + y),
// l = bf16(that - m); returned as floats (exact in bf16)
__device__ __forceinline__ void gt_split3(float x, float y, float (&t)[3]) {
  const float h = __bfloat162float(__float2bfloat16_rn(x));
  const float r = __fadd_rn(__fsub_rn(x, h), y);
  const float m = __bfloat162float(__float2bfloat16_rn(r));
  t[0] = h;
  t[1] = m;
  t[2] = __bfloat162float(__float2bfloat16_rn(__fsub_rn(r, m)));
}

// two floats exact in bf16 -> packed bf16 pair, the first in the low half
__device__ __forceinline__ uint32_t gt_pack(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

}  // namespace

template <int DIG>
__global__ void __launch_bounds__(GT_THREADS, 1) k_gram_tc(const float *__restrict__ Uh, const float *__restrict__ Ul,
                                                           const float2 *__restrict__ rf, int64_t R, int k, int M,
                                                           const unsigned *__restrict__ amax, double *__restrict__ G,
                                                           int *status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((128u - (gt_saddr(smem_raw) & 127u)) & 127u);
  using Md = GtMode<DIG>;
  uint8_t *stage[2] = {smem, smem + Md::STAGE};
  double *contrib = (double *)(smem + 2 * Md::STAGE);         // [q][c][c']
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t chunks = (R + GT_CHUNK - 1) / GT_CHUNK;
  const int64_t items = chunks * M;

  // the padding operand rows (224..255, or 96..127) stay zero
  for (int i = tid; i < (int)(2 * Md::STAGE / 16); i += GT_THREADS) ((uint4 *)smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(gt_saddr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(gt_saddr(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(gt_saddr(&tmem_base)),
                 "r"(Md::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = tmem_base;

  uint32_t issued[2] = {0, 0}, waited[2] = {0, 0};   // commits per stage buffer, and completions seen
  int sbuf = 0;
  bool aborted = false;
  const int c = lane;            // conversion: column c, rows 8 warp .. 8 warp + 7 of the stage
  for (int64_t it = blockIdx.x; it < items && !aborted; it += gridDim.x) {
    const int m = (int)(it / chunks);
    const int64_t r0 = (it - (int64_t)m * chunks) * GT_CHUNK;
    const int64_t r1 = min(R, r0 + GT_CHUNK);
    const int s_c = c < k ? 47 - gt_colexp(amax[m * 32 + c]) : 0;
    const int nst = (int)((r1 - r0 + GT_KS - 1) / GT_KS);
    // this thread's inputs (rows 8 warp .. +7 of a stage, column c), fetched one stage
    // ahead so that the loads are in flight while the previous stage is converted
    float nh[8], nl[8];
    float2 nf[8];
    auto fetch = [&](int64_t rb) {
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const int64_t r = rb + 8 * warp + i;
        const bool ok = r < r1 && c < k;
        nh[i] = ok ? Uh[r * k + c] : 0.f;
        nl[i] = ok ? Ul[r * k + c] : 0.f;
        nf[i] = ok ? rf[r * M + m] : make_float2(0.f, 0.f);
      }
    };
    fetch(r0);
    for (int st = 0; st < nst; st++) {
      float uh[8], ul[8];
      float2 uf[8];
#pragma unroll
      for (int i = 0; i < 8; i++) { uh[i] = nh[i]; ul[i] = nl[i]; uf[i] = nf[i]; }
      if (st + 1 < nst) fetch(r0 + (int64_t)(st + 1) * GT_KS);
      // the buffer's previous MMAs must be done before it is rewritten
      if (issued[sbuf] > waited[sbuf]) {
        if (!cta_wait_bounded(gt_saddr(&mbar[sbuf]), waited[sbuf] & 1)) { aborted = true; break; }
        waited[sbuf]++;
      }
      uint32_t pk[DIG][4];
      if constexpr (DIG == 7) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          int d0[DIG], d1[DIG];
          {
            const float2 v0 = gt_ffmul(uh[i], ul[i], uf[i].x, uf[i].y);
            const float2 v1 = gt_ffmul(uh[i + 1], ul[i + 1], uf[i + 1].x, uf[i + 1].y);
            gt_digits(gt_fix(v0.x, s_c) + gt_fix_lo(v0.y, s_c), d0);   // rows past the end hold zeros
            gt_digits(gt_fix(v1.x, s_c) + gt_fix_lo(v1.y, s_c), d1);
          }
#pragma unroll
          for (int q = 0; q < DIG; q++) pk[q][i >> 1] = gt_bf2(d0[q], d1[q]);
        }
      } else {
        // A = (U hi + lo)(rowfactor hi + lo) 2^-f as a float-float, then its three bf16 terms
        const float sc = __uint_as_float((uint32_t)(127 + s_c - 47) << 23);   // 2^-f, exact
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          float t0[3], t1[3];
          const float2 v0 = gt_ffmul(uh[i], ul[i], uf[i].x, uf[i].y);
          const float2 v1 = gt_ffmul(uh[i + 1], ul[i + 1], uf[i + 1].x, uf[i + 1].y);
          gt_split3(__fmul_rn(v0.x, sc), __fmul_rn(v0.y, sc), t0);
          gt_split3(__fmul_rn(v1.x, sc), __fmul_rn(v1.y, sc), t1);
#pragma unroll
          for (int q = 0; q < DIG; q++) pk[q][i >> 1] = gt_pack(t0[q], t1[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < DIG; q++) {
        const int mn = q * GT_COLS + c;
        *(uint4 *)(stage[sbuf] + (mn >> 3) * GT_SBO + warp * 128 + (mn & 7) * 16) =
            make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        const uint32_t base = gt_saddr(stage[sbuf]);
#pragma unroll
        for (int ks = 0; ks < GT_KS / 16; ks++) {
          const uint64_t b = gt_desc(base + ks * 256);
          const uint32_t acc = (st | ks) != 0;
          gt_mma(tmem, gt_desc(base + ks * 256), b, Md::IDESC, acc);                  // rows 0..127
          if constexpr (DIG == 7)
            gt_mma(tmem + 256, gt_desc(base + 16 * GT_SBO + ks * 256), b, Md::IDESC, acc);   // rows 128..255
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            gt_saddr(&mbar[sbuf])));
      }
      issued[sbuf]++;
      sbuf ^= 1;
    }
    if (aborted) break;
    // every MMA of the chunk is complete once both buffers' commits have arrived
    for (int b = 0; b < 2 && !aborted; b++) {
      if (issued[b] > waited[b]) {
        if (!cta_wait_bounded(gt_saddr(&mbar[b]), waited[b] & 1)) aborted = true;
        else waited[b]++;
      }
    }
    if (aborted) break;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if constexpr (DIG == 7) {
      // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 of D1 (w % 8 < 4) or D2:
      // operand row 32 q + c with q = w % 8 (D1) or 4 + w % 4 (D2), c = lane; warps w and
      // w + 8 share the lanes and split the 8-column blocks
      const int w8 = warp & 7, quarter = w8 & 3, q = w8 < 4 ? w8 : 4 + quarter;
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (w8 < 4 ? 0u : 256u);
      if (q < DIG) {
#pragma unroll 1
        for (int cb = warp < 8 ? 0 : 2; cb < (warp < 8 ? 2 : 4); cb++) {
          float v[DIG][8];
#pragma unroll
          for (int qq = 0; qq < DIG; qq++) gt_ld8(tbase + qq * GT_COLS + cb * 8, v[qq]);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
          for (int j = 0; j < 8; j++) {
            // sum_q' 128^q' P_q' = lo + 2^28 hi, each part exact in 64 bits (|P| <= 2^24)
            int64_t lo = 0, hi = 0;
#pragma unroll
            for (int qq = 0; qq < 4; qq++) lo += (int64_t)__float2int_rn(v[qq][j]) << (7 * qq);
#pragma unroll
            for (int qq = 4; qq < DIG; qq++) hi += (int64_t)__float2int_rn(v[qq][j]) << (7 * (qq - 4));
            const double val = fma((double)hi, 268435456.0, (double)lo);
            contrib[(q * GT_COLS + c) * GT_COLS + cb * 8 + j] = ldexp(val, 7 * q - 94);
          }
        }
      }
    } else {
      // epilogue: warp w reads TMEM lanes 32 q .. +31 (q = w % 4: operand row 32 q + c of
      // term q, c = lane) and the columns 32 q' + 8 cb .. +7 (cb = w / 4) of the three
      // terms q'; their sum is row (q, c) of the term-pair sums, columns 8 cb ..
      const int q = warp & 3, cb = warp >> 2;
      if (q < DIG) {
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16);
        float v[DIG][8];
#pragma unroll
        for (int qq = 0; qq < DIG; qq++) gt_ld8(tbase + qq * GT_COLS + cb * 8, v[qq]);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
        for (int j = 0; j < 8; j++) {
          double val = 0;
#pragma unroll
          for (int qq = 0; qq < DIG; qq++) val += (double)v[qq][j];
          contrib[(q * GT_COLS + c) * GT_COLS + cb * 8 + j] = val;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();   // TMEM read (the next chunk's MMAs overwrite it) and contrib complete
    for (int e = tid; e < GT_COLS * GT_COLS; e += GT_THREADS) {
      const int a = e / GT_COLS, b = e - a * GT_COLS;
      if (a <= b && b < k) {
        double s = 0;
#pragma unroll
        for (int qq = 0; qq < DIG; qq++) s += contrib[qq * GT_COLS * GT_COLS + e];
        atomicAdd(&G[((int64_t)m * 32 + a) * 32 + b], s);
      }
    }
    __syncthreads();   // contrib reused by the next chunk
  }
  if (aborted) {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
    // let the MMAs in flight finish before TMEM is freed (bounded)
    for (int b = 0; b < 2; b++)
      if (issued[b] > waited[b]) cta_wait_bounded(gt_saddr(&mbar[b]), waited[b] & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(Md::TMEM_COLS));
}

template <int DIG>
static cudaError_t launch_mode(const float *Uh, const float *Ul, const float2 *rf, int64_t R, int k, int M,
                               const unsigned *amax, double *G, int *status, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t items = ((R + GT_CHUNK - 1) / GT_CHUNK) * M;
  const int grid = (int)std::min<int64_t>(sms, items);
  const size_t sm = 2 * GtMode<DIG>::STAGE + GtMode<DIG>::CONTRIB + 128;
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc<DIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_gram_tc<DIG><<<grid, GT_THREADS, sm, st>>>(Uh, Ul, rf, R, k, M, amax, G, status);
  return cudaGetLastError();
}

cudaError_t launch_gram_tc(const float *Uh, const float *Ul, const float2 *rf, int64_t R, int k, int M,
                           const unsigned *amax, double *G, int exact, int *status, cudaStream_t st) {
  if (R <= 0 || M <= 0) return cudaSuccess;
  return exact ? launch_mode<7>(Uh, Ul, rf, R, k, M, amax, G, status, st)
               : launch_mode<3>(Uh, Ul, rf, R, k, M, amax, G, status, st);
}

}  // namespace pmd
