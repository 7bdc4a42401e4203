// Reduced-precision prediction on the fifth-generation tensor cores:
//   T = F W^T   (F int64 [R][32] counts, W fp64 [M <= 64][32] weights)   (Sec. 2)
//
// Each count and each weight is rounded to FP32 (24 bits) and split exactly into
// three bf16 parts, x = x1 + x2 + x3.  The six products x1 y1, x1 y2, x2 y1, x1 y3,
// x2 y2, x3 y1 carry every term down to 2^-24 of |x y|; they are issued as 12
// tcgen05.mma instructions (M = 128 rows, N = 64 models, K = 16) accumulating in
// FP32 in tensor memory.  Relative error <= ~2^-21 of sum_i |F_ri W_mi|.
//
// One CTA (8 warps) owns a 128-row tile at a time (persistent over tiles).  Row tiles
// (32 KB of contiguous counts) are streamed into shared memory by the bulk-copy
// engine (cp.async.bulk, mbarrier transaction counts), double-buffered, so the next
// tile arrives while the current one is converted and multiplied.  The
// int64 -> float conversion uses integer operations and FP32 adds only (the
// 64-bit conversion instructions run on the FP64 pipe of this GPU).  Operands are
// written to shared memory in the no-swizzle K-major core-matrix layout (8 rows x
// 16 bytes per core matrix), made visible to the tensor core with a proxy fence,
// and the MMAs are issued by one thread and committed to an mbarrier.  Every
// mbarrier wait is bounded; on timeout the kernel records ST_TIMEOUT and stops.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "eval_common.cuh"
#include "kernels.h"
#include "mbar_wait.cuh"

namespace pmd {

constexpr int TC_ROWS = 128;      // MMA M
constexpr int TC_N = 64;          // MMA N (models, padded)
constexpr int TC_K = 32;          // features
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_A_BYTES = TC_ROWS * TC_K * 2;   // one bf16 split of a row tile: 8 KB
constexpr uint32_t TC_B_BYTES = TC_N * TC_K * 2;      // one bf16 split of the weights: 4 KB
constexpr uint32_t TC_F_BYTES = TC_ROWS * TC_K * 8;   // one raw row tile of counts: 32 KB

// instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major, N = 64, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_ROWS >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in the no-swizzle K-major layout: core matrices of
// 8 rows x 8 elements (128 B), the 4 k-groups of a row group contiguous (LBO = 128 B),
// row groups 512 B apart (SBO = 512 B)
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;   // leading (K) byte offset
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;   // stride (M/N) byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  return d;
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate));
}

// Exact float -> double bit pattern with integer operations (the conversion
// instruction would run on the FP64 pipe).
__device__ __noinline__ double f32_to_f64_rare(float f) {   // zero, subnormal, inf, nan
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xFF, m = u & 0x7FFFFF;
  uint64_t bits;
  if (e == 0xFF) bits = sign | (0x7FFull << 52) | ((uint64_t)m << 29);   // inf / nan
  else if (m == 0) bits = sign;                                          // zero
  else {                                                                  // subnormal float
    const int lz = __clz(m) - 8;                                          // leading zeros in 23 bits
    bits = sign | ((uint64_t)(897 - lz - 1) << 52) | ((uint64_t)((m << (lz + 1)) & 0x7FFFFF) << 29);
  }
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f), mag = u & 0x7FFFFFFFu;
  if (mag - 0x00800000u < 0x7F000000u) {   // normal: exponent rebias 1023 - 127 = 896
    const uint32_t hi = (u & 0x80000000u) | ((mag >> 3) + 0x38000000u);
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  return f32_to_f64_rare(f);
}

// TMEM 16 lanes x 256 bits, 4 repetitions along the columns: thread t holds lanes
// t/4 and t/4 + 8, columns 8 j + 2 (t%4) and 8 j + 2 (t%4) + 1 of repetition j as
// v[4 j + {0, 1}] (lane t/4) and v[4 j + {2, 3}] (lane t/4 + 8).
__device__ __forceinline__ void tmem_ld16x256(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Exact 23-bit chunks to float without conversion instructions: (2^23 + x) as float minus 2^23.
__device__ __forceinline__ float chunk_to_float(uint32_t x) {
  return __fsub_rn(__uint_as_float(0x4B000000u | x), 8388608.0f);
}

// int64 -> float with |error| <= 2^-23 |v|, using integer ops and FP32 arithmetic only.
// v = c2 2^46 + c1 2^23 + c0 with c0, c1 in [0, 2^23) and c2 = v >> 46 signed; each part
// converts exactly.  s = c2 2^23 + c1 is exact whenever |s| < 2^24, which covers every
// case where the final sum s 2^23 + c0 cancels (s in {-1, 0}); otherwise both roundings
// are relative to a value >= 2^47.
__device__ __forceinline__ float i64_to_float(int64_t v) {
  const uint32_t lo = (uint32_t)v;
  const int32_t hi = (int32_t)(v >> 32);
  const float c0 = chunk_to_float(lo & 0x7FFFFFu);
  const float c1 = chunk_to_float(__funnelshift_r(lo, (uint32_t)hi, 23) & 0x7FFFFFu);
  const float c2 = __fsub_rn(__int_as_float(0x4B400000 + (hi >> 14)), 12582912.0f);   // 1.5 * 2^23
  return __fmaf_rn(__fmaf_rn(c2, 8388608.0f, c1), 8388608.0f, c0);
}

// Tiled tensor copy of one 128-row tile of counts (box 16 x 2 x 128 int64 over the view
// F[R][2][16]) with the 128-byte swizzle; rows past R are zero-filled, and the
// transaction count is always the full box.
__device__ __forceinline__ void tile_load(uint32_t dst, const CUtensorMap *map, int32_t row0, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(TC_F_BYTES) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(dst),
      "l"((uint64_t)map), "r"(0), "r"(0), "r"(row0), "r"(mbar)
      : "memory");
}

// Byte offset of 16-byte chunk c (0..15) of row r in a swizzled tile: each 128-byte
// line (half row) has its chunk index XORed with the line index mod 8.
__device__ __forceinline__ uint32_t swz_chunk(int r, int c) {
  const int line = 2 * r + (c >> 3);
  return (uint32_t)(line * 128 + (((c & 7) ^ (line & 7)) << 4));
}

// packed bf16 pair -> the two floats (low half, high half)
__device__ __forceinline__ float bf_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf_hi(uint32_t p) { return __uint_as_float(p & 0xFFFF0000u); }

// two floats -> packed bf16 pair (round to nearest even), x in the low half
__device__ __forceinline__ uint32_t pack_bf2(float x, float y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *(const uint32_t *)&h;
}

// Two counts -> three packed bf16 pairs, exact splits x = x1 + x2 + x3 of their floats.
__device__ __forceinline__ void split_pair(longlong2 v, uint32_t &p1, uint32_t &p2, uint32_t &p3) {
  const float x = i64_to_float(v.x), y = i64_to_float(v.y);
  p1 = pack_bf2(x, y);
  const float rx = __fsub_rn(x, bf_lo(p1)), ry = __fsub_rn(y, bf_hi(p1));
  p2 = pack_bf2(rx, ry);
  p3 = pack_bf2(__fsub_rn(rx, bf_lo(p2)), __fsub_rn(ry, bf_hi(p2)));
}

// (value, row) pairs: the smaller value, the smaller row on ties
__device__ __forceinline__ bool vr_less(float a, int ra, float b, int rb) { return a < b || (a == b && ra < rb); }

// mode 0: write T (fp64 [R][M]);  mode 1: per-model running argmin -> part[blockIdx][M]
//
// Per tile: wait for the tile's counts, convert them into the three bf16 operand
// splits, issue the MMAs and the load of the CTA's next tile (the raw buffer is free
// once converted), wait for the MMAs, then the epilogue.  Several CTAs per SM overlap
// one another's loads, conversions and epilogues.  Warps w and w + 4 share TMEM lanes
// 32 (w % 4) .. +31 (rows of the tile); warp w < 4 takes accumulator columns (models)
// 0..31, warp w + 4 columns 32..63.
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_predict_tc(const __grid_constant__ CUtensorMap fmap, int64_t R,
                                                            const double *__restrict__ W, int M,
                                                            double *__restrict__ T, ArgPart *__restrict__ part,
                                                            int *status) {
  extern __shared__ uint8_t smem_raw[];
  // the swizzled tile needs a 1024-byte aligned destination
  uint8_t *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  uint8_t *sF = smem;                              // 32 KB raw row tile (swizzled)
  uint8_t *sA = smem + TC_F_BYTES;                 // 3 splits x 8 KB
  uint8_t *sB = sA + 3 * TC_A_BYTES;               // 3 splits x 4 KB
  __shared__ __align__(8) uint64_t mbar_mma, mbar_ld;
  __shared__ uint32_t tmem_base;
  __shared__ float fin_t[TC_THREADS];
  __shared__ int64_t fin_r[TC_THREADS];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (R + TC_ROWS - 1) / TC_ROWS;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar_mma)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar_ld)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&fmap) : "memory");
  }
  // weights: three bf16 splits, K-major, models >= M are zero
  for (int i = tid; i < TC_N * TC_K / 2; i += TC_THREADS) {
    const int n = i / (TC_K / 2), k = 2 * (i - n * (TC_K / 2));
    const float w0 = n < M ? __double2float_rn(W[(int64_t)n * TC_K + k]) : 0.f;
    const float w1 = n < M ? __double2float_rn(W[(int64_t)n * TC_K + k + 1]) : 0.f;
    const uint32_t p1 = pack_bf2(w0, w1);
    const float r0 = __fsub_rn(w0, bf_lo(p1)), r1 = __fsub_rn(w1, bf_hi(p1));
    const uint32_t p2 = pack_bf2(r0, r1);
    const uint32_t p3 = pack_bf2(__fsub_rn(r0, bf_lo(p2)), __fsub_rn(r1, bf_hi(p2)));
    const uint32_t o = kmajor_off(n, k);
    *(uint32_t *)(sB + o) = p1;
    *(uint32_t *)(sB + TC_B_BYTES + o) = p2;
    *(uint32_t *)(sB + 2 * TC_B_BYTES + o) = p3;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                 "r"(TC_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = tmem_base;
  if (tid == 0 && (int64_t)blockIdx.x < ntiles)
    tile_load(smem_addr(sF), &fmap, (int32_t)(blockIdx.x * TC_ROWS), smem_addr(&mbar_ld));

  const int half = warp >> 2, quarter = warp & 3;
  float best_t = __int_as_float(0x7f800000);   // argmin mode: model 32 half + lane over rows 32 quarter .. +31
  int64_t best_r = INT64_MAX;
  uint32_t ph_mma = 0, ph_ld = 0;
  bool aborted = false;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * TC_ROWS;
    if (!cta_wait_bounded(smem_addr(&mbar_ld), ph_ld)) { aborted = true; break; }
    ph_ld ^= 1;
    // operands: counts -> float -> three exact bf16 splits, 16-byte K-major core-matrix rows
    // warp w converts row groups w and w + 8 (8 rows x 4 k-groups each); lane i + 8 s takes
    // row i of the group and k-group (2 (i / 4) + s) mod 4, which keeps both the swizzled
    // reads and the operand stores of every quarter warp on distinct banks
#pragma unroll
    for (int j = 0; j < TC_ROWS * 4 / TC_THREADS; j++) {
      const int i = lane & 7, sq = lane >> 3;
      const int row = (warp + 8 * j) * 8 + i, kg = (2 * (i >> 2) + sq) & 3;   // 8 counts: chunks 4 kg .. 4 kg + 3
      uint32_t w1[4], w2[4], w3[4];
#pragma unroll
      for (int q = 0; q < 4; q++)
        split_pair(*(const longlong2 *)(sF + swz_chunk(row, 4 * kg + q)), w1[q], w2[q], w3[q]);
      const uint32_t o = kmajor_off(row, kg * 8);
      *(uint4 *)(sA + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
      *(uint4 *)(sA + TC_A_BYTES + o) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      *(uint4 *)(sA + 2 * TC_A_BYTES + o) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      // products x1y1, x1y2, x2y1, x1y3, x2y2, x3y1, each over K = 32 in two K = 16 steps
#pragma unroll
      for (int p = 0; p < 6; p++) {
        const int pa = p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0);
        const int pb = p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0);
#pragma unroll
        for (int kc = 0; kc < 2; kc++) {
          const uint64_t ad = sdesc(smem_addr(sA + pa * TC_A_BYTES + kc * 256));
          const uint64_t bd = sdesc(smem_addr(sB + pb * TC_B_BYTES + kc * 256));
          tc_mma(tmem, ad, bd, (p | kc) != 0);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(&mbar_mma)));
      // the raw tile is converted: stream in this CTA's next tile
      const int64_t next = tile + gridDim.x;
      if (next < ntiles) tile_load(smem_addr(sF), &fmap, (int32_t)(next * TC_ROWS), smem_addr(&mbar_ld));
    }
    if (!cta_wait_bounded(smem_addr(&mbar_mma), ph_mma)) { aborted = true; break; }
    ph_mma ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (MODE == 0) {
      // thread t: rows 16 s + t/4 and 16 s + t/4 + 8 of the warp's 32, column pairs
      // 8 j + 2 (t%4) of the warp's 32 columns; each warp store writes 8 rows x 64 bytes
      const int rq = lane >> 2, cq = 2 * (lane & 3);
      float vv[2][16];
      tmem_ld16x256(tmem + ((uint32_t)(quarter * 32) << 16) + half * 32, vv[0]);
      tmem_ld16x256(tmem + ((uint32_t)(quarter * 32 + 16) << 16) + half * 32, vv[1]);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
      for (int s = 0; s < 2; s++) {
        const float *v = vv[s];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int64_t row = r0 + quarter * 32 + 16 * s + rq + 8 * h;
          if (row < R) {
            if (M == TC_N) {
              double *out = T + row * TC_N + half * 32 + cq;
#pragma unroll
              for (int j = 0; j < 4; j++)
                *(double2 *)(out + 8 * j) = make_double2(f32_to_f64(v[4 * j + 2 * h]), f32_to_f64(v[4 * j + 2 * h + 1]));
            } else {
#pragma unroll
              for (int j = 0; j < 4; j++) {
                const int col = half * 32 + 8 * j + cq;
                if (col < M) T[row * M + col] = f32_to_f64(v[4 * j + 2 * h]);
                if (col + 1 < M) T[row * M + col + 1] = f32_to_f64(v[4 * j + 2 * h + 1]);
              }
            }
          }
        }
      }
    } else {
      // thread = row 32 quarter + lane; per column (model) the minimum over the warp's
      // rows by a butterfly that halves the columns each lane keeps: lane l ends with
      // column l.  Rows past R hold zero-filled counts and are masked to +inf.
      float acc[32];
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + half * 32, acc);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
      const bool live = r0 + quarter * 32 + lane < R;
      if (!live) {
#pragma unroll
        for (int c = 0; c < 32; c++) acc[c] = __int_as_float(0x7f800000);
      }
      float v[32];
#pragma unroll
      for (int c = 0; c < 32; c++) v[c] = acc[c];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;   // keeps the upper half of its columns
#pragma unroll
        for (int c = 0; c < o; c++) {
          const float send = up ? v[c] : v[c + o];
          const float keep = up ? v[c + o] : v[c];
          v[c] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
      }
      const float tmin = v[0];   // minimum of column `lane` over the warp's rows
      // rows of later tiles are larger: only a strictly smaller value improves
      const unsigned better = __ballot_sync(0xffffffffu, tmin < best_t);
      if (better) {
#pragma unroll
        for (int c = 0; c < 32; c++) {
          if (better & (1u << c)) {
            const float m = __shfl_sync(0xffffffffu, tmin, c);
            const unsigned hit = __ballot_sync(0xffffffffu, acc[c] == m);
            if (lane == c) { best_t = m; best_r = r0 + quarter * 32 + (__ffs(hit) - 1); }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();   // TMEM read before the next tile's MMAs overwrite it
  }
  if (aborted) {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
    // let a tile load still in flight land before the CTA exits (bounded)
    cta_wait_bounded(smem_addr(&mbar_ld), ph_ld);
  }
  if (MODE == 1 && !aborted) {
    // combine the four row quarters of each model, then publish this CTA's partial result
    const int model = half * 32 + lane;
    fin_t[quarter * TC_N + model] = best_t;
    fin_r[quarter * TC_N + model] = best_r;
    __syncthreads();
    if (tid < TC_N && tid < M) {
      float bt = fin_t[tid];
      int64_t br = fin_r[tid];
      for (int q = 1; q < 4; q++) {
        const float ot = fin_t[q * TC_N + tid];
        const int64_t orr = fin_r[q * TC_N + tid];
        if (ot < bt || (ot == bt && orr < br)) { bt = ot; br = orr; }
      }
      part[(int64_t)blockIdx.x * M + tid] = ArgPart{(double)bt, br};
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_N));
}

// raw tile + operand splits + 1 KB alignment slack: 69 KB, three CTAs per SM
static size_t tc_smem() { return TC_F_BYTES + 3 * TC_A_BYTES + 3 * TC_B_BYTES + 1024; }
constexpr int TC_CTAS_PER_SM = 3;

int tc_parts(int sms) { return sms * TC_CTAS_PER_SM; }
size_t tc_argmin_scratch_bytes(int M, int sms) { return (size_t)tc_parts(sms) * M * 16; }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

cudaError_t launch_predict_tc(const int64_t *F, int64_t R, int k, const double *W, int M, double *T, int64_t *arg,
                              double *mn, void *scratch, int sms, int *status, cudaStream_t st) {
  if (k != TC_K || M > TC_N || M <= 0 || R > INT32_MAX - TC_ROWS) return cudaErrorInvalidValue;
  if (((uintptr_t)F & 15) != 0) return cudaErrorMisalignedAddress;   // tensor copies need 16-byte alignment
  if (R == 0) {   // no rows: argmin is -1 with time +inf
    return arg ? launch_argmin_reduce(nullptr, 0, M, arg, mn, st) : cudaSuccess;
  }
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[3] = {16, 2, (cuuint64_t)R};
  const cuuint64_t strides[2] = {128, 256};   // bytes: half row, row
  const cuuint32_t box[3] = {16, 2, TC_ROWS};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, (void *)F, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int64_t ntiles = (R + TC_ROWS - 1) / TC_ROWS;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)tc_parts(sms)));
  const size_t sm = tc_smem();
  if (!arg) {
    cudaFuncSetAttribute(k_predict_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_predict_tc<0><<<grid, TC_THREADS, sm, st>>>(map, R, W, M, T, nullptr, status);
  } else {
    ArgPart *part = (ArgPart *)scratch;
    cudaFuncSetAttribute(k_predict_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_predict_tc<1><<<grid, TC_THREADS, sm, st>>>(map, R, W, M, nullptr, part, status);
    return launch_argmin_reduce(part, grid, M, arg, mn, st);
  }
  return cudaGetLastError();
}

}  // namespace pmd
