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
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "eval_common.cuh"
#include "kernels.h"

namespace pmd {

constexpr int TC_ROWS = 128;      // MMA M
constexpr int TC_N = 64;          // MMA N (models, padded)
constexpr int TC_K = 32;          // features
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_A_BYTES = TC_ROWS * TC_K * 2;   // one bf16 split of a row tile: 8 KB
constexpr uint32_t TC_B_BYTES = TC_N * TC_K * 2;      // one bf16 split of the weights: 4 KB
constexpr uint32_t TC_F_BYTES = TC_ROWS * TC_K * 8;   // one raw row tile of counts: 32 KB
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // give up an mbarrier wait after 2 s

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

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// Exact float -> double bit pattern with integer operations (the conversion
// instruction would run on the FP64 pipe).
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xFF, m = u & 0x7FFFFF;
  uint64_t bits;
  if (e == 0xFF) bits = sign | (0x7FFull << 52) | ((uint64_t)m << 29);          // inf / nan
  else if (e != 0) bits = sign | ((uint64_t)(e + 896) << 52) | ((uint64_t)m << 29);  // normal: 1023 - 127 = 896
  else if (m == 0) bits = sign;                                                   // zero
  else {                                                                           // subnormal float
    const int lz = __clz(m) - 8;                                                   // leading zeros in 23 bits
    bits = sign | ((uint64_t)(897 - lz - 1) << 52) | ((uint64_t)((m << (lz + 1)) & 0x7FFFFF) << 29);
  }
  return __longlong_as_double((long long)bits);
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

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// Bounded mbarrier wait shared by the whole CTA: returns true if every thread saw the
// phase complete within TC_WAIT_NS.
__device__ __forceinline__ bool cta_wait(uint32_t mbar, uint32_t parity) {
  int timed_out = 0;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try(mbar, parity)) {
    if (globaltimer() - t0 > TC_WAIT_NS) { timed_out = 1; break; }
  }
  return !__syncthreads_or(timed_out);
}

// packed bf16 pair -> the two floats (low half, high half)
__device__ __forceinline__ float bf_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf_hi(uint32_t p) { return __uint_as_float(p & 0xFFFF0000u); }

// two floats -> packed bf16 pair (round to nearest even), x in the low half
__device__ __forceinline__ uint32_t pack_bf2(float x, float y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *(const uint32_t *)&h;
}

// 8 consecutive counts -> three 16-byte vectors of exact bf16 splits (x = x1 + x2 + x3)
__device__ __forceinline__ void convert8(const int64_t *src, uint4 &o1, uint4 &o2, uint4 &o3) {
  uint32_t w1[4], w2[4], w3[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const longlong2 v = *(const longlong2 *)(src + 2 * q);
    const float x = i64_to_float(v.x), y = i64_to_float(v.y);
    w1[q] = pack_bf2(x, y);
    const float rx = __fsub_rn(x, bf_lo(w1[q])), ry = __fsub_rn(y, bf_hi(w1[q]));
    w2[q] = pack_bf2(rx, ry);
    w3[q] = pack_bf2(__fsub_rn(rx, bf_lo(w2[q])), __fsub_rn(ry, bf_hi(w2[q])));
  }
  o1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
  o2 = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  o3 = make_uint4(w3[0], w3[1], w3[2], w3[3]);
}

// mode 0: write T (fp64 [R][M]);  mode 1: per-model running argmin -> part[blockIdx][M]
//
// Warps w and w + 4 share TMEM lanes 32 (w % 4) .. +31 (rows of the tile); warp w < 4
// reads accumulator columns 0..31 (models), warp w + 4 columns 32..63.
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_predict_tc(const int64_t *__restrict__ F, int64_t R,
                                                            const double *__restrict__ W, int M,
                                                            double *__restrict__ T, double *__restrict__ part_t,
                                                            int64_t *__restrict__ part_r, int *status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sF = smem;                              // 2 x 32 KB raw row tiles
  uint8_t *sA = smem + 2 * TC_F_BYTES;             // 3 splits x 8 KB
  uint8_t *sB = sA + 3 * TC_A_BYTES;               // 3 splits x 4 KB
  __shared__ __align__(8) uint64_t mbar_mma, mbar_ld[2];
  __shared__ uint32_t tmem_base;
  __shared__ float fin_t[TC_THREADS];
  __shared__ int64_t fin_r[TC_THREADS];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

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
  const int64_t ntiles = (R + TC_ROWS - 1) / TC_ROWS;
  auto tile_bytes = [&](int64_t tile) { return (uint32_t)(min((int64_t)TC_ROWS, R - tile * TC_ROWS) * TC_K * 8); };
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar_mma)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar_ld[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar_ld[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
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
    bulk_load(smem_addr(sF), F + (int64_t)blockIdx.x * TC_ROWS * TC_K, tile_bytes(blockIdx.x), smem_addr(&mbar_ld[0]));

  float best_t = __int_as_float(0x7f800000);   // argmin mode: model tid % 64, rows 32 (tid / 64) .. +31
  int64_t best_r = INT64_MAX;
  uint32_t ph_mma = 0, ph_ld[2] = {0, 0};
  bool aborted = false;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
    const int buf = it & 1;
    const int64_t r0 = tile * TC_ROWS;
    // stream the next tile into the other buffer (its previous contents were consumed last iteration)
    const int64_t next = tile + gridDim.x;
    if (tid == 0 && next < ntiles)
      bulk_load(smem_addr(sF + (buf ^ 1) * TC_F_BYTES), F + next * TC_ROWS * TC_K, tile_bytes(next),
                smem_addr(&mbar_ld[buf ^ 1]));
    if (!cta_wait(smem_addr(&mbar_ld[buf]), ph_ld[buf])) { aborted = true; break; }
    ph_ld[buf] ^= 1;
    // operands: counts -> float -> three exact bf16 splits, 16-byte K-major core-matrix rows
    const int nrows = (int)min((int64_t)TC_ROWS, R - r0);
    const int64_t *src = (const int64_t *)(sF + buf * TC_F_BYTES);
#pragma unroll
    for (int j = 0; j < TC_ROWS * 4 / TC_THREADS; j++) {
      const int item = tid + j * TC_THREADS;
      const int row = item >> 2, kg = item & 3;
      uint4 o1 = make_uint4(0, 0, 0, 0), o2 = o1, o3 = o1;
      if (row < nrows) convert8(src + row * TC_K + kg * 8, o1, o2, o3);
      const uint32_t o = kmajor_off(row, kg * 8);
      *(uint4 *)(sA + o) = o1;
      *(uint4 *)(sA + TC_A_BYTES + o) = o2;
      *(uint4 *)(sA + 2 * TC_A_BYTES + o) = o3;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      // products x1y1, x1y2, x2y1, x1y3, x2y2, x3y1, each over K = 32 in two K = 16 steps
      const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
      uint32_t acc = 0;
#pragma unroll
      for (int p = 0; p < 6; p++)
#pragma unroll
        for (int kc = 0; kc < 2; kc++) {
          const uint64_t ad = sdesc(smem_addr(sA + pa[p] * TC_A_BYTES + kc * 256));
          const uint64_t bd = sdesc(smem_addr(sB + pb[p] * TC_B_BYTES + kc * 256));
          tc_mma(tmem, ad, bd, acc);
          acc = 1;
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(&mbar_mma)));
    }
    if (!cta_wait(smem_addr(&mbar_mma), ph_mma)) { aborted = true; break; }
    ph_mma ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    // epilogue: this thread's row and half of the models
    const int half = warp >> 2;
    float acc[32];
    tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + half * 32, acc);
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
    // per-warp 32 x 32 float block in the raw buffer of this tile (consumed), columns
    // XOR-swizzled by the row: row-wise writes and column-wise reads are conflict-free
    float *blk = (float *)(sF + buf * TC_F_BYTES) + warp * 1024;
#pragma unroll
    for (int c = 0; c < 32; c++) blk[lane * 32 + (c ^ lane)] = acc[c];
    __syncwarp();
    const int64_t wrow = r0 + (warp & 3) * 32;   // first row of this warp's block
    if (MODE == 0) {
      // coalesced T rows: half-warps write one 256-byte half row each
      if (M == TC_N) {
        const int cp = (lane & 15) * 2;
#pragma unroll 4
        for (int it = 0; it < 16; it++) {
          const int j = 2 * it + (lane >> 4);
          const float x = blk[j * 32 + (cp ^ j)], y = blk[j * 32 + ((cp + 1) ^ j)];
          if (wrow + j < R) *(double2 *)(T + (wrow + j) * TC_N + half * 32 + cp) = make_double2(f32_to_f64(x), f32_to_f64(y));
        }
      } else {
        const int col = half * 32 + lane;
#pragma unroll 4
        for (int j = 0; j < 32; j++)
          if (wrow + j < R && col < M) T[(wrow + j) * M + col] = f32_to_f64(blk[j * 32 + (lane ^ j)]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();   // TMEM read; blocks complete
    if (MODE == 1) {
      // model m = tid % 64 scans rows 32 q .. 32 q + 31 (the block of warp (q, m / 32))
      const int m = tid % TC_N, q = tid / TC_N;
      const float *col = (const float *)(sF + buf * TC_F_BYTES) + ((m >> 5) * 4 + q) * 1024;
      const int mc = m & 31, rb = q * 32;
      float bt = __int_as_float(0x7f800000);
      int bi = 0;
      if (rb + 32 <= nrows) {
#pragma unroll
        for (int j = 0; j < 32; j++) {   // rows in increasing order: the first minimum wins
          const float x = col[j * 32 + (mc ^ j)];
          const bool p = x < bt;
          bt = p ? x : bt;
          bi = p ? j : bi;
        }
      } else {
        for (int j = 0; j < nrows - rb; j++) {
          const float x = col[j * 32 + (mc ^ j)];
          if (x < bt) { bt = x; bi = j; }
        }
      }
      if (bt < best_t) { best_t = bt; best_r = r0 + rb + bi; }
    }
    // the raw buffer is refilled by the bulk-copy engine next iteration
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    __syncthreads();
  }
  if (aborted) {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
    // let any bulk copy still in flight land before the CTA exits (bounded)
    for (int b = 0; b < 2; b++) cta_wait(smem_addr(&mbar_ld[b]), ph_ld[b]);
  }
  if (MODE == 1 && !aborted) {
    // combine the four row ranges of each model, then publish this CTA's partial result
    fin_t[tid] = best_t;
    fin_r[tid] = best_r;
    __syncthreads();
    if (tid < TC_N && tid < M) {
      for (int q = 1; q < TC_THREADS / TC_N; q++) {
        const float ot = fin_t[q * TC_N + tid];
        const int64_t orr = fin_r[q * TC_N + tid];
        if (ot < best_t || (ot == best_t && orr < best_r)) { best_t = ot; best_r = orr; }
      }
      part_t[(int64_t)blockIdx.x * M + tid] = (double)best_t;
      part_r[(int64_t)blockIdx.x * M + tid] = best_r;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_N));
}

__global__ void k_argmin_tc_reduce(const double *__restrict__ pt, const int64_t *__restrict__ pr, int n_part, int M,
                                   int64_t *arg, double *mn) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double bt = __longlong_as_double(0x7ff0000000000000ll);
  int64_t br = INT64_MAX;
  for (int p = 0; p < n_part; p++) {
    const double t = pt[(int64_t)p * M + m];
    const int64_t r = pr[(int64_t)p * M + m];
    if (t < bt || (t == bt && r < br)) { bt = t; br = r; }
  }
  arg[m] = br == INT64_MAX ? -1 : br;
  mn[m] = bt;
}

static size_t tc_smem(int) { return 2 * TC_F_BYTES + 3 * TC_A_BYTES + 3 * TC_B_BYTES + 1024; }

// two resident CTAs per SM (101 KB of shared memory each)
int tc_parts(int sms) { return sms * 2; }
static int tc_grid(int, int sms) { return sms * 2; }
size_t tc_argmin_scratch_bytes(int M, int sms) { return (size_t)tc_parts(sms) * M * 16; }

cudaError_t launch_predict_tc(const int64_t *F, int64_t R, int k, const double *W, int M, double *T, int64_t *arg,
                              double *mn, void *scratch, int sms, int *status, cudaStream_t st) {
  if (k != TC_K || M > TC_N || M <= 0) return cudaErrorInvalidValue;
  if (((uintptr_t)F & 15) != 0) return cudaErrorMisalignedAddress;   // bulk copies need 16-byte alignment
  if (R == 0) {   // no rows: argmin is -1 with time +inf
    if (arg) k_argmin_tc_reduce<<<(M + 63) / 64, 64, 0, st>>>(nullptr, nullptr, 0, M, arg, mn);
    return cudaGetLastError();
  }
  const int64_t ntiles = (R + TC_ROWS - 1) / TC_ROWS;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)tc_grid(arg ? 1 : 0, sms)));
  if (!arg) {
    const size_t sm = tc_smem(0);
    cudaFuncSetAttribute(k_predict_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_predict_tc<0><<<grid, TC_THREADS, sm, st>>>(F, R, W, M, T, nullptr, nullptr, status);
  } else {
    const size_t sm = tc_smem(1);
    double *pt = (double *)scratch;
    int64_t *pr = (int64_t *)((char *)scratch + (size_t)tc_parts(sms) * M * 8);
    cudaFuncSetAttribute(k_predict_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_predict_tc<1><<<grid, TC_THREADS, sm, st>>>(F, R, W, M, nullptr, pt, pr, status);
    k_argmin_tc_reduce<<<(M + 63) / 64, 64, 0, st>>>(pt, pr, grid, M, arg, mn);
  }
  return cudaGetLastError();
}

}  // namespace pmd
