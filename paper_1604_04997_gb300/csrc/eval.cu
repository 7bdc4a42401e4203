// K1: materialised count evaluation (pm_eval_counts).
// K2: persistent fused evaluation -> FP64-accurate prediction -> top-k ranking
//     (pm_eval_predict_topk), the batched form of Sec. 2's re-evaluation of p_i(n)
//     over a tuning search space and of configuration selection (Sec. 6.1).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "eval_common.cuh"
#include "kernels.h"

namespace pmd {

// ------------------------------------------------------------------------------------ K1

constexpr int K1_THREADS = 128;

template <int K>
__global__ void __launch_bounds__(K1_THREADS) k_eval_counts(const uint32_t *__restrict__ arena,
                                                           const int64_t *__restrict__ tab_off,
                                                           const int64_t *__restrict__ points, int64_t n_points,
                                                           int P, int64_t *__restrict__ out, int *status) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t *sT = (uint32_t *)smem;                                   // table, <= 16 KB
  int64_t *stage = (int64_t *)(smem + pmt::MAX_TABLE_WORDS * 4);     // [threads][K+1]
  int64_t *slots = stage + K1_THREADS * (K + 1);                     // [24][threads]
  const int tid = threadIdx.x;
  const uint32_t *gT = arena + tab_off[blockIdx.y];
  const int words = (int)gT[pmt::H_WORDS];
  if (gT[pmt::H_MAGIC] != pmt::MAGIC || words > pmt::MAX_TABLE_WORDS || (int)gT[pmt::H_K] != K) {
    if (tid == 0) atomicOr(status, ST_BAD_TABLE);
    return;
  }
  for (int i = tid; i < words / 4; i += K1_THREADS) ((uint4 *)sT)[i] = ((const uint4 *)gT)[i];
  int64_t *row = stage + tid * (K + 1);
#pragma unroll
  for (int c = 0; c < K; c++) row[c] = 0;
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * K1_THREADS;
  const int64_t p = p0 + tid;
  if (p < n_points) {
    int32_t n[4];
    if (!point_in_box(sT, points + p * P, P, n)) {
      atomicOr(status, ST_OUT_OF_BOX);
    } else {
      bool ok = eval_table(
          sT, n, slots + tid, K1_THREADS,
          [&](int col, int64_t v) { if (col < K) row[col] = v; },
          [&](int col, int64_t v) { if (col < K) row[col] = v; });
      if (!ok) {
        atomicOr(status, ST_BAD_TABLE);
#pragma unroll
        for (int c = 0; c < K; c++) row[c] = 0;
      }
    }
  }
  __syncthreads();
  const int64_t nvalid = min((int64_t)K1_THREADS, n_points - p0);
  int64_t *dst = out + ((int64_t)blockIdx.y * n_points + p0) * K;
  const int total = (int)nvalid * K;
  for (int i = tid; i < total; i += K1_THREADS) {   // streaming stores: the rows are not reread
    int r = i / K, c = i - r * K;
    __stcs(dst + i, stage[r * (K + 1) + c]);
  }
}

size_t k1_smem_bytes(int K) {
  return (size_t)pmt::MAX_TABLE_WORDS * 4 + (size_t)K1_THREADS * (K + 1) * 8 +
         (size_t)pmt::MAX_SLOTS * K1_THREADS * 8;
}

cudaError_t launch_eval_counts(const uint32_t *arena, const int64_t *d_tab_off, int n_tables, const int64_t *points,
                               int64_t n_points, int P, int K, int64_t *out, int *status, cudaStream_t st) {
  if (n_points == 0 || n_tables == 0) return cudaSuccess;
  dim3 grid((unsigned)((n_points + K1_THREADS - 1) / K1_THREADS), (unsigned)n_tables);
  size_t sm = k1_smem_bytes(K);
  if (K == 32) {
    cudaFuncSetAttribute(k_eval_counts<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_eval_counts<32><<<grid, K1_THREADS, sm, st>>>(arena, d_tab_off, points, n_points, P, out, status);
  } else if (K == 12) {
    cudaFuncSetAttribute(k_eval_counts<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_eval_counts<12><<<grid, K1_THREADS, sm, st>>>(arena, d_tab_off, points, n_points, P, out, status);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ K2

constexpr int K2_TOPK = 16;
constexpr int TB_WORDS = 1024;  // per-warp staging buffer (4 KB), double-buffered
constexpr uint64_t OFF_MASK = (1ull << 40) - 1;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_all;\n" ::); }

// A += W * v (mod 2^128): W a 128-bit two's-complement weight (four 32-bit limbs),
// v a signed 64-bit slot value.  Twelve 32-bit multiply-adds in carry chains, then
// the sign correction of v (v = v_unsigned - 2^64 when negative).  Since the exact
// sum of all terms lies within +-2^124, the modular sum is that sum.
__device__ __forceinline__ void mac128(uint32_t (&A)[4], const uint4 &W, int64_t v) {
  const uint32_t s0 = (uint32_t)v, s1 = (uint32_t)((uint64_t)v >> 32);
  asm("mad.lo.cc.u32  %0, %4, %8, %0;\n\t"
      "madc.lo.cc.u32 %1, %5, %8, %1;\n\t"
      "madc.lo.cc.u32 %2, %6, %8, %2;\n\t"
      "madc.lo.u32    %3, %7, %8, %3;\n\t"
      "mad.hi.cc.u32  %1, %4, %8, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %8, %2;\n\t"
      "madc.hi.u32    %3, %6, %8, %3;\n\t"
      "mad.lo.cc.u32  %1, %4, %9, %1;\n\t"
      "madc.lo.cc.u32 %2, %5, %9, %2;\n\t"
      "madc.lo.u32    %3, %6, %9, %3;\n\t"
      "mad.hi.cc.u32  %2, %4, %9, %2;\n\t"
      "madc.hi.u32    %3, %5, %9, %3;\n\t"
      : "+r"(A[0]), "+r"(A[1]), "+r"(A[2]), "+r"(A[3])
      : "r"(W.x), "r"(W.y), "r"(W.z), "r"(W.w), "r"(s0), "r"(s1));
  if (v < 0) {
    asm("sub.cc.u32 %0, %0, %2;\n\tsubc.u32 %1, %1, %3;\n\t" : "+r"(A[2]), "+r"(A[3]) : "r"(W.x), "r"(W.y));
  }
}

// Fill the 128-bit slot weights of the K2 programs: Weff = sum over contributions of
// W_col * coef, with W_col = round(w_col 2^E) the fixed-point weights (|W| < 2^56).
__global__ void __launch_bounds__(128) k_k2_weights(uint32_t *__restrict__ prog, const uint4 *__restrict__ targets,
                                                    const uint4 *__restrict__ contrib, int n_targets,
                                                    const double *__restrict__ w) {
  __shared__ uint4 sW[32];   // each weight sign-extended to 128 bits
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double x = w[lane];
    double mx = fabs(x);
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0) frexp(mx, &e);
    const int64_t W = llrint(ldexp(x, 56 - e));
    const uint32_t sx = W < 0 ? 0xFFFFFFFFu : 0u;
    sW[lane] = make_uint4((uint32_t)W, (uint32_t)((uint64_t)W >> 32), sx, sx);
  }
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_targets; i += gridDim.x * blockDim.x) {
    const uint4 tg = targets[i];
    uint32_t A[4] = {0, 0, 0, 0};
    for (uint32_t c = 0; c < tg.z; c++) {
      const uint4 cb = contrib[tg.y + c];
      mac128(A, sW[cb.x & 31], (int64_t)((uint64_t)cb.z | ((uint64_t)cb.w << 32)));
    }
    *(uint4 *)(prog + tg.x) = make_uint4(A[0], A[1], A[2], A[3]);
  }
}

cudaError_t launch_k2_weights(uint32_t *prog, const uint4 *targets, const uint4 *contrib, int n_targets,
                              const double *w, cudaStream_t st) {
  const int grid = std::max(1, std::min(1024, (n_targets + 127) / 128));
  k_k2_weights<<<grid, 128, 0, st>>>(prog, targets, contrib, n_targets, w);
  return cudaGetLastError();
}

// Evaluate a K2 program (table + weight image) at n and return the exact fixed-point
// prediction S = sum_col W_col p_col(n) (128 bits).  Same values, pieces and products
// as eval_table; the column sums and the dot product are one pass over the piece's
// weighted slots, plus the held columns and post-ops.  Returns false on a malformed
// program.
__device__ __forceinline__ bool eval_dot(const uint32_t *__restrict__ T, const int32_t *n, int64_t *slots, int ss,
                                         Acc128 &S) {
  const int P = (int)T[pmt::H_NPARAMS];
  const int A = (int)T[pmt::H_NATOMS];
  const int NC = (int)T[pmt::H_NCONDS];
  if (P > 4 || P + A > pmt::MAX_VALUES || NC > pmt::MAX_CONDS) return false;
#pragma unroll
  for (int p = 0; p < 4; p++) {
    if (p < P) slots[p * ss] = n[p];
    slots[(pmt::HOLD_SLOT + p) * ss] = 0;
  }
  slots[pmt::CONST_SLOT * ss] = 1;
  const uint32_t *at = T + T[pmt::H_OFF_ATOMS];
  for (int a = 0; a < A; a++, at += pmt::ATOM_WORDS) {
    const uint4 q0 = *(const uint4 *)at, q1 = *(const uint4 *)(at + 4);
    int32_t num = (int32_t)q1.x;
    num += (int32_t)q0.x * n[0];
    if (P > 1) num += (int32_t)q0.y * n[1];
    if (P > 2) num += (int32_t)q0.z * n[2];
    if (P > 3) num += (int32_t)q0.w * n[3];
    slots[(P + a) * ss] = floor_div(num, q1.y, q1.z, (q1.w >> 8) & 0xFF, (q1.w >> 16) & 1);
  }
  uint32_t bits = 0;
  const uint32_t *cd = T + T[pmt::H_OFF_CONDS];
  for (int c = 0; c < NC; c++) {
    const int nt = (int)cd[0];
    int64_t s = ld64(cd + 1);
    for (int t = 0; t < nt; t++)
      s += (int64_t)(int32_t)cd[4 + 2 * t] * slots[min(cd[3 + 2 * t], (uint32_t)pmt::MAX_SLOTS - 1) * ss];
    bits |= (uint32_t)(s >= 0) << c;
    cd += 3 + 2 * nt;
  }
  const uint32_t *lut = T + T[pmt::H_OFF_LUT];
  const uint32_t piece = (lut[bits >> 2] >> (8 * (bits & 3))) & 0xFF;
  if (piece >= T[pmt::H_NPIECES]) return false;
  const uint4 pc = *(const uint4 *)(T + T[pmt::H_OFF_PIECES] + 4 * piece);
  if (P + A + pc.y > (uint32_t)pmt::MAX_PRODS) return false;
  const uint32_t *pr = T + T[pmt::H_OFF_PRODS] + pc.x;
  int64_t *dst = slots + (P + A) * ss;
  for (uint32_t j = 0; j < pc.y; j++, dst += ss) {
    const uint32_t w = pr[j];
    *dst = (int64_t)((uint64_t)slots[min(w & 0xFF, (uint32_t)pmt::MAX_SLOTS - 1) * ss] *
                     (uint64_t)slots[min((w >> 8) & 0xFF, (uint32_t)pmt::MAX_SLOTS - 1) * ss]);
  }
  const uint32_t I = (T[pmt::H_OFF_ENTRIES] + 3) & ~3u;
  const uint4 ip = *(const uint4 *)(T + I + 8 * piece), iq = *(const uint4 *)(T + I + 8 * piece + 4);
  const uint4 *dw = (const uint4 *)(T + ip.x);
  const uint32_t *ds = T + ip.z;
  const uint32_t d0 = ip.w;   // 1: the first weight belongs to the constant slot (value 1)
  uint32_t acc[4] = {0, 0, 0, 0};
  if (d0) {
    const uint4 c = dw[0];
    acc[0] = c.x; acc[1] = c.y; acc[2] = c.z; acc[3] = c.w;
  }
  for (uint32_t d = d0; d < ip.y; d++) mac128(acc, dw[d], slots[min(ds[d], (uint32_t)pmt::MAX_SLOTS - 1) * ss]);
  if (iq.w) {   // post-ops whose smaller operand depends on n
    const uint4 *hl = (const uint4 *)(T + iq.x);
    for (uint32_t h = 0; h < iq.y; h++) {
      const uint4 E = hl[h];
      const uint64_t coef = (uint64_t)E.z | ((uint64_t)E.w << 32);
      int64_t *hs = slots + (pmt::HOLD_SLOT + ((E.x >> 8) & 3)) * ss;
      *hs += (int64_t)(coef * (uint64_t)slots[min(E.x & 0xFF, (uint32_t)pmt::MAX_SLOTS - 1) * ss]);
    }
    const uint4 *pw = (const uint4 *)(T + iq.z);
    for (uint32_t q = 0; q < iq.w; q++) {
      const uint4 w = pw[2 * q];
      const uint32_t hw = pw[2 * q + 1].x;
      const int64_t va = slots[(pmt::HOLD_SLOT + (hw & 3)) * ss];
      const int64_t vb = slots[(pmt::HOLD_SLOT + ((hw >> 8) & 3)) * ss];
      mac128(acc, w, va < vb ? va : vb);
    }
  }
  S.lo = (uint64_t)acc[0] | ((uint64_t)acc[1] << 32);
  S.hi = (uint64_t)acc[2] | ((uint64_t)acc[3] << 32);
  if (T[pmt::H_DEN] != 1) {   // S = D * prediction exactly: shift by t, times d^-1 mod 2^128
    const uint32_t sh = T[pmt::H_DEN_SHIFT] & 63;
    const uint64_t lo = sh ? (S.lo >> sh) | (S.hi << (64 - sh)) : S.lo;
    const uint64_t hi = (uint64_t)((int64_t)S.hi >> sh);
    const uint64_t ilo = ld64(T + pmt::H_DEN_INV), ihi = ld64(T + pmt::H_DEN_INV + 2);
    S.lo = lo * ilo;
    S.hi = __umul64hi(lo, ilo) + lo * ihi + hi * ilo;
  }
  return true;
}

// A ranking entry packs the top 48 bits of the monotone key (sign, exponent and 40
// mantissa bits: 2^-40 relative resolution) above a 16-bit variant index, so one
// signed 64-bit comparison orders by (key, variant) and exact ties (duplicate
// variants) fall to the smaller index.  INT64_MAX marks an empty slot.
constexpr int64_t K2_EMPTY = INT64_MAX;
__device__ __forceinline__ int64_t pack_entry(int64_t key, int vid) {
  return (int64_t)(((uint64_t)(key >> 16) << 16) | (uint32_t)vid);
}
__device__ __forceinline__ int entry_vid(int64_t e) { return (int)(e & 0xFFFF); }
__device__ __forceinline__ int64_t entry_key(int64_t e) { return (int64_t)((uint64_t)e & ~0xFFFFull); }

// The 16 best entries of one point, sorted ascending.
struct TopK {
  int64_t k[K2_TOPK];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < K2_TOPK; q++) k[q] = K2_EMPTY;
  }
  __device__ __forceinline__ void insert(int64_t e) {
#pragma unroll
    for (int q = K2_TOPK - 1; q > 0; q--) k[q] = e < k[q - 1] ? k[q - 1] : (e < k[q] ? e : k[q]);
    if (e < k[0]) k[0] = e;
  }
};

// Merge n sorted lists of 16 (element (list, q) at list*stride_list + q*stride_q) for this lane.
template <int MAXN>
__device__ __forceinline__ void merge_lists(const int64_t *ks, int n, int stride_list, int stride_q, TopK &out) {
  int head[MAXN];
#pragma unroll
  for (int w = 0; w < MAXN; w++) head[w] = 0;
#pragma unroll
  for (int q = 0; q < K2_TOPK; q++) {
    int best = -1;
    int64_t bk = K2_EMPTY;
#pragma unroll
    for (int w = 0; w < MAXN; w++) {
      if (w < n && head[w] < K2_TOPK) {
        const int64_t xk = __ldcg(ks + w * stride_list + head[w] * stride_q);
        if (best < 0 || xk < bk) { best = w; bk = xk; }
      }
    }
#pragma unroll
    for (int w = 0; w < MAXN; w++) if (w == best) head[w]++;
    out.k[q] = bk;
  }
}

constexpr int K2_BUF = 4;  // buffered insertion candidates per lane

// One CTA takes a work unit (a chunk of NW*32 points of one template, a slice of its
// variants).  Each lane owns one point; all warps walk the slice's variants in order,
// the CTA staging each table once into shared memory (double-buffered cp.async, one
// barrier per variant) and reading it as warp-wide broadcasts.  Counts are exact; the
// predicted time is the exact fixed-point sum S = sum_i count_i W_i (128-bit, integer
// pipes only), ranked by a monotone 64-bit key.  Each lane keeps its point's 16 best
// (key, variant) pairs in registers; candidates that beat the lane's 16th key are
// buffered and inserted together when some lane's buffer fills, so the divergent
// insertion path runs rarely.  A chunk split into S variant slices is finished by the
// last of its S units (partial lists in a scratch buffer, a fence and an atomic
// counter; no waiting).
// Launch bounds ask for 24 / NW CTAs per SM (at most 80 registers a thread): with the
// 37 KB of shared memory a 4-warp CTA takes, six CTAs fit, one more than the register
// use of an unbounded build allows.
template <int NW>
__global__ void __launch_bounds__(NW * 32, 24 / NW) k_eval_predict_topk(K2Args a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t *tbuf = (uint32_t *)smem;                                  // [2][TB_WORDS]
  int64_t *slots = (int64_t *)(tbuf + 2 * TB_WORDS);                  // [NW][24 slots][32 lanes]
  int64_t *bk = slots + NW * pmt::MAX_SLOTS * 32;                     // [NW][K2_BUF][32] candidate entries
  __shared__ int s_E, s_unit;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t *myslots = slots + warp * pmt::MAX_SLOTS * 32 + lane;
  int64_t *mybk = bk + warp * K2_BUF * 32 + lane;

  if (threadIdx.x == 0) s_E = weight_exponent(a.w, 32);   // the programs' weights are round(w 2^E)
  __syncthreads();

  while (true) {
    if (threadIdx.x == 0) s_unit = atomicAdd(a.unit_counter, 1);
    __syncthreads();
    const int u = s_unit;
    __syncthreads();
    if (u >= a.n_units) break;
    const int4 U = a.units[u];          // chunk, slice, first variant, end variant
    const int4 C = a.chunks[U.x];       // template, first point, point count, first partial slot
    const int t = C.x;
    const int S = a.tmpl_slices[t];
    const int P = a.tmpl_nparams[t];
    const int pl = warp * 32 + lane;    // this lane's point within the chunk
    const int64_t p = (int64_t)C.y + pl;
    const bool live = pl < C.z;         // the lane has a point
    bool valid = live;                  // ... inside the box (else its ranking stays empty)
    int32_t n[4] = {0, 0, 0, 0};
    if (live) {
      const int64_t *src = a.points + p * 4;
      const int4 lo = a.tmpl_box[2 * t], hi = a.tmpl_box[2 * t + 1];
      const int l4[4] = {lo.x, lo.y, lo.z, lo.w}, h4[4] = {hi.x, hi.y, hi.z, hi.w};
      bool ok = true;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if (q < P) {
          const int64_t x = src[q];
          ok = ok && x >= l4[q] && x <= h4[q];
          n[q] = (int32_t)x;
        }
      }
      if (!ok) { atomicOr(a.status, ST_OUT_OF_BOX); valid = false; }
    }
    TopK tk;
    tk.init();
    // Candidates of this unit arrive in increasing variant order, so one passes iff
    // its 48-bit key is below the 16th entry's: thr is that key (low 16 bits clear),
    // and for thr > 0 the exact test is S < key_floor(thr).
    int64_t thr = entry_key(K2_EMPTY);
    Acc128 thr_s = {~0ull, (uint64_t)INT64_MAX};
    int nbuf = 0;
    auto flush = [&]() {
      for (int b = 0; b < nbuf; b++) tk.insert(mybk[b * 32]);
      nbuf = 0;
      thr = entry_key(tk.k[K2_TOPK - 1]);
      if (tk.k[K2_TOPK - 1] == K2_EMPTY) { thr_s.lo = ~0ull; thr_s.hi = (uint64_t)INT64_MAX; }
      else if (thr > 0) thr_s = key_floor(thr);
    };
    const int v0 = a.var_off[t];
    const int vb = U.z, ve = U.w;
    auto stage = [&](int vv, int buf) {
      if (vv < ve) {
        const uint64_t po = a.tab_off[vv];
        const int words = min((int)(po >> 40), TB_WORDS);
        const uint32_t *g = a.prog + (po & OFF_MASK);
        for (int i = threadIdx.x; i < words / 4; i += NW * 32) cp_async16(tbuf + buf * TB_WORDS + 4 * i, g + 4 * i);
      }
      cp_async_commit();
    };
    stage(vb, 0);
    for (int v = vb; v < ve; v++) {
      const int buf = (v - vb) & 1;
      cp_async_wait0();
      __syncthreads();                  // table v visible; table v-1 no longer read by any warp
      stage(v + 1, buf ^ 1);            // overlaps with the evaluation of table v
      if (valid) {
        Acc128 S;
        if (!eval_dot(tbuf + buf * TB_WORDS, n, myslots, 32, S)) {
          atomicOr(a.status, ST_BAD_TABLE);
          S.lo = ~0ull;
          S.hi = (uint64_t)INT64_MAX;
        }
        // strict: an equal key of a later variant ranks after the earlier one
        const bool pass = thr > 0 ? acc_less(S, thr_s) : entry_key(pack_entry(acc_key(S), 0)) < thr;
        if (pass) {
          mybk[nbuf * 32] = pack_entry(acc_key(S), v - v0);
          nbuf++;
        }
      }
      if (__any_sync(0xffffffffu, nbuf == K2_BUF)) flush();
    }
    flush();
    cp_async_wait0();
    bool write_out = S == 1;
    if (S > 1) {
      // publish this slice's lists, then the last slice of the chunk merges all of them
      const int64_t slot0 = (int64_t)(C.w + U.y) * K2_TOPK * (NW * 32) + pl;
#pragma unroll
      for (int q = 0; q < K2_TOPK; q++) a.part_k[slot0 + q * (NW * 32)] = tk.k[q];
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_unit = atomicAdd(a.chunk_count + U.x, 1) == S - 1;
      __syncthreads();
      if (s_unit) {
        __threadfence();
        const int64_t b = (int64_t)C.w * K2_TOPK * (NW * 32) + pl;
        merge_lists<K2_MAX_SLICES>(a.part_k + b, S, K2_TOPK * (NW * 32), NW * 32, tk);
        write_out = true;
      }
    }
    if (write_out && live) {
      int32_t *oi = a.top_idx + p * a.topk;
      double *ot = a.top_t + p * a.topk;
      const int E = s_E;
#pragma unroll
      for (int q = 0; q < K2_TOPK; q++) {
        if (q < a.topk) {
          const bool real = tk.k[q] != K2_EMPTY;
          oi[q] = real ? entry_vid(tk.k[q]) : -1;
          ot[q] = real ? key_value(entry_key(tk.k[q]), E) : __longlong_as_double(0x7ff0000000000000ll);
        }
      }
    }
    __syncthreads();
  }
}

int k2_table_words() { return TB_WORDS; }

size_t k2_smem_bytes(int nw) {
  return (size_t)2 * TB_WORDS * 4 + (size_t)nw * pmt::MAX_SLOTS * 32 * 8 + (size_t)nw * K2_BUF * 32 * 8;
}

int k2_points_per_cta(int nw) { return nw * 32; }

cudaError_t launch_eval_predict_topk(const K2Args &args, int nw, int grid, cudaStream_t st) {
  size_t sm = k2_smem_bytes(nw);
  if (nw == 8) {
    cudaFuncSetAttribute(k_eval_predict_topk<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_eval_predict_topk<8><<<grid, 8 * 32, sm, st>>>(args);
  } else if (nw == 4) {
    cudaFuncSetAttribute(k_eval_predict_topk<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_eval_predict_topk<4><<<grid, 4 * 32, sm, st>>>(args);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int k2_max_blocks_per_sm(int nw) {
  int nb = 0;
  size_t sm = k2_smem_bytes(nw);
  if (nw == 8) {
    cudaFuncSetAttribute(k_eval_predict_topk<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval_predict_topk<8>, 8 * 32, sm);
  } else {
    cudaFuncSetAttribute(k_eval_predict_topk<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval_predict_topk<4>, 4 * 32, sm);
  }
  return nb;
}

}  // namespace pmd
