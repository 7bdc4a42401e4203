// Fused evaluation -> FP64-accurate prediction -> top-k ranking over a tuning space
// (pm_eval_predict_topk): the batched form of Sec. 2's re-evaluation of the properties
// p_i(n) of many kernel variants at many parameter points, contracted with one weight
// vector (sum_i alpha_i p_i) and ranked for configuration selection (Sec. 6.1).
//
// Work unit = (32 points of one template, one ranking group of its variants); one CTA
// of NW warps per unit, one point per lane, every warp on the same 32 points:
//   1. stage the group's image (basis definitions, conditions, programs, variant map)
//      in shared memory;
//   2. evaluate the group's basis (parameters, atoms floor((a.n + b)/c), monomials, in
//      dependency levels) and its piece conditions once per point;
//   3. each warp walks every NW-th variant: the piece from the condition bits, then the
//      exact fixed-point prediction S = sum_term Weff_term * basis_term (128 bits), the
//      runtime min(loads, stores) post-ops and the exact division by the table's
//      denominator; a candidate that beats the lane's threshold is buffered and the
//      buffers are inserted into register-resident sorted lists of 16 when one fills;
//   4. the warps share their 16th entries through shared memory (any warp's 16th
//      entry bounds the unit's final 16th), then merge their lists.
// A chunk whose template is split into several groups is finished by the last of its
// units (partial lists in scratch, a fence and an atomic counter; no waiting).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "eval_common.cuh"
#include "kernels.h"

namespace pmd {

constexpr int RK_TOPK = 16;
constexpr int RK_BUF = 4;                   // buffered insertion candidates per lane
constexpr int RK_EXCHANGE = 16;             // variants of a warp between threshold exchanges
constexpr int64_t RK_EMPTY = INT64_MAX;     // an empty list entry

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_all;\n" ::); }

// A += W * v (mod 2^128): W a 128-bit two's-complement weight (four 32-bit limbs), v a
// signed 64-bit value.  Twelve 32-bit multiply-adds in carry chains, then the sign
// correction of v (v = v_unsigned - 2^64 when negative).  The exact sum of all terms
// of one prediction lies within +-2^124 (weights with sum |W| <= 2^62, counts times
// the table's denominator below 2^62), so the modular sum is that sum.
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

// A += W * s (mod 2^128) for an unsigned 32-bit value s: seven multiply-adds.
__device__ __forceinline__ void mac128_u32(uint32_t (&A)[4], const uint4 &W, uint32_t s) {
  asm("mad.lo.cc.u32  %0, %4, %8, %0;\n\t"
      "madc.lo.cc.u32 %1, %5, %8, %1;\n\t"
      "madc.lo.cc.u32 %2, %6, %8, %2;\n\t"
      "madc.lo.u32    %3, %7, %8, %3;\n\t"
      "mad.hi.cc.u32  %1, %4, %8, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %8, %2;\n\t"
      "madc.hi.u32    %3, %6, %8, %3;\n\t"
      : "+r"(A[0]), "+r"(A[1]), "+r"(A[2]), "+r"(A[3])
      : "r"(W.x), "r"(W.y), "r"(W.z), "r"(W.w), "r"(s));
}

// Fill the 128-bit term weights of the ranking programs: Weff = sum over contributions
// of W_col * coef, with W_col = round(w_col 2^E) the fixed-point weights (sum |W| <=
// 2^62, so with counts D * p_col < 2^62 a program's sum stays within +-2^124).
__global__ void __launch_bounds__(128) k_k2_weights(uint32_t *__restrict__ prog, const uint4 *__restrict__ targets,
                                                    const uint4 *__restrict__ contrib, int n_targets,
                                                    const double *__restrict__ w) {
  __shared__ uint4 sW[32];   // each weight sign-extended to 128 bits
  __shared__ int s_E;
  if (threadIdx.x == 0) s_E = weight_exponent(w, 32);   // the same E as the ranking kernel's
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int64_t W = llrint(ldexp(w[lane], s_E));      // |W| <= 2^62
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
    if (tg.w & 1) {   // a 96-bit weight: the fourth word holds the term's basis entry
      prog[tg.x] = A[0];
      prog[tg.x + 1] = A[1];
      prog[tg.x + 2] = A[2];
    } else {
      *(uint4 *)(prog + tg.x) = make_uint4(A[0], A[1], A[2], A[3]);
    }
  }
}

cudaError_t launch_k2_weights(uint32_t *prog, const uint4 *targets, const uint4 *contrib, int n_targets,
                              const double *w, cudaStream_t st) {
  const int grid = std::max(1, std::min(1024, (n_targets + 127) / 128));
  k_k2_weights<<<grid, 128, 0, st>>>(prog, targets, contrib, n_targets, w);
  return cudaGetLastError();
}

// A ranking entry packs the top 48 bits of the monotone key (sign, exponent and 40
// mantissa bits: 2^-40 relative resolution) above a 16-bit variant index, so one
// signed 64-bit comparison orders by (key, variant) and exact ties (variants with
// equal predictions) fall to the smaller index.
__device__ __forceinline__ int64_t pack_entry(int64_t key, int vid) {
  return (int64_t)(((uint64_t)(key >> 16) << 16) | (uint32_t)vid);
}
__device__ __forceinline__ int entry_vid(int64_t e) { return (int)(e & 0xFFFF); }
__device__ __forceinline__ int64_t entry_key(int64_t e) { return (int64_t)((uint64_t)e & ~0xFFFFull); }

// The 16 best entries of one point, sorted ascending.
struct TopK {
  int64_t k[RK_TOPK];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < RK_TOPK; q++) k[q] = RK_EMPTY;
  }
  __device__ __forceinline__ void insert(int64_t e) {
#pragma unroll
    for (int q = RK_TOPK - 1; q > 0; q--) k[q] = e < k[q - 1] ? k[q - 1] : (e < k[q] ? e : k[q]);
    if (e < k[0]) k[0] = e;
  }
  // sort the 16 entries ascending (bitonic sorting network)
  __device__ __forceinline__ void sort() {
#pragma unroll
    for (int kk = 2; kk <= RK_TOPK; kk <<= 1)
#pragma unroll
      for (int j = kk >> 1; j > 0; j >>= 1)
#pragma unroll
        for (int i = 0; i < RK_TOPK; i++) {
          const int l = i ^ j;
          if (l > i) {
            const int64_t a = k[i], b = k[l];
            const bool up = (i & kk) == 0;
            k[i] = (a < b) == up ? a : b;
            k[l] = (a < b) == up ? b : a;
          }
        }
  }
  // the 16 smallest of this list and RK_BUF sorted entries b (ascending)
  __device__ __forceinline__ void merge_short(const int64_t (&b)[RK_BUF]) {
#pragma unroll
    for (int q = 0; q < RK_BUF; q++) {
      const int i = RK_TOPK - 1 - q;
      k[i] = b[q] < k[i] ? b[q] : k[i];
    }
    bitonic_clean();
  }
  __device__ __forceinline__ void bitonic_clean() {
#pragma unroll
    for (int d = RK_TOPK / 2; d > 0; d >>= 1)
#pragma unroll
      for (int q = 0; q < RK_TOPK; q++)
        if ((q & d) == 0) {
          const int64_t a = k[q], c = k[q + d];
          k[q] = a < c ? a : c;
          k[q + d] = a < c ? c : a;
        }
  }
  // the 16 smallest of this list and another sorted list (element q at p[q * stride]):
  // the elementwise minimum of this list and the other one reversed is a bitonic
  // sequence holding them, sorted by a four-stage bitonic merge
  __device__ __forceinline__ void merge(const int64_t *p, int stride) {
#pragma unroll
    for (int q = 0; q < RK_TOPK; q++) {
      const int64_t e = p[(RK_TOPK - 1 - q) * stride];
      k[q] = e < k[q] ? e : k[q];
    }
    bitonic_clean();
  }
};

// Candidate threshold: an entry e = (key48, variant) that the point's final 16th entry
// cannot exceed.  For a positive key K, key48(S) < K <=> S < key_floor(K) = lo and
// key48(S) == K <=> lo <= S < key_floor(K + 2^16) = hi, so the common test is one
// 128-bit compare S < hi; only then is the entry formed (a tie at K takes K itself).
// Without a threshold, or with a key <= 0, lo = hi = the largest value and every
// candidate's entry is formed and compared.
struct Threshold {
  int64_t e;
  Acc128 lo, hi;
  __device__ __forceinline__ void set(int64_t x) {
    e = x;
    if (x != RK_EMPTY && entry_key(x) > 0) {
      lo = key_floor(entry_key(x));
      hi = key_floor(entry_key(x) + 0x10000);
    } else {
      lo.lo = hi.lo = ~0ull;
      lo.hi = hi.hi = (uint64_t)INT64_MAX;
    }
  }
  __device__ __forceinline__ bool maybe(const Acc128 &S) const { return acc_less(S, hi); }
  __device__ __forceinline__ int64_t entry(const Acc128 &S, int v) const {
    return acc_less(S, lo) ? pack_entry(acc_key(S), v) : (entry_key(e) | (uint32_t)v);
  }
};

template <int N> struct IC { static constexpr int value = N; };   // a compile-time count

__device__ __forceinline__ int32_t pick4(const int32_t (&n)[4], uint32_t i) {
  int32_t x = n[0];
  x = i == 1 ? n[1] : x;
  x = i == 2 ? n[2] : x;
  x = i == 3 ? n[3] : x;
  return x;
}
__device__ __forceinline__ int64_t pick4(int64_t h0, int64_t h1, int64_t h2, int64_t h3, uint32_t i) {
  int64_t x = h0;
  x = i == 1 ? h1 : x;
  x = i == 2 ? h2 : x;
  x = i == 3 ? h3 : x;
  return x;
}

size_t rank_smem_bytes(int nw, int img_words, int basis_cap) {
  const size_t a = (size_t)((img_words + 3) & ~3) * 4 + (size_t)basis_cap * 32 * 8;
  const size_t lists = (size_t)(nw / 2) * RK_TOPK * 32 * 8;
  return std::max(a, lists) + 64 * 4 + (size_t)nw * 32 * 8 + (size_t)nw * RK_BUF * 32 * 8;
}

template <int NW>
__global__ void __maxnreg__(96) k_rank(RankArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int img_cap = (a.img_words + 3) & ~3;
  uint32_t *img = (uint32_t *)smem;                        // the group's image
  uint32_t *blo = img + img_cap;                           // basis, low words [basis_cap][32]
  uint32_t *bhi = blo + a.basis_cap * 32;                  // basis, high words
  int64_t *lists = (int64_t *)smem;                        // after the walk: [NW][16][32]
  const size_t region = max((size_t)img_cap * 4 + (size_t)a.basis_cap * 256, (size_t)(NW / 2) * RK_TOPK * 256);
  uint32_t *mask = (uint32_t *)(smem + region);            // condition bits per point [2][32]
  volatile int64_t *thrx = (int64_t *)(mask + 64);         // each warp's 16th entries [NW][32]
  int64_t *bufs = (int64_t *)(mask + 64) + NW * 32;        // [NW][RK_BUF][32]
  int64_t *mybuf = bufs + warp * RK_BUF * 32 + lane;
  __shared__ int s_E, s_unit, s_last;

  if (threadIdx.x == 0) s_E = weight_exponent(a.w, 32);   // the programs' weights are round(w 2^E)
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(a.unit_counter, 1);
    __syncthreads();
    const int u = s_unit;
    if (u >= a.n_units) break;
    const int2 U = a.units[u];
    const int4 C = a.chunks[U.x];          // template, first point, point count, first partial slot
    const int t = C.x;
    const int4 TM = a.tmpl[3 * t], LO = a.tmpl[3 * t + 1], HI = a.tmpl[3 * t + 2];
    const int P = TM.x, S_groups = TM.y;
    const bool live = lane < C.z;
    const int64_t p = (int64_t)C.y + lane;
    TopK tk;
    tk.init();
    if (U.y >= 0) {
      const int4 G0 = a.groups[2 * U.y], G1 = a.groups[2 * U.y + 1];
      for (int i = threadIdx.x; i < G0.y / 4; i += NW * 32) cp_async16(img + 4 * i, a.img + G0.x + 4 * i);
      cp_async_commit();
      // this lane's point: two 16-byte loads, then the box check
      bool valid = live;
      const int32_t l4[4] = {LO.x, LO.y, LO.z, LO.w}, h4[4] = {HI.x, HI.y, HI.z, HI.w};
      int32_t n[4] = {l4[0], l4[1], l4[2], l4[3]};
      if (live) {
        const longlong2 *src = (const longlong2 *)(a.points + p * 4);
        const longlong2 q0 = __ldg(src), q1 = __ldg(src + 1);
        const int64_t x[4] = {q0.x, q0.y, q1.x, q1.y};
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (q < P) ok = ok && x[q] >= l4[q] && x[q] <= h4[q];
        if (ok) {
#pragma unroll
          for (int q = 0; q < 4; q++) n[q] = q < P ? (int32_t)x[q] : 0;
        } else {
          if (warp == 0) atomicOr(a.status, ST_OUT_OF_BOX);
          valid = false;   // ranks nothing; its basis is evaluated at the box's corner
        }
      }
      if (threadIdx.x < 64) mask[threadIdx.x] = 0;
      thrx[warp * 32 + lane] = RK_EMPTY;
      cp_async_wait0();
      __syncthreads();
      // the basis, level by level (a product's factors are in earlier levels)
      const int nlev = (int)img[RankLayout::H_NLEV], ncond = (int)img[RankLayout::H_NCOND];
      const uint32_t *bdef = img + img[RankLayout::H_OFF_BASIS];
      int e0 = 0;
      for (int L = 0; L < nlev; L++) {
        const int e1 = (int)img[RankLayout::H_LEVEL_END + L];
        for (int e = e0 + warp; e < e1; e += NW) {
          const uint4 d0 = *(const uint4 *)(bdef + 8 * e), d1 = *(const uint4 *)(bdef + 8 * e + 4);
          const uint32_t kind = d1.w & 3;
          int64_t val;
          if (kind == 0) {
            val = pick4(n, d0.x & 3);
          } else if (kind == 1) {
            val = 1;
          } else if (kind == 2) {
            // floor((a . n + b) / c): a in d0, b = d1.x, c = d1.y, magic = d1.z
            const int32_t num = (int32_t)d1.x + (int32_t)d0.x * n[0] + (int32_t)d0.y * n[1] + (int32_t)d0.z * n[2] +
                                (int32_t)d0.w * n[3];
            val = floor_div(num, d1.y, d1.z, (d1.w >> 8) & 0xFF, (d1.w >> 16) & 1);
          } else {
            const uint64_t x = (uint64_t)blo[d0.x * 32 + lane] | ((uint64_t)bhi[d0.x * 32 + lane] << 32);
            const uint64_t y = (uint64_t)blo[d0.y * 32 + lane] | ((uint64_t)bhi[d0.y * 32 + lane] << 32);
            val = (int64_t)(x * y);
          }
          blo[e * 32 + lane] = (uint32_t)val;
          bhi[e * 32 + lane] = (uint32_t)((uint64_t)val >> 32);
        }
        __syncthreads();
        e0 = e1;
      }
      // conditions: const + sum coef * value >= 0, one bit each (64-bit coefficients; the
      // sums are exact in 64 bits, wrapping included, since each true sum is below 2^63)
      {
        const uint32_t *cd = img + img[RankLayout::H_OFF_COND];
        for (int q = 0; q < ncond; q++) {
          const int nt = (int)cd[0];
          if ((q % NW) == warp) {
            uint64_t s = (uint64_t)ld64(cd + 1);
            for (int k = 0; k < nt; k++) {
              const uint32_t e = cd[3 + 3 * k];
              const uint64_t x = (uint64_t)blo[e * 32 + lane] | ((uint64_t)bhi[e * 32 + lane] << 32);
              s += x * (uint64_t)ld64(cd + 4 + 3 * k);
            }
            if ((int64_t)s >= 0) atomicOr(&mask[(q >> 5) * 32 + lane], 1u << (q & 31));
          }
          cd += 3 + 3 * nt;
        }
      }
      __syncthreads();
      const uint32_t cm0 = mask[lane], cm1 = mask[32 + lane];
      const uint16_t *vmap = (const uint16_t *)(img + img[RankLayout::H_OFF_VARMAP]);
      const int nv = G0.w, vbase = G0.z;
      const uint32_t bmax = img[RankLayout::H_B] - 1;   // every basis index is clamped to the basis
      Threshold th;
      th.set(RK_EMPTY);
      int nbuf = 0;
      auto flush = [&]() {
        // the buffered entries, sorted, merged into the list by a bitonic network
        int64_t b[RK_BUF];
#pragma unroll
        for (int q = 0; q < RK_BUF; q++) b[q] = q < nbuf ? mybuf[q * 32] : RK_EMPTY;
#pragma unroll
        for (int i = 0; i < RK_BUF; i++)
#pragma unroll
          for (int j = 0; j + 1 < RK_BUF - i; j++) {
            const int64_t x = b[j], y = b[j + 1];
            b[j] = x < y ? x : y;
            b[j + 1] = x < y ? y : x;
          }
        tk.merge_short(b);
        nbuf = 0;
        if (tk.k[RK_TOPK - 1] < th.e) th.set(tk.k[RK_TOPK - 1]);
      };
      const uint16_t *vidm = (const uint16_t *)(img + img[RankLayout::H_OFF_VIDMAP]);
      const uint4 *runs = (const uint4 *)(img + img[RankLayout::H_OFF_RUNS]);
      const int nruns = (int)img[RankLayout::H_NRUNS];
      // walk a program's nodes to its leaf at this lane's point: the table's conditions
      // pick the piece, the post-op conditions the leaf (most programs are one leaf)
      auto leaf_of = [&](uint32_t off) -> uint4 {
        uint4 N = *(const uint4 *)(img + off);
        while (N.x & 3) {
          const uint32_t nc = (N.x >> 8) & 0xFF;
          uint32_t bits = 0;
#pragma unroll 1
          for (uint32_t c = 0; c < nc; c++) {
            const uint32_t gi = c < 5 ? (N.y >> (6 * c)) & 63 : (N.z >> (6 * (c - 5))) & 63;
            bits |= (((gi < 32 ? cm0 : cm1) >> (gi & 31)) & 1u) << c;
          }
          uint32_t o;
          if ((N.x & 3) == 1) o = (N.x >> 16) + 4 * ((img[N.w + (bits >> 2)] >> (8 * (bits & 3))) & 0xFF);
          else o = N.z + 4 * bits;
          N = *(const uint4 *)(img + o);
        }
        return N;
      };
      auto term64 = [&](uint32_t (&A)[4], const uint4 &R) {
        const uint32_t e = min(R.w, bmax) * 32 + lane;
        mac128(A, make_uint4(R.x, R.y, R.z, (uint32_t)((int32_t)R.z >> 31)),
               (int64_t)((uint64_t)blo[e] | ((uint64_t)bhi[e] << 32)));
      };
      auto term32 = [&](uint32_t (&A)[4], const uint4 &R) {
        mac128_u32(A, make_uint4(R.x, R.y, R.z, (uint32_t)((int32_t)R.z >> 31)), blo[min(R.w, bmax) * 32 + lane]);
      };
      // S from the leaf's accumulator; a table with a denominator D holds D * prediction,
      // divided exactly: a shift by t, then the inverse of d modulo 2^128
      auto finish = [&](const uint32_t (&A)[4], uint32_t dz) -> Acc128 {
        Acc128 S;
        S.lo = (uint64_t)A[0] | ((uint64_t)A[1] << 32);
        S.hi = (uint64_t)A[2] | ((uint64_t)A[3] << 32);
        if (dz) {
          const uint32_t *D = img + dz;
          const uint32_t sh = D[0] & 63;
          const uint64_t lo = sh ? (S.lo >> sh) | (S.hi << (64 - sh)) : S.lo;
          const uint64_t hi = (uint64_t)((int64_t)S.hi >> sh);
          const uint64_t ilo = ld64(D + 4), ihi = ld64(D + 6);
          S.lo = lo * ilo;
          S.hi = __umul64hi(lo, ilo) + lo * ihi + hi * ilo;
        }
        return S;
      };
      // any leaf: term counts read from the leaf record
      auto evaluate = [&](int pos) -> Acc128 {
        const uint4 N = leaf_of(vmap[pos]);
        const uint4 *rec = (const uint4 *)(img + N.y);
        const uint4 c0 = *rec++;
        uint32_t A[4] = {c0.x, c0.y, c0.z, c0.w};
        const uint32_t n64 = (N.x >> 8) & 0xFF, n32 = (N.x >> 16) & 0xFF, nwide = N.x >> 24;
#pragma unroll 1
        for (uint32_t i = 0; i < n64; i++) term64(A, *rec++);
#pragma unroll 1
        for (uint32_t i = 0; i < n32; i++) term32(A, *rec++);
#pragma unroll 1
        for (uint32_t i = 0; i < nwide; i++, rec += 2) {
          const uint32_t e = min(rec[1].x, bmax) * 32 + lane;
          mac128(A, rec[0], (int64_t)((uint64_t)blo[e] | ((uint64_t)bhi[e] << 32)));
        }
        return finish(A, N.z);
      };
      auto exchange = [&]() {   // share 16th entries with the other warps
        thrx[warp * 32 + lane] = tk.k[RK_TOPK - 1];
        int64_t m = th.e;
#pragma unroll
        for (int w = 0; w < NW; w++) {
          const int64_t x = thrx[w * 32 + lane];
          m = x < m ? x : m;
        }
        if (m < th.e) th.set(m);
      };
      int since = 0;
      // one candidate after the fill: one 128-bit compare; the few that may pass are
      // buffered.  Returns true when the warp should stop to flush its buffers (a lane's
      // buffer is full) or to exchange thresholds (every RK_EXCHANGE variants).
      auto offer = [&](const Acc128 &S, int pos) -> bool {
        const bool m = valid && th.maybe(S);
        bool stop = ++since >= RK_EXCHANGE;
        if (__any_sync(0xffffffffu, m)) {
          if (m) {
            const int64_t e = th.entry(S, vbase + vidm[pos]);
            if (e < th.e) {
              mybuf[nbuf * 32] = e;
              nbuf++;
            }
          }
          stop = stop || __any_sync(0xffffffffu, nbuf == RK_BUF);
        }
        return stop;
      };
      // the first 16 positions of the warp fill its list, sorted once
      const int fill_end = min(nv, RK_TOPK * NW);
#pragma unroll 1
      for (int f = 0, pos = warp; f < RK_TOPK; f++, pos += NW) {
        int64_t e = RK_EMPTY;
        if (pos < fill_end) {   // lanes without a valid point evaluate the box's corner
          const int64_t x = pack_entry(acc_key(evaluate(pos)), vbase + vidm[pos]);
          e = valid ? x : RK_EMPTY;
        }
#pragma unroll
        for (int q = 0; q + 1 < RK_TOPK; q++) tk.k[q] = tk.k[q + 1];
        tk.k[RK_TOPK - 1] = e;
      }
      tk.sort();
      th.set(tk.k[RK_TOPK - 1]);
      exchange();
      // the variants of a run of one shape (term counts fixed at compile time) from pos
      // on, until the warp must stop; returns the next position.  The flush and the
      // exchange sit once in the run loop below, outside the per-shape code, which keeps
      // the kernel's hot code small.
      auto run_fixed = [&](auto c64, auto c32, int pos, int end) -> int {
        constexpr int N64 = decltype(c64)::value, N32 = decltype(c32)::value;
        while (pos < end) {
          const uint4 N1 = leaf_of(vmap[pos]);
          const uint4 *r1 = (const uint4 *)(img + N1.y);
          const uint4 c = r1[0];
          uint32_t A1[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int i = 1; i <= N64; i++) term64(A1, r1[i]);
#pragma unroll
          for (int i = N64 + 1; i <= N64 + N32; i++) term32(A1, r1[i]);
          const bool stop = offer(finish(A1, N1.z), pos);
          pos += NW;
          if (stop) break;
        }
        return pos;
      };
      auto run_generic = [&](int pos, int end) -> int {
        while (pos < end) {
          const bool stop = offer(evaluate(pos), pos);
          pos += NW;
          if (stop) break;
        }
        return pos;
      };
      for (int r = 0; r < nruns; r++) {
        const uint4 R = runs[r];
        const int start = max((int)R.y, fill_end), end = (int)(R.y + R.z);
        if (start >= end) continue;
        int pos = start + ((warp - start % NW) + NW) % NW;   // this warp's first position
        while (pos < end) {
          switch (R.x) {
#define PM_RUN(a, b) case (a) | ((b) << 8): pos = run_fixed(IC<a>{}, IC<b>{}, pos, end); break;
            PM_RUN(0, 1) PM_RUN(0, 2) PM_RUN(0, 3) PM_RUN(1, 1) PM_RUN(1, 2) PM_RUN(1, 3) PM_RUN(1, 6)
            PM_RUN(1, 10) PM_RUN(2, 1) PM_RUN(2, 2) PM_RUN(3, 2) PM_RUN(3, 3) PM_RUN(4, 2) PM_RUN(5, 1)
#undef PM_RUN
            default:
              pos = run_generic(pos, end);
          }
          if (__any_sync(0xffffffffu, nbuf == RK_BUF)) flush();
          if (since >= RK_EXCHANGE) {
            since = 0;
            exchange();
          }
        }
      }
      flush();
      // merge the warps' lists in a tree (the image and basis are no longer read)
      __syncthreads();
#pragma unroll
      for (int half = NW / 2; half > 0; half >>= 1) {
        if (warp >= half && warp < 2 * half) {
#pragma unroll
          for (int q = 0; q < RK_TOPK; q++) lists[((warp - half) * RK_TOPK + q) * 32 + lane] = tk.k[q];
        }
        __syncthreads();
        if (warp < half) tk.merge(lists + warp * RK_TOPK * 32 + lane, 32);
        __syncthreads();
      }
      if (S_groups > 1) {
        // publish this group's lists; the last group of the chunk merges all of them
        if (warp == 0) {
          const int64_t slot0 = ((int64_t)C.w + G1.y) * RK_TOPK * 32 + lane;
#pragma unroll
          for (int q = 0; q < RK_TOPK; q++) a.part_k[slot0 + q * 32] = tk.k[q];
          __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(a.chunk_count + U.x, 1) == S_groups - 1;
        __syncthreads();
        if (!s_last) continue;
        if (warp == 0) {
          __threadfence();
          tk.init();
          for (int g = 0; g < S_groups; g++) tk.merge(a.part_k + ((int64_t)C.w + g) * RK_TOPK * 32 + lane, 32);
        }
      }
    }
    if (warp == 0 && live) {
      int32_t *oi = a.top_idx + p * a.topk;
      double *ot = a.top_t + p * a.topk;
      const int E = s_E;
#pragma unroll
      for (int q = 0; q < RK_TOPK; q++) {
        if (q < a.topk) {
          const bool real = tk.k[q] != RK_EMPTY;
          oi[q] = real ? entry_vid(tk.k[q]) : -1;
          ot[q] = real ? key_value(entry_key(tk.k[q]), E) : __longlong_as_double(0x7ff0000000000000ll);
        }
      }
    }
  }
}

template <int NW>
static cudaError_t launch_nw(const RankArgs &args, int grid, cudaStream_t st) {
  const size_t sm = rank_smem_bytes(NW, args.img_words, args.basis_cap);
  cudaError_t e = cudaFuncSetAttribute(k_rank<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_rank<NW><<<grid, NW * 32, sm, st>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_rank(const RankArgs &args, int nw, int grid, cudaStream_t st) {
  if (nw == 4) return launch_nw<4>(args, grid, st);
  if (nw == 8) return launch_nw<8>(args, grid, st);
  return cudaErrorInvalidValue;
}

template <int NW>
static int occupancy(int img_words, int basis_cap) {
  int nb = 0;
  const size_t sm = rank_smem_bytes(NW, img_words, basis_cap);
  if (cudaFuncSetAttribute(k_rank<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rank<NW>, NW * 32, sm) != cudaSuccess) return 0;
  return nb;
}

int rank_max_blocks_per_sm(int nw, int img_words, int basis_cap) {
  if (nw == 4) return occupancy<4>(img_words, basis_cap);
  if (nw == 8) return occupancy<8>(img_words, basis_cap);
  return 0;
}

}  // namespace pmd
