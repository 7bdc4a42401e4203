// K1: materialised count evaluation (pm_eval_counts).
// K2: persistent fused evaluation -> FP64-accurate prediction -> top-k ranking
//     (pm_eval_predict_topk), the batched form of Sec. 2's re-evaluation of p_i(n)
//     over a tuning search space and of configuration selection (Sec. 6.1).
#include <cuda_runtime.h>
#include <stdint.h>

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
  int64_t *prods = stage + K1_THREADS * (K + 1);                     // [16][threads]
  int32_t *vals = (int32_t *)(prods + pmt::MAX_PRODS * K1_THREADS);  // [32][threads]
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
          sT, n, vals + tid, K1_THREADS, prods + tid, K1_THREADS,
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
  for (int i = tid; i < total; i += K1_THREADS) {
    int r = i / K, c = i - r * K;
    dst[i] = stage[r * (K + 1) + c];
  }
}

size_t k1_smem_bytes(int K) {
  return (size_t)pmt::MAX_TABLE_WORDS * 4 + (size_t)K1_THREADS * (K + 1) * 8 +
         (size_t)pmt::MAX_PRODS * K1_THREADS * 8 + (size_t)pmt::MAX_VALUES * K1_THREADS * 4;
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
constexpr int TB_WORDS = 768;   // per-warp staging buffer (3 KB), double-buffered
constexpr int K2_VMAX = 16;     // value slots per lane

// Ranking key: a normalised float-float time (hi = fl(hi + lo)) and the variant index.
__device__ __forceinline__ bool key_less(float ah, float al, int ai, float bh, float bl, int bi) {
  return ah < bh || (ah == bh && (al < bl || (al == bl && ai < bi)));
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_all;\n" ::); }

struct TopK {
  float h[K2_TOPK], l[K2_TOPK];
  int id[K2_TOPK];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < K2_TOPK; q++) { h[q] = __int_as_float(0x7f800000); l[q] = 0.f; id[q] = 0x7fffffff; }
  }
  __device__ __forceinline__ void insert(float th, float tl, int ti) {
    if (!key_less(th, tl, ti, h[K2_TOPK - 1], l[K2_TOPK - 1], id[K2_TOPK - 1])) return;
#pragma unroll
    for (int q = K2_TOPK - 1; q >= 0; q--) {
      if (key_less(th, tl, ti, h[q], l[q], id[q])) {
        if (q == 0 || key_less(h[q - 1], l[q - 1], id[q - 1], th, tl, ti)) { h[q] = th; l[q] = tl; id[q] = ti; }
        else { h[q] = h[q - 1]; l[q] = l[q - 1]; id[q] = id[q - 1]; }
      }
    }
  }
};

// Merge n sorted lists of 16 (stored at base + list*stride_list + q*stride_q, SoA) for this lane.
template <int MAXN, bool CG>
__device__ __forceinline__ void merge_lists(const float *hs, const float *ls, const int *is, int n, int stride_list,
                                            int stride_q, TopK &out) {
  int head[MAXN];
#pragma unroll
  for (int w = 0; w < MAXN; w++) head[w] = 0;
#pragma unroll
  for (int q = 0; q < K2_TOPK; q++) {
    int best = -1;
    float bh = 0.f, bl = 0.f;
    int bi = 0x7fffffff;
#pragma unroll
    for (int w = 0; w < MAXN; w++) {
      if (w < n && head[w] < K2_TOPK) {
        const int o = w * stride_list + head[w] * stride_q;
        float xh, xl;
        int xi;
        if (CG) { xh = __ldcg(hs + o); xl = __ldcg(ls + o); xi = __ldcg(is + o); }
        else { xh = hs[o]; xl = ls[o]; xi = is[o]; }
        if (best < 0 || key_less(xh, xl, xi, bh, bl, bi)) { best = w; bh = xh; bl = xl; bi = xi; }
      }
    }
#pragma unroll
    for (int w = 0; w < MAXN; w++) if (w == best) head[w]++;
    out.h[q] = bh;
    out.l[q] = bl;
    out.id[q] = bi;
  }
}

// Warp w of a CTA evaluates variants vb+w, vb+w+NW, ... < ve of the unit's template
// for the unit's points (one point per lane; the table is shared by the warp and read
// as broadcasts from shared memory).  Each lane keeps the 16 best (time, variant)
// pairs of its point in registers.  The CTA merges its warps' lists; a point chunk
// split into S variant slices is finished by the last of its S units (partial lists
// in a scratch buffer, a fence and an atomic counter; no waiting).
template <int NW>
__global__ void __launch_bounds__(NW * 32) k_eval_predict_topk(K2Args a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t *tbuf = (uint32_t *)smem;                                  // [NW][2][TB_WORDS]
  int32_t *vals = (int32_t *)(tbuf + NW * 2 * TB_WORDS);              // [NW][VMAX][32]
  int64_t *prods = (int64_t *)(vals + NW * K2_VMAX * 32);             // [NW][16][32]
  float *mh = (float *)smem;                                          // merge lists [NW][16][32] (alias tbuf)
  float *ml = mh + NW * K2_TOPK * 32;
  int *mi = (int *)(ml + NW * K2_TOPK * 32);
  __shared__ float s_wh[pmt::MAX_COLS], s_wl[pmt::MAX_COLS];
  __shared__ double s_unscale;
  __shared__ int s_unit, s_last;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *mybuf = tbuf + warp * 2 * TB_WORDS;
  int32_t *myvals = vals + warp * K2_VMAX * 32 + lane;
  int64_t *myprods = prods + warp * pmt::MAX_PRODS * 32 + lane;

  if (threadIdx.x == 0) {
    // power-of-two scaling of the weights into the FP32 range
    double mx = 0;
    for (int c = 0; c < 32; c++) mx = fmax(mx, fabs(a.w[c]));
    int e = 0;
    if (mx > 0) frexp(mx, &e);
    const double sc = ldexp(1.0, -e);
    for (int c = 0; c < pmt::MAX_COLS; c++) {
      FF f = split_weight(c < 32 ? a.w[c] * sc : 0.0);
      s_wh[c] = f.hi;
      s_wl[c] = f.lo;
    }
    s_unscale = ldexp(1.0, e);
  }
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
    const int64_t p = (int64_t)C.y + lane;
    const bool live = lane < C.z;
    const int P = a.tmpl_nparams[t];
    int64_t pt[4] = {0, 0, 0, 0};
    if (live) {
      const int64_t *src = a.points + p * 4;
#pragma unroll
      for (int q = 0; q < 4; q++) pt[q] = src[q];
    }
    TopK tk;
    tk.init();
    const int v0 = a.var_off[t];
    const int ve = U.w;
    int v = U.z + warp;
    auto stage_table = [&](int vv, int slot) {
      if (vv < ve) {
        const uint32_t *g = a.arena + a.tab_off[vv];
        const int words = (int)g[pmt::H_WORDS];
        if (words <= TB_WORDS)
          for (int i = lane; i < words / 4; i += 32) cp_async16(mybuf + slot * TB_WORDS + 4 * i, g + 4 * i);
      }
      cp_async_commit();
    };
    stage_table(v, 0);
    int slot = 0;
    for (; v < ve; v += NW) {
      stage_table(v + NW, slot ^ 1);
      cp_async_wait1();
      __syncwarp();
      const uint32_t *gT = a.arena + a.tab_off[v];
      const int words = (int)gT[pmt::H_WORDS];
      const uint32_t *T = words <= TB_WORDS ? mybuf + slot * TB_WORDS : gT;
      if (live) {
        int32_t n[4];
        if (!point_in_box(T, pt, P, n)) {
          atomicOr(a.status, ST_OUT_OF_BOX);
        } else {
          float s = 0.f, c = 0.f;
          const bool ok = eval_table(
              T, n, myvals, 32, myprods, 32,
              [&](int col, int64_t val) { if (col < 32) dot2_add(s, c, val, s_wh[col], s_wl[col]); },
              [&](int col, int64_t val) { dot2_add(s, c, val, s_wh[col], s_wl[col]); });
          if (!ok) atomicOr(a.status, ST_BAD_TABLE);
          // normalise (s, c) to hi = fl(s + c) with the exact remainder in lo (TwoSum)
          const float hi = __fadd_rn(s, c);
          const float z = __fsub_rn(hi, s);
          const float lo = __fadd_rn(__fsub_rn(s, __fsub_rn(hi, z)), __fsub_rn(c, z));
          tk.insert(hi, lo, v - v0);
        }
      }
      __syncwarp();
      slot ^= 1;
    }
    cp_async_wait0();
    __syncthreads();  // table buffers are reused as merge buffers below
#pragma unroll
    for (int q = 0; q < K2_TOPK; q++) {
      const int o = (warp * K2_TOPK + q) * 32 + lane;
      mh[o] = tk.h[q];
      ml[o] = tk.l[q];
      mi[o] = tk.id[q];
    }
    __syncthreads();
    if (warp == 0) {
      TopK m;
      merge_lists<NW, false>(mh + lane, ml + lane, mi + lane, NW, K2_TOPK * 32, 32, m);
      bool write_out = S == 1;
      if (S > 1) {
        // publish this slice's list, then the last slice of the chunk merges all of them
        const int64_t slot0 = (int64_t)(C.w + U.y) * K2_TOPK * 32 + lane;
#pragma unroll
        for (int q = 0; q < K2_TOPK; q++) {
          a.part_h[slot0 + q * 32] = m.h[q];
          a.part_l[slot0 + q * 32] = m.l[q];
          a.part_i[slot0 + q * 32] = m.id[q];
        }
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) last = atomicAdd(a.chunk_count + U.x, 1) == S - 1;
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
          __threadfence();
          const int64_t b = (int64_t)C.w * K2_TOPK * 32 + lane;
          merge_lists<K2_MAX_SLICES, true>(a.part_h + b, a.part_l + b, a.part_i + b, S, K2_TOPK * 32, 32, m);
          write_out = true;
        }
      }
      if (write_out && live) {
        int32_t *oi = a.top_idx + p * a.topk;
        double *ot = a.top_t + p * a.topk;
#pragma unroll
        for (int q = 0; q < K2_TOPK; q++) {
          if (q < a.topk) {
            const bool real = m.id[q] != 0x7fffffff;
            oi[q] = real ? m.id[q] : -1;
            ot[q] = real ? ((double)m.h[q] + (double)m.l[q]) * s_unscale : __longlong_as_double(0x7ff0000000000000ll);
          }
        }
      }
    }
    __syncthreads();
  }
}

size_t k2_smem_bytes(int nw) {
  static_assert(3 * K2_TOPK * 32 * 4 <= 2 * TB_WORDS * 4, "merge lists must fit in the table buffers");
  return (size_t)nw * 2 * TB_WORDS * 4 + (size_t)nw * K2_VMAX * 32 * 4 + (size_t)nw * pmt::MAX_PRODS * 32 * 8;
}

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
