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
  int32_t *vals = (int32_t *)(stage + K1_THREADS * (K + 1));         // [32][threads]
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
          sT, n, vals + tid, K1_THREADS,
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
  return (size_t)pmt::MAX_TABLE_WORDS * 4 + (size_t)K1_THREADS * (K + 1) * 8 + (size_t)pmt::MAX_VALUES * K1_THREADS * 4;
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

__device__ __forceinline__ bool tk_less(double a, int ia, double b, int ib) {
  return a < b || (a == b && ia < ib);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Warp w of a CTA evaluates variants w, w+NW, ... of the unit's template for the
// unit's 32 points (one point per lane; the table is shared by the warp and read
// as broadcasts from shared memory).  Each lane keeps the 16 best (time, variant)
// pairs of its point in registers; the NW lists are merged at the end.
template <int NW>
__global__ void __launch_bounds__(NW * 32) k_eval_predict_topk(K2Args a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t *tbuf = (uint32_t *)smem;                                  // [NW][2][TB_WORDS]
  int32_t *vals = (int32_t *)(tbuf + NW * 2 * TB_WORDS);              // [NW][32 values][32 lanes]
  double *mt = (double *)smem;                                        // [NW][32][16] merge buffer (aliases tbuf)
  int32_t *mi = (int32_t *)(mt + NW * 32 * K2_TOPK);                  // [NW][32][16]
  __shared__ float s_wh[pmt::MAX_COLS], s_wl[pmt::MAX_COLS];
  __shared__ double s_unscale;
  __shared__ int s_unit;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *mybuf = tbuf + warp * 2 * TB_WORDS;
  int32_t *myvals = vals + warp * pmt::MAX_VALUES * 32 + lane;

  if (threadIdx.x == 0) {
    // power-of-two scaling of the weights into the FP32 range
    double mx = 0;
    for (int c = 0; c < 32; c++) mx = fmax(mx, fabs(a.w[c]));
    int e = 0;
    if (mx > 0) frexp(mx, &e);
    double sc = ldexp(1.0, -e);
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
    const int4 U = a.units[u];           // template, first point, point count, -
    const int t = U.x;
    const int64_t p = (int64_t)U.y + lane;
    const bool live = lane < U.z;
    const int P = a.tmpl_nparams[t];
    int64_t pt[4] = {0, 0, 0, 0};
    if (live) {
      const int64_t *src = a.points + p * 4;
#pragma unroll
      for (int q = 0; q < 4; q++) pt[q] = src[q];
    }
    double kt[K2_TOPK];
    int ki[K2_TOPK];
#pragma unroll
    for (int q = 0; q < K2_TOPK; q++) { kt[q] = __longlong_as_double(0x7ff0000000000000ll); ki[q] = 0x7fffffff; }

    const int v0 = a.var_off[t], v1 = a.var_off[t + 1];
    // prefetch the warp's first table
    int v = v0 + warp;
    auto stage_table = [&](int vv, int slot) {
      if (vv < v1) {
        const uint32_t *g = a.arena + a.tab_off[vv];
        int words = (int)g[pmt::H_WORDS];
        if (words <= TB_WORDS)
          for (int i = lane; i < words / 4; i += 32) cp_async16(mybuf + slot * TB_WORDS + 4 * i, g + 4 * i);
      }
      cp_async_commit();
    };
    stage_table(v, 0);
    int slot = 0;
    for (; v < v1; v += NW) {
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
          bool ok = eval_table(
              T, n, myvals, 32,
              [&](int col, int64_t val) { if (col < 32) dot2_add(s, c, val, s_wh[col], s_wl[col]); },
              [&](int col, int64_t val) { dot2_add(s, c, val, s_wh[col], s_wl[col]); });
          if (!ok) atomicOr(a.status, ST_BAD_TABLE);
          const double tv = ((double)s + (double)c) * s_unscale;
          const int id = v - v0;
          if (tk_less(tv, id, kt[K2_TOPK - 1], ki[K2_TOPK - 1])) {
#pragma unroll
            for (int q = K2_TOPK - 1; q >= 0; q--) {
              if (tk_less(tv, id, kt[q], ki[q])) {
                if (q == 0 || tk_less(kt[q - 1], ki[q - 1], tv, id)) { kt[q] = tv; ki[q] = id; }
                else { kt[q] = kt[q - 1]; ki[q] = ki[q - 1]; }
              }
            }
          }
        }
      }
      __syncwarp();
      slot ^= 1;
    }
    asm volatile("cp.async.wait_all;\n" ::);
    __syncthreads();  // table buffers are reused as merge buffers below
    // merge the NW per-warp lists of each point
    double *myt = mt + (warp * 32 + lane) * K2_TOPK;
    int32_t *myi = mi + (warp * 32 + lane) * K2_TOPK;
#pragma unroll
    for (int q = 0; q < K2_TOPK; q++) { myt[q] = kt[q]; myi[q] = ki[q]; }
    __syncthreads();
    if (warp == 0 && live) {
      int head[NW];
#pragma unroll
      for (int w = 0; w < NW; w++) head[w] = 0;
      int32_t *oi = a.top_idx + p * a.topk;
      double *ot = a.top_t + p * a.topk;
      for (int q = 0; q < a.topk; q++) {
        int best = -1;
        double bt = 0;
        int bi = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) {
          if (head[w] < K2_TOPK) {
            double x = mt[(w * 32 + lane) * K2_TOPK + head[w]];
            int xi = mi[(w * 32 + lane) * K2_TOPK + head[w]];
            if (best < 0 || tk_less(x, xi, bt, bi)) { best = w; bt = x; bi = xi; }
          }
        }
#pragma unroll
        for (int w = 0; w < NW; w++) if (w == best) head[w]++;
        const bool real = bi != 0x7fffffff;
        oi[q] = real ? bi : -1;
        ot[q] = bt;
      }
    }
    __syncthreads();
  }
}

size_t k2_smem_bytes(int nw) {
  static_assert(32 * K2_TOPK * 12 <= 2 * TB_WORDS * 4, "merge buffers must fit in the table buffers");
  return (size_t)nw * 2 * TB_WORDS * 4 + (size_t)nw * pmt::MAX_VALUES * 32 * 4;
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
