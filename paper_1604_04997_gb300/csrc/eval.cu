// K1: materialised count evaluation (pm_eval_counts), Sec. 2's re-evaluation of the
//     properties p_i(n) of compiled tables at many parameter points.
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

}  // namespace pmd
