// Serving kernels: one batch of autotuner queries (Sec. 6.1 configuration selection).
//
// A query asks for the topk fastest of n candidate (kernel variant, parameter point)
// pairs under one device model.  Each candidate's properties p_i(n) are evaluated from
// its compiled table (Sec. 2: counts re-evaluated for changed n) and contracted with the
// model's weights to FP64 accuracy (exact fixed-point products and 128-bit sums, as in
// the batched ranking kernel).  Two launches per batch:
//   k_serve_eval  one thread per candidate -> a monotone 64-bit ranking key
//   k_serve_topk  one CTA per query -> topk (key, candidate) pairs, ordered by
//                 (time, candidate index), converted to times.
#include "eval_common.cuh"

namespace pmd {

constexpr int SV_THREADS = 128;      // candidates per k_serve_eval CTA
constexpr int SV_TOPK_THREADS = 256;

// Per-model fixed-point weights W_i = round(w_i 2^E) (sum |W_i| <= 2^62) as 28-bit limb
// triples; thread 0 finds E with the same serial loop in every CTA of a batch, so every
// CTA derives the same values.
__device__ __forceinline__ void load_model_limbs(const double *w, Limbs3 *s_w, int *s_E) {
  if (threadIdx.x == 0) *s_E = weight_exponent(w, 32);
  __syncthreads();
  if (threadIdx.x < 32) s_w[threadIdx.x] = to_limbs3(llrint(ldexp(w[threadIdx.x], *s_E)));
}

__global__ void __launch_bounds__(SV_THREADS) k_serve_eval(ServeArgs a) {
  __shared__ int64_t slots[pmt::MAX_SLOTS * SV_THREADS];
  __shared__ Limbs3 s_w[32];
  __shared__ int s_E;
  const int2 b = a.blocks[blockIdx.x];
  const SQuery q = a.queries[b.x];
  load_model_limbs(a.models + (int64_t)q.model * 32, s_w, &s_E);
  __syncthreads();
  const int i = b.y * SV_THREADS + threadIdx.x;
  if (i >= q.n) return;
  const int64_t c = q.begin + i;
  const uint32_t *T = a.arena + a.cand_off[c];
  int64_t key = INT64_MAX;   // out-of-box candidates never rank
  int32_t n[4];
  if (!point_in_box(T, a.points + c * 4, (int)T[pmt::H_NPARAMS], n)) {
    atomicOr(a.q_status + b.x, ST_OUT_OF_BOX);
  } else {
    LimbAcc la;
    la.zero();
    const bool ok = eval_table(
        T, n, slots + threadIdx.x, SV_THREADS,
        [&](int col, int64_t val) { if (col < 32) la.add((uint64_t)val, s_w[col]); },
        [&](int col, int64_t val) { la.add((uint64_t)val, s_w[col]); });
    if (!ok) atomicOr(a.q_status + b.x, ST_BAD_TABLE);
    else key = acc_key(la.sum());
  }
  a.keys[c] = key;
}

// Sorted (key, index) list of the 16 smallest pairs seen by one thread.
struct SvList {
  int64_t k[SV_MAX_TOPK];
  int32_t id[SV_MAX_TOPK];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < SV_MAX_TOPK; j++) { k[j] = INT64_MAX; id[j] = 0x7fffffff; }
  }
  // indices arrive in increasing order: an equal key ranks after the ones already held
  __device__ __forceinline__ void insert(int64_t key, int32_t idx) {
    if (!(key < k[SV_MAX_TOPK - 1])) return;
#pragma unroll
    for (int j = SV_MAX_TOPK - 1; j > 0; j--) {
      const bool shift = key < k[j - 1];
      const bool here = !shift && key < k[j];
      if (shift) { k[j] = k[j - 1]; id[j] = id[j - 1]; }
      else if (here) { k[j] = key; id[j] = idx; }
    }
    if (key < k[0]) { k[0] = key; id[0] = idx; }
  }
  __device__ __forceinline__ void pop() {
#pragma unroll
    for (int j = 0; j < SV_MAX_TOPK - 1; j++) { k[j] = k[j + 1]; id[j] = id[j + 1]; }
    k[SV_MAX_TOPK - 1] = INT64_MAX;
    id[SV_MAX_TOPK - 1] = 0x7fffffff;
  }
};

__device__ __forceinline__ bool pair_less(int64_t ka, int32_t ia, int64_t kb, int32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

__global__ void __launch_bounds__(SV_TOPK_THREADS) k_serve_topk(ServeArgs a) {
  __shared__ Limbs3 s_w[32];
  __shared__ int s_E;
  __shared__ int64_t r_k[SV_TOPK_THREADS / 32];
  __shared__ int32_t r_i[SV_TOPK_THREADS / 32];
  const SQuery q = a.queries[blockIdx.x];
  load_model_limbs(a.models + (int64_t)q.model * 32, s_w, &s_E);
  SvList L;
  L.init();
  for (int i = threadIdx.x; i < q.n; i += SV_TOPK_THREADS) L.insert(a.keys[q.begin + i], i);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r < q.topk; r++) {
    // block-wide smallest head; every index is held by exactly one thread
    int64_t bk = L.k[0];
    int32_t bi = L.id[0];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const int64_t ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (pair_less(ok, oi, bk, bi)) { bk = ok; bi = oi; }
    }
    if (lane == 0) { r_k[warp] = bk; r_i[warp] = bi; }
    __syncthreads();
    bk = r_k[0];
    bi = r_i[0];
#pragma unroll
    for (int w = 1; w < SV_TOPK_THREADS / 32; w++)
      if (pair_less(r_k[w], r_i[w], bk, bi)) { bk = r_k[w]; bi = r_i[w]; }
    __syncthreads();
    if (L.id[0] == bi && bi != 0x7fffffff) L.pop();
    if (threadIdx.x == 0) {
      const bool real = bi != 0x7fffffff;
      a.out_idx[(int64_t)blockIdx.x * SV_MAX_TOPK + r] = real ? bi : -1;
      a.out_t[(int64_t)blockIdx.x * SV_MAX_TOPK + r] =
          real ? key_value(bk, s_E) : __longlong_as_double(0x7ff0000000000000ll);
    }
  }
}

cudaError_t launch_serve(const ServeArgs &a, int n_blocks, cudaStream_t st) {
  if (n_blocks > 0) k_serve_eval<<<n_blocks, SV_THREADS, 0, st>>>(a);
  if (a.n_queries > 0) k_serve_topk<<<a.n_queries, SV_TOPK_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pmd
