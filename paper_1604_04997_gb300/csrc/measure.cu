// Measurement and test kernels for fitting the run-time model on this GPU (Sec. 4.1,
// Sec. 5), timed as in Sec. 4.2.  Every kernel performs, per work-item, exactly the
// loads, stores, floating-point operations and barriers of its IR description
// (workloads.probe_ir); index arithmetic is not counted (Sec. 2.2).  Guards match
// the IR's: a work-item outside the index space does no counted work but still
// takes part in its group's barriers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pm.h"
#include "pm_internal.h"
#include "pm_measure.h"
#include "trace.h"

namespace {

// ------------------------------------------------------------------ 1-D streaming kernels

template <class E>
__global__ void k_copy(const E *__restrict__ a, E *__restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

template <class E>
__global__ void k_sum4(const E *__restrict__ a0, const E *__restrict__ a1, const E *__restrict__ a2,
                       const E *__restrict__ a3, E *__restrict__ c, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a0[i] + a1[i] + a2[i] + a3[i];
}

template <class E>
__global__ void k_index(E *__restrict__ a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = __int_as_float((int)i) == 0.f ? E(0) : E(1);   // a value from the index, no counted flop
}

template <class E>
__global__ void k_vsa(const E *__restrict__ a, const E *__restrict__ b, E *__restrict__ c, int64_t n, int s, E alpha,
                      E beta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[s * i] = alpha * a[s * i] + beta * b[s * i];
}

// o[i] = sum over k' < K, j < s of a[k'][s i + j]: s consecutive elements per work-item
// and iteration, so a group's loads fill every element of its span.
__global__ void k_filled(const float *__restrict__ a, float *__restrict__ o, int64_t n, int s, int K) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.f;
  for (int k = 0; k < K; k++) {
    const float *row = a + (int64_t)k * s * n + s * i;
    for (int j = 0; j < s; j++) acc = acc + row[j];
  }
  o[i] = acc;
}

// ------------------------------------------------------------------ 2-D arithmetic / empty

__global__ void k_empty() {}

// Values just above and just below 1 from integer bits (index arithmetic, not counted
// flops), so that long products and quotients stay bounded.
template <class E> __device__ __forceinline__ E val_hi(uint32_t bits);
template <class E> __device__ __forceinline__ E val_lo(uint32_t bits);
template <> __device__ __forceinline__ float val_hi<float>(uint32_t b) { return __uint_as_float(0x3F800000u | ((b & 0x7FFu) << 1)); }
template <> __device__ __forceinline__ float val_lo<float>(uint32_t b) { return __uint_as_float(0x3F7FF000u | (b & 0xFFFu)); }
template <> __device__ __forceinline__ double val_hi<double>(uint32_t b) {
  return __longlong_as_double(0x3FF0000000000000ll | ((long long)(b & 0x7FFu) << 30));
}
template <> __device__ __forceinline__ double val_lo<double>(uint32_t b) {
  return __longlong_as_double(0x3FEFFE0000000000ll | ((long long)(b & 0xFFFu) << 29));
}

// Per work-item: k iterations of 8 operations of one type (0 add/sub, 1 mul, 2 div,
// 3 exp + add, 4 rsqrt + add), each on a distinct value, then one store.
template <class E, int TYPE>
__global__ void k_arith(E *__restrict__ o, int64_t n, int K) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t y = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= n || y >= n) return;
  const uint32_t h = (uint32_t)(x * 7 + y * 13);
  E acc = TYPE == 0 ? E(0) : E(1);
#pragma unroll 1
  for (int k = 0; k < K; k++) {
    const uint32_t b = h + (uint32_t)k * 8u;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const E v = (q & 1) ? val_lo<E>(b + q) : val_hi<E>(b + q);
      if (TYPE == 0) acc = (q & 1) ? acc - v : acc + v;
      if (TYPE == 1) acc = acc * v;
      if (TYPE == 2) acc = acc / v;
      if (TYPE == 3) acc = acc + (E)expf((float)v);
      if (TYPE == 4) acc = acc + (E)rsqrtf((float)v);
    }
  }
  o[y * n + x] = acc;
}

// ------------------------------------------------------------------ transposes (T x T tiles)

template <int T>
__global__ void k_transpose_p(const float *__restrict__ in, float *__restrict__ out, int64_t n) {
  __shared__ float t[T][T + 1];
  const int lx = threadIdx.x, ly = threadIdx.y;
  const int64_t Y = (int64_t)T * blockIdx.y + ly, X = (int64_t)T * blockIdx.x + lx;
  if (Y < n && X < n) t[ly][lx] = in[Y * n + X];
  __syncthreads();
  const int64_t Yt = (int64_t)T * blockIdx.x + ly, Xt = (int64_t)T * blockIdx.y + lx;
  if (Yt < n && Xt < n) out[Yt * n + Xt] = t[lx][ly];
}

__global__ void k_transpose_r(const float *__restrict__ in, float *__restrict__ out, int64_t n) {
  const int64_t Y = (int64_t)blockDim.y * blockIdx.y + threadIdx.y, X = (int64_t)blockDim.x * blockIdx.x + threadIdx.x;
  if (Y < n && X < n) out[X * n + Y] = in[Y * n + X];
}

__global__ void k_transpose_w(const float *__restrict__ in, float *__restrict__ out, int64_t n) {
  const int64_t Y = (int64_t)blockDim.y * blockIdx.y + threadIdx.y, X = (int64_t)blockDim.x * blockIdx.x + threadIdx.x;
  if (Y < n && X < n) out[Y * n + X] = in[X * n + Y];
}

// ------------------------------------------------------------------ matmuls, C = A B

template <int T>
__global__ void k_matmul(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C, int64_t n,
                         int64_t m, int64_t l) {
  __shared__ float As[T][T], Bs[T][T];
  const int lx = threadIdx.x, ly = threadIdx.y;
  const int64_t Y = (int64_t)T * blockIdx.y + ly, X = (int64_t)T * blockIdx.x + lx;
  float acc = 0.f;
  for (int64_t kt = 0; kt < (m + T - 1) / T; kt++) {
    if (Y < n && T * kt + lx < m) As[ly][lx] = A[Y * m + T * kt + lx];
    if (T * kt + ly < m && X < l) Bs[ly][lx] = B[(T * kt + ly) * l + X];
    __syncthreads();
    if (Y < n && X < l) {
      const int kmax = (int)(m - T * kt < T ? m - T * kt : T);
      for (int k = 0; k < kmax; k++) acc += As[ly][k] * Bs[k][lx];
    }
    __syncthreads();
  }
  if (Y < n && X < l) C[Y * l + X] = acc;
}

__global__ void k_matmul_naive(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C,
                               int64_t n, int64_t m, int64_t l) {
  const int64_t Y = (int64_t)blockDim.y * blockIdx.y + threadIdx.y, X = (int64_t)blockDim.x * blockIdx.x + threadIdx.x;
  if (Y >= n || X >= l) return;
  float acc = 0.f;
  for (int64_t k = 0; k < m; k++) acc += A[Y * m + k] * B[k * l + X];
  C[Y * l + X] = acc;
}

// ------------------------------------------------------------------ test kernels

__global__ void k_stencil(const float *__restrict__ u, float *__restrict__ v, int64_t n, float c0, float c1) {
  const int64_t Y = (int64_t)blockDim.y * blockIdx.y + threadIdx.y + 1, X = (int64_t)blockDim.x * blockIdx.x + threadIdx.x + 1;
  if (Y < n - 1 && X < n - 1)
    v[Y * n + X] = c0 * u[Y * n + X] + c1 * (u[(Y - 1) * n + X] + u[(Y + 1) * n + X] + u[Y * n + X - 1] + u[Y * n + X + 1]);
}

// 8 matrices per group of 32 x 8 work-items; work-item (lr, lm) forms row lr of batch M
__global__ void k_matvec(const double *__restrict__ A, const double *__restrict__ x, double *__restrict__ y, int64_t b) {
  const int lr = threadIdx.x, lm = threadIdx.y;
  const int64_t M = 8 * (int64_t)blockIdx.x + lm;
  if (M >= b) return;
  double acc = 0.0;
  for (int k = 0; k < 32; k++) acc += A[(M * 32 + lr) * 32 + k] * x[M * 32 + k];
  y[M * 32 + lr] = acc;
}

// E elements per group, W work-items: each sums E / W elements, then a tree in local memory
__global__ void k_reduction(const float *__restrict__ a, float *__restrict__ out, int64_t n, int E) {
  extern __shared__ float s[];
  const int W = blockDim.x, l = threadIdx.x;
  float acc = 0.f;
  for (int ro = 0; ro < E / W; ro++) {
    const int64_t X = (int64_t)E * blockIdx.x + (int64_t)W * ro + l;
    if (X < n) acc = acc + a[X];
  }
  s[l] = acc;
  __syncthreads();
  for (int S = W / 2; S >= 1; S /= 2) {
    if (l < S) s[l] = s[l] + s[l + S];
    if (S > 1) __syncthreads();
  }
  if (l == 0) out[blockIdx.x] = s[0];
}

__global__ void k_axpy(const double *__restrict__ x, double *__restrict__ y, int64_t n, int E, double alpha) {
  const int W = blockDim.x;
  for (int ro = 0; ro < E / W; ro++) {
    const int64_t X = (int64_t)E * blockIdx.x + (int64_t)W * ro + threadIdx.x;
    if (X < n) y[X] = alpha * x[X] + y[X];
  }
}

__global__ void k_vecadd(const float *__restrict__ a, const float *__restrict__ b, float *__restrict__ c, int64_t n,
                         int E) {
  const int W = blockDim.x;
  for (int ro = 0; ro < E / W; ro++) {
    const int64_t X = (int64_t)E * blockIdx.x + (int64_t)W * ro + threadIdx.x;
    if (X < n) c[X] = a[X] + b[X];
  }
}

// All-pairs gravitation: work-item i sums the pull of every body j on body i.  Per
// pair: 3 subtractions, the squared distance (3 mul, 3 add with the softening), one
// rsqrt, inv^3 (2 mul), the mass factor (1 mul) and 3 accumulations (3 mul, 3 add).
__global__ void k_nbody(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                        const float *__restrict__ m, float *__restrict__ ax, float *__restrict__ ay,
                        float *__restrict__ az, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float xi = x[i], yi = y[i], zi = z[i];
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int64_t j = 0; j < n; j++) {
    const float dx = x[j] - xi, dy = y[j] - yi, dz = z[j] - zi;
    const float r2 = dx * dx + dy * dy + dz * dz + 1e-3f;
    const float inv = rsqrtf(r2);
    const float s = m[j] * (inv * inv * inv);
    sx = sx + dx * s;
    sy = sy + dy * s;
    sz = sz + dz * s;
  }
  ax[i] = sx;
  ay[i] = sy;
  az[i] = sz;
}

// 5 x 5 convolution over the valid region of an n x n image
__global__ void k_conv5(const float *__restrict__ in, const float *__restrict__ w, float *__restrict__ out,
                        int64_t n) {
  const int64_t Y = (int64_t)blockDim.y * blockIdx.y + threadIdx.y, X = (int64_t)blockDim.x * blockIdx.x + threadIdx.x;
  if (Y >= n - 4 || X >= n - 4) return;
  float acc = 0.f;
#pragma unroll
  for (int fy = 0; fy < 5; fy++)
#pragma unroll
    for (int fx = 0; fx < 5; fx++) acc = acc + w[fy * 5 + fx] * in[(Y + fy) * n + X + fx];
  out[Y * n + X] = acc;
}

unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

extern "C" pm_status pmm_time(const pmm_config *cfg, int32_t runs, int32_t skip, double *h_min_ms, double *h_mean_ms,
                              void *stream) {
  PM_TRACE("pmm_time");
  if (!cfg || !h_min_ms || !h_mean_ms) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: null argument");
  const pmm_config c = *cfg;
  if (runs <= skip || skip < 0 || runs > 1000) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: need 0 <= skip < runs <= 1000");
  if (c.kind < 0 || c.kind >= PMM_NKINDS) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: unknown kind");
  const int64_t n = c.n, m = c.m, l = c.l;
  const bool mm = c.kind == PMM_MATMUL || c.kind == PMM_MATMUL_NAIVE;
  if (n < 1 || n > (int64_t(1) << 30) || (mm && (m < 1 || l < 1 || m > 65536 || l > 65536 || n > 65536)))
    return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: bad sizes");
  const bool two_d = c.kind == PMM_EMPTY || c.kind == PMM_ARITH || c.kind == PMM_TRANSPOSE_P ||
                     c.kind == PMM_TRANSPOSE_R || c.kind == PMM_TRANSPOSE_W || mm || c.kind == PMM_STENCIL ||
                     c.kind == PMM_CONV5;
  if (c.kind == PMM_NBODY && n > (int64_t(1) << 20)) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: n-body n <= 2^20");
  if (c.kind == PMM_CONV5 && n < 5) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: convolution needs n >= 5");
  if (two_d && n > 65536) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: 2-D n must be <= 65536");
  const int gx = c.gx, gy = c.gy;
  if (gx < 1 || gy < 1 || gx * gy > 1024) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: bad group size");
  const int s = c.variant;
  if ((c.kind == PMM_VSA || c.kind == PMM_FILLED) && (s < 1 || s > 16))
    return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: stride must be 1..16");
  if ((c.kind == PMM_FILLED || c.kind == PMM_ARITH) && (c.k < 1 || c.k > 100000))
    return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: k must be 1..100000");
  if (c.kind == PMM_ARITH && (s < 0 || s > 4)) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: arithmetic type 0..4");
  const bool f64 = c.f64 != 0;
  if (f64 && !(c.kind == PMM_COPY || c.kind == PMM_SUM4 || c.kind == PMM_INDEX || c.kind == PMM_VSA ||
                (c.kind == PMM_ARITH && s <= 2)))
    return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: fp64 only for copy, sum4, index, scale-add and add/mul/div arithmetic");
  const size_t es = f64 ? 8 : 4;
  if ((c.kind == PMM_TRANSPOSE_P || c.kind == PMM_MATMUL) && !(gx == gy && (gx == 16 || gx == 32)))
    return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: tiles are 16x16 or 32x32");
  if ((c.kind == PMM_TRANSPOSE_R || c.kind == PMM_TRANSPOSE_W || c.kind == PMM_MATMUL_NAIVE ||
       c.kind == PMM_STENCIL) && gx != gy)
    return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: square tiles");
  const int E = s * s;
  if ((c.kind == PMM_REDUCTION || c.kind == PMM_AXPY || c.kind == PMM_VECADD) &&
      (gy != 1 || E < gx || E % gx || (c.kind == PMM_REDUCTION && (gx & (gx - 1)))))
    return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: variant^2 elements per group, a multiple of gx (a power of two for reductions)");
  if (c.kind == PMM_MATVEC && (gx != 256 || gy != 1)) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: matvec groups are 256");

  // device buffers: sizes in bytes
  std::vector<size_t> bytes;
  switch (c.kind) {
    case PMM_COPY: bytes = {(size_t)n * es, (size_t)n * es}; break;
    case PMM_SUM4: bytes = std::vector<size_t>(5, (size_t)n * es); break;
    case PMM_INDEX: bytes = {(size_t)n * es}; break;
    case PMM_VSA: bytes = std::vector<size_t>(3, (size_t)n * s * es); break;
    case PMM_FILLED: bytes = {(size_t)c.k * s * n * 4, (size_t)n * 4}; break;
    case PMM_ARITH: bytes = {(size_t)n * n * es}; break;
    case PMM_TRANSPOSE_P: case PMM_TRANSPOSE_R: case PMM_TRANSPOSE_W: case PMM_STENCIL:
      bytes = {(size_t)n * n * 4, (size_t)n * n * 4}; break;
    case PMM_MATMUL: case PMM_MATMUL_NAIVE: bytes = {(size_t)n * m * 4, (size_t)m * l * 4, (size_t)n * l * 4}; break;
    case PMM_MATVEC: bytes = {(size_t)n * 1024 * 8, (size_t)n * 32 * 8, (size_t)n * 32 * 8}; break;
    case PMM_REDUCTION: bytes = {(size_t)n * 4, (size_t)ceil_div(n, E) * 4}; break;
    case PMM_AXPY: bytes = {(size_t)n * 8, (size_t)n * 8}; break;
    case PMM_VECADD: bytes = std::vector<size_t>(3, (size_t)n * 4); break;
    case PMM_NBODY: bytes = std::vector<size_t>(7, (size_t)n * 4); break;
    case PMM_CONV5: bytes = {(size_t)n * n * 4, 25 * 4, (size_t)n * n * 4}; break;
    default: break;
  }
  size_t total = 0;
  for (size_t b : bytes) total += b;
  if (total > (size_t(64) << 30)) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: more than 64 GiB of buffers");
  std::vector<void *> buf(bytes.size(), nullptr);
  auto release = [&]() { for (void *p : buf) if (p) cudaFree(p); };
  for (size_t i = 0; i < bytes.size(); i++) {
    if (cudaMalloc(&buf[i], std::max<size_t>(bytes[i], 16)) != cudaSuccess) {
      release();
      return pm_set_error_c(PM_ERR_NOMEM, "pmm_time: device allocation failed");
    }
    cudaMemset(buf[i], 0, bytes[i]);
  }
  auto F = [&](int i) { return (float *)buf[i]; };
  auto D = [&](int i) { return (double *)buf[i]; };
  cudaStream_t st = (cudaStream_t)stream;
  auto launch = [&]() {
    const dim3 b1(gx), b2(gx, gy);
    switch (c.kind) {
      case PMM_EMPTY: k_empty<<<dim3(ceil_div(n, gx), ceil_div(n, gy)), b2, 0, st>>>(); break;
      case PMM_COPY:
        if (f64) k_copy<double><<<ceil_div(n, gx), b1, 0, st>>>(D(0), D(1), n);
        else k_copy<float><<<ceil_div(n, gx), b1, 0, st>>>(F(0), F(1), n);
        break;
      case PMM_SUM4:
        if (f64) k_sum4<double><<<ceil_div(n, gx), b1, 0, st>>>(D(0), D(1), D(2), D(3), D(4), n);
        else k_sum4<float><<<ceil_div(n, gx), b1, 0, st>>>(F(0), F(1), F(2), F(3), F(4), n);
        break;
      case PMM_INDEX:
        if (f64) k_index<double><<<ceil_div(n, gx), b1, 0, st>>>(D(0), n);
        else k_index<float><<<ceil_div(n, gx), b1, 0, st>>>(F(0), n);
        break;
      case PMM_VSA:
        if (f64) k_vsa<double><<<ceil_div(n, gx), b1, 0, st>>>(D(0), D(1), D(2), n, s, 1.5, 0.5);
        else k_vsa<float><<<ceil_div(n, gx), b1, 0, st>>>(F(0), F(1), F(2), n, s, 1.5f, 0.5f);
        break;
      case PMM_FILLED: k_filled<<<ceil_div(n, gx), b1, 0, st>>>(F(0), F(1), n, s, c.k); break;
      case PMM_ARITH: {
        const dim3 g(ceil_div(n, gx), ceil_div(n, gy));
        if (f64) {
          if (s == 0) k_arith<double, 0><<<g, b2, 0, st>>>(D(0), n, c.k);
          else if (s == 1) k_arith<double, 1><<<g, b2, 0, st>>>(D(0), n, c.k);
          else k_arith<double, 2><<<g, b2, 0, st>>>(D(0), n, c.k);
        } else if (s == 0) k_arith<float, 0><<<g, b2, 0, st>>>(F(0), n, c.k);
        else if (s == 1) k_arith<float, 1><<<g, b2, 0, st>>>(F(0), n, c.k);
        else if (s == 2) k_arith<float, 2><<<g, b2, 0, st>>>(F(0), n, c.k);
        else if (s == 3) k_arith<float, 3><<<g, b2, 0, st>>>(F(0), n, c.k);
        else k_arith<float, 4><<<g, b2, 0, st>>>(F(0), n, c.k);
        break;
      }
      case PMM_TRANSPOSE_P: {
        const dim3 g(ceil_div(n, gx), ceil_div(n, gx));
        if (gx == 16) k_transpose_p<16><<<g, b2, 0, st>>>(F(0), F(1), n);
        else k_transpose_p<32><<<g, b2, 0, st>>>(F(0), F(1), n);
        break;
      }
      case PMM_TRANSPOSE_R: k_transpose_r<<<dim3(ceil_div(n, gx), ceil_div(n, gx)), b2, 0, st>>>(F(0), F(1), n); break;
      case PMM_TRANSPOSE_W: k_transpose_w<<<dim3(ceil_div(n, gx), ceil_div(n, gx)), b2, 0, st>>>(F(0), F(1), n); break;
      case PMM_MATMUL: {
        const dim3 g(ceil_div(l, gx), ceil_div(n, gx));
        if (gx == 16) k_matmul<16><<<g, b2, 0, st>>>(F(0), F(1), F(2), n, m, l);
        else k_matmul<32><<<g, b2, 0, st>>>(F(0), F(1), F(2), n, m, l);
        break;
      }
      case PMM_MATMUL_NAIVE:
        k_matmul_naive<<<dim3(ceil_div(l, gx), ceil_div(n, gx)), b2, 0, st>>>(F(0), F(1), F(2), n, m, l);
        break;
      case PMM_STENCIL:
        k_stencil<<<dim3(ceil_div(std::max<int64_t>(n - 2, 0), gx), ceil_div(std::max<int64_t>(n - 2, 0), gx)), b2, 0,
                    st>>>(F(0), F(1), n, 0.5f, 0.125f);
        break;
      case PMM_MATVEC: k_matvec<<<ceil_div(n, 8), dim3(32, 8), 0, st>>>(D(0), D(1), D(2), n); break;
      case PMM_REDUCTION: k_reduction<<<ceil_div(n, E), b1, gx * 4, st>>>(F(0), F(1), n, E); break;
      case PMM_AXPY: k_axpy<<<ceil_div(n, E), b1, 0, st>>>(D(0), D(1), n, E, 1.5); break;
      case PMM_VECADD: k_vecadd<<<ceil_div(n, E), b1, 0, st>>>(F(0), F(1), F(2), n, E); break;
      case PMM_NBODY: k_nbody<<<ceil_div(n, gx), b1, 0, st>>>(F(0), F(1), F(2), F(3), F(4), F(5), F(6), n); break;
      case PMM_CONV5:
        k_conv5<<<dim3(ceil_div(std::max<int64_t>(n - 4, 1), gx), ceil_div(std::max<int64_t>(n - 4, 1), gy)), b2, 0,
                  st>>>(F(0), F(1), F(2), n);
        break;
      default: break;
    }
  };
  // an empty stencil interior or matmul grid still launches with at least one group
  if (c.kind == PMM_STENCIL && n < 3) { release(); return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_time: stencil needs n >= 3"); }
  std::vector<cudaEvent_t> ev(2 * runs);
  for (auto &e : ev) cudaEventCreate(&e);
  for (int r = 0; r < runs; r++) {
    cudaEventRecord(ev[2 * r], st);
    launch();
    cudaEventRecord(ev[2 * r + 1], st);
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  double mn = 1e300, sum = 0;
  for (int r = skip; r < runs && e == cudaSuccess; r++) {
    float ms = 0;
    e = cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
    mn = std::min(mn, (double)ms);
    sum += ms;
  }
  for (auto &x : ev) cudaEventDestroy(x);
  release();
  if (e != cudaSuccess) return pm_set_error(PM_ERR_CUDA, std::string("pmm_time: ") + cudaGetErrorString(e));
  *h_min_ms = mn;
  *h_mean_ms = sum / (runs - skip);
  return PM_OK;
}

// ------------------------------------------------------------------------------------ integer issue rate

namespace {

constexpr int II_CHAINS = 8;          // independent chains per lane
constexpr int II_OPS = 3;             // PTX operations per chain step: mad.lo, xor, add
constexpr int II_ITERS = 4096;

// Each lane advances 8 independent chains by one 32-bit multiply-add (the FMA pipe) and
// an xor and an add (the ALU pipe) per step, about the mix of the counting kernels.
__global__ void __launch_bounds__(256) k_int_issue(uint32_t *out, int iters) {
  uint32_t a[II_CHAINS], b[II_CHAINS];
#pragma unroll
  for (int j = 0; j < II_CHAINS; j++) {
    a[j] = threadIdx.x * 2654435761u + j;
    b[j] = blockIdx.x + 977u * j;
  }
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int j = 0; j < II_CHAINS; j++) {
      asm volatile("mad.lo.u32 %0, %0, 1664525, 1013904223;\n\t"
                   "xor.b32 %1, %1, %0;\n\t"
                   "add.u32 %0, %0, %1;\n\t"
                   : "+r"(a[j]), "+r"(b[j]));
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < II_CHAINS; j++) s ^= a[j] + b[j];
  if (s == 0x12345678u) out[0] = s;   // keeps the chains live; practically never stored
}

}  // namespace

extern "C" pm_status pmm_int_issue_rate(double *h_lane_ops_per_s, void *stream) {
  PM_TRACE("pmm_int_issue_rate");
  if (!h_lane_ops_per_s) return pm_set_error_c(PM_ERR_INVALID_ARG, "pmm_int_issue_rate: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 148, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_int_issue, 256, 0);
  const int grid = sms * std::max(1, per_sm);
  uint32_t *out = nullptr;
  cudaError_t e = cudaMalloc(&out, 4);
  if (e != cudaSuccess) return pm_set_error(PM_ERR_NOMEM, "pmm_int_issue_rate: device allocation");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_int_issue<<<grid, 256, 0, st>>>(out, II_ITERS);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; r++) {
    cudaEventRecord(e0, st);
    k_int_issue<<<grid, 256, 0, st>>>(out, II_ITERS);
    cudaEventRecord(e1, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return pm_set_error(PM_ERR_CUDA, std::string("pmm_int_issue_rate: ") + cudaGetErrorString(e));
  *h_lane_ops_per_s = (double)grid * 256 * II_ITERS * II_CHAINS * II_OPS / (best * 1e-3);
  return PM_OK;
}
