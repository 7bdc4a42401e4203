// Test hook for the bounded mbarrier wait of the tensor-core kernels (mbar_wait.cuh):
// one CTA initialises an mbarrier that expects one arrival and waits on its first
// phase with the given limit.  With complete = 1 a thread arrives first and the wait
// succeeds; with complete = 0 nothing arrives, the wait gives up after limit_ns, and
// the kernel reports that instead of hanging.  This is how the give-up path of the
// prediction and Gram kernels is tested without a kernel broken on purpose.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mbar_wait.cuh"
#include "pm.h"

namespace pmd {

__global__ void k_wait_probe(unsigned long long limit_ns, int complete, unsigned long long *out) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&mbar);
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
  __syncthreads();
  if (complete && threadIdx.x == 0)
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a) : "memory");
  const unsigned long long t0 = globaltimer_ns();
  const bool ok = cta_wait_bounded(a, 0, limit_ns);
  const unsigned long long t1 = globaltimer_ns();
  if (threadIdx.x == 0) {
    out[0] = ok ? 0ull : 1ull;
    out[1] = t1 - t0;
  }
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(a) : "memory");
}

}  // namespace pmd

// d_out: two uint64 on the device, [gave up (0/1), nanoseconds waited].  limit_ns is
// capped at 0.1 s.  Returns PM_OK once the kernel is launched.
extern "C" int pmx_wait_probe(unsigned long long limit_ns, int complete, unsigned long long *d_out, void *stream) {
  if (!d_out || limit_ns == 0 || limit_ns > 100000000ull) return PM_ERR_INVALID_ARG;
  pmd::k_wait_probe<<<1, 128, 0, (cudaStream_t)stream>>>(limit_ns, complete, d_out);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}
