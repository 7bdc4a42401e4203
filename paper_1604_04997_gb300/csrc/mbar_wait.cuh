// Bounded mbarrier waits for the tensor-core kernels (predict_tc.cu, gram_tc.cu).
// A wait polls mbarrier.try_wait on one phase parity and gives up after a time limit
// read from the global nanosecond timer, so that a copy or an MMA that never
// completes turns into an error status (ST_TIMEOUT) instead of a kernel that never
// returns.  pmx_wait_probe (probe.cu) runs the same wait on a barrier that nothing
// completes, so the give-up path is exercised by a test without a broken kernel.
#pragma once
#include <stdint.h>

namespace pmd {

constexpr unsigned long long MBAR_WAIT_NS = 2000000000ull;   // 2 s

// true once the phase with the given parity has completed
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// Wait of the whole CTA on one mbarrier phase (every thread calls it): true if every
// thread saw the phase complete within limit_ns, false if any gave up.
__device__ __forceinline__ bool cta_wait_bounded(uint32_t mbar, uint32_t parity,
                                                 unsigned long long limit_ns = MBAR_WAIT_NS) {
  int timed_out = 0;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try(mbar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) {
      timed_out = 1;
      break;
    }
  }
  return !__syncthreads_or(timed_out);
}

}  // namespace pmd
