// ttsh_wait.cuh - the bounded wait every kernel of the library uses for an mbarrier phase
// (TMA and bulk-copy completion, tensor-core completion).
#pragma once

namespace ttsh {

// Bounded wait for phase `parity` of the shared-memory mbarrier at `bar`: mbarrier.try_wait
// polls until the phase completes or `limit_ns` of global time has passed; false = timed out
// (the caller records it in its status word and carries on, so a lost completion never hangs
// the GPU).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s for the production waits
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    unsigned done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

}  // namespace ttsh
