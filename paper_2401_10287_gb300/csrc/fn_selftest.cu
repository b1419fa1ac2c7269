// Failure-path self-test: a kernel whose barrier wait can never complete.
//
// The tensor-core kernels bound every mbarrier wait by %globaltimer; when a wait expires
// they set the timeout bit of the device status word and return, and fn_sync reports
// FN_ERR_TIMEOUT.  This kernel exercises that path without a fault: each thread of one CTA
// waits on a shared-memory mbarrier that nothing arrives at, bounded by a deadline and,
// independently, by an iteration cap, then records the timeout bit.
#include "fn_internal.cuh"

namespace fn {

__global__ void __launch_bounds__(32) k_expired_wait(uint64_t wait_ns, uint64_t max_iters, int* status) {
  __shared__ uint64_t bar;
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(&bar);
  const uint32_t one = 1u, parity = 0u;
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(one) : "memory");
  __syncthreads();
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  bool done = false;
  for (uint64_t it = 0; it < max_iters && !done; ++it) {
    uint32_t d;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(d)
        : "r"(addr), "r"(parity)
        : "memory");
    done = d != 0;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > wait_ns) break;
  }
  if (!done && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

void launch_expired_wait(const fn_system* s, int wait_us, cudaStream_t st) {
  // one iteration takes well over 1 ns, so a cap of wait_us * 1000 iterations ends the loop
  // (wait_us <= 100000) within seconds even if the timer stalled
  const uint64_t cap = (uint64_t)wait_us * 1000ull;
  k_expired_wait<<<1, 32, 0, st>>>((uint64_t)wait_us * 1000ull, cap, s->ws.status);
}

}  // namespace fn
