// Bulk asynchronous global -> shared copies with mbarrier completion (sm_90+
// PTX: cp.async.bulk, mbarrier.*), written as thin inline-PTX wrappers.
//
// Use pattern (one warp owning a buffer and its barrier):
//   lane 0: mbar_init(bar, 1) once, then fence_mbarrier_init(); __syncwarp()
//   lane 0: fence_proxy_async(); mbar_expect_tx(bar, bytes); bulk_g2s(dst, src, bytes, bar)
//   all lanes: mbar_wait(bar, parity) -- the phase completes when the copy's
//              bytes have landed; parity alternates 0, 1, 0, ... per use
// Addresses and sizes of cp.async.bulk must be multiples of 16 bytes.
#pragma once

#include <cstdint>

namespace sph {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// makes barrier initialisations visible to the asynchronous (copy) proxy
__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// orders this thread's earlier shared-memory accesses before later
// asynchronous-proxy accesses (a buffer read by the warp, then refilled by a copy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one arrival that also announces `bytes` of transactions to complete the phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// waits for the phase of the given parity, giving up after about `cycles` SM
// clock cycles (false: the copy did not complete in time)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long cycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > cycles) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace sph
