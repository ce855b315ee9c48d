// mbarrier and bulk-copy primitives (inline PTX) shared by the kernels that stage data
// through shared memory with the Tensor Memory Accelerator. Every wait is bounded.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace tn {

constexpr uint64_t kWaitNs = 4000000000ull;  // 4 s bound on any wait

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity` to complete; false after limit_ns (%globaltimer).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  if (mbar_test(b, parity)) return true;
  const uint64_t t0 = gtime();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_test(b, parity)) return true;
    if (gtime() - t0 > limit_ns) return false;
  }
}

// One contiguous global -> shared copy by the bulk-copy engine (cp.async.bulk): both
// addresses 16-byte aligned, bytes a multiple of 16; completion counts `bytes` against the
// barrier's transaction count.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(su32(bar))
      : "memory");
}

}  // namespace tn
