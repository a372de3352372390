// tma.cuh - bulk asynchronous copies (TMA engine) and mbarriers, inline PTX for sm_100-family.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tmem.cuh"

namespace hse {

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Arrive once and add `bytes` to the barrier's expected transaction count.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Wait for the barrier phase with a time limit (~1 s of SM clock); false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  const long long deadline = clock64() + 2000000000LL;
  while (!mbar_try_wait(bar, phase)) {
    if (clock64() > deadline) return false;
  }
  return true;
}

// Order earlier generic-proxy shared-memory accesses before later async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) global -> this CTA's
// shared memory, completing on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_copy_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr_u32(smem_dst)),
               "l"(gsrc), "r"(bytes), "r"(smem_addr_u32(bar))
               : "memory");
}

// 2-D tensor copy (TMA) of one box at coordinates (c0, c1) into this CTA's shared memory
// (128-byte aligned destination), completing on `bar`.
__device__ __forceinline__ void tensor_copy_2d_g2s(void* smem_dst, const void* tmap, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr_u32(smem_dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(smem_addr_u32(bar))
      : "memory");
}

}  // namespace hse
