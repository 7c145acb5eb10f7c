// Tensor-memory-accelerator (TMA) copies and mbarrier waits, written from the
// PTX instruction set: a CTA stages tiles of the padded level arrays into
// shared memory with cp.async.bulk.tensor, completion counted in bytes on an
// mbarrier per ring slot.  Every wait is bounded by a poll count; a wait that
// runs out returns false and the caller reports it (no kernel spins forever).
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace hhg {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One arrival (the issuing thread) per phase.
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The issuing thread arrives and announces the bytes the copies will deliver.
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Counts `bytes` of the current phase's announced transaction as delivered
// (used to withdraw bytes announced in excess).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity; false if it did not
// complete within `polls` tests.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long polls) {
  const uint32_t a = smem_addr(bar);
  for (long long it = 0; it < polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Shared memory last read through the generic proxy is about to be written
// by the async proxy (a TMA copy into a reused ring slot).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 4-D tiled load of the box at coordinates (c0, c1, c2, c3) of the map.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace hhg
