// One-dimensional TMA bulk copies (cp.async.bulk) between global and shared memory, with
// an mbarrier for the loads.  Used where a block moves one contiguous, 16-byte aligned
// slice per operand: one thread issues the copy, the copy engine moves it at full width,
// and no thread spends registers or issue slots on the transfer.
//
// Every wait is bounded: after kMbarSpinLimit polls the waiting thread gives up, sets a
// flag in the context's device status word (lq_sync reports it as LQ_ERR_TIMEOUT), waits
// once more, again bounded, so that the block does not leave while its own copies may
// still be landing in its shared memory, and the block then skips its work (its outputs
// are left unwritten) instead of hanging the GPU.
#pragma once

#include <stdint.h>

namespace tma {

constexpr long kMbarSpinLimit = 1L << 24;

__device__ __forceinline__ uint32_t smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive on the barrier and tell it `bytes` more will be delivered by async copies.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem(bar)), "r"(bytes) : "memory");
}

// Global -> shared bulk copy completing on `bar` (dst, src 16-byte aligned, bytes % 16 == 0).
__device__ __forceinline__ void load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem(bar))
      : "memory");
}

// Bounded wait for phase `phase` of the barrier; false if `limit` polls did not see it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, long limit = kMbarSpinLimit) {
  for (long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Make this thread's generic-proxy shared-memory writes visible to the async proxy.
__device__ __forceinline__ void fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared -> global bulk store, committed as a bulk group; wait_all() waits until every
// committed store has finished reading shared memory (the block may then exit or reuse it;
// the global writes complete on their own, before the kernel is complete).
__device__ __forceinline__ void store(void* dst, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem(src_smem)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void wait_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

}  // namespace tma
