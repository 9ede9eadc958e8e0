// tma.cuh -- bulk asynchronous copies from global to shared memory (the
// tensor memory accelerator's untiled form, cp.async.bulk) completed on a
// shared-memory mbarrier, and a bounded wait for them.
//
// A copy needs 16-byte aligned source and destination and a size that is a
// multiple of 16 bytes.  A block that issued copies must not exit before they
// have landed: some thread of it waits for the barrier on every path.
#pragma once

#include <stdint.h>

namespace sg {

// Polls of an mbarrier before a wait gives up (each poll may itself suspend
// the thread for a short, hardware-defined time).
constexpr uint32_t kBulkWaitPolls = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// One arrival expected; the phase also waits for the transaction bytes.
__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The single arrival, announcing `bytes` of copies that complete on bar.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Wait for phase `parity` of bar to complete; false if it did not within
// kBulkWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kBulkWaitPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace sg
