// tma.cuh -- bulk asynchronous copies (cp.async.bulk, the TMA engine) from global to shared
// memory, completed on an mbarrier, with bounded waits.
#pragma once

#include <cstdint>

namespace lbehd {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make the initialisation visible to the asynchronous proxy that completes the copies.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Poll the barrier's phase at most max_polls times; false if it never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, int max_polls)
{
    for (int k = 0; k < max_polls; k++)
        if (mbar_try_wait(bar, phase))
            return true;
    return false;
}

}  // namespace lbehd
