// mbarrier waits and bulk global-to-shared copies shared by the tensor-core GEMMs and the
// triangular solves.  Every wait is bounded: kWaitLimit polls, then the caller is told it failed.
#pragma once

#include <cstdint>

namespace pdd {

static constexpr long long kWaitLimit = 1LL << 22;   // polls before a wait is declared failed

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try(mbar, parity)) return true;
    return false;
}

// the same wait for a role that has nothing else to do meanwhile: each poll suspends the thread up
// to `ns` nanoseconds (it resumes as soon as the phase completes), so a waiting warp stops taking
// issue slots from the warps doing the work; bounded by kSleepWaitLimit polls
static constexpr long long kSleepWaitLimit = 1LL << 20;

__device__ __forceinline__ bool mbar_try_sleep(uint32_t mbar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_sleep(uint32_t mbar, uint32_t parity, uint32_t ns = 2000) {
    for (long long i = 0; i < kSleepWaitLimit; ++i)
        if (mbar_try_sleep(mbar, parity, ns)) return true;
    return false;
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

}  // namespace pdd
