// Inline-PTX helpers: mbarrier phases, bulk global->shared copies (the
// non-tensor form of TMA), proxy fences and bounded waits.
//
// Every wait is bounded by a cycle budget.  A wait that runs out returns false;
// the caller records FTLM_ETIMEOUT in the device error word, then waits out the
// copies it has already issued (drain, with its own bound) before it leaves, so
// that no asynchronous copy can land in shared memory after the CTA exits.
#pragma once

#include <stdint.h>

namespace ftlm {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr unsigned long long kDrainCycles = 1ull << 32;  // about two seconds at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// generic-proxy accesses of shared memory before later async-proxy accesses (and back)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared; completion on bar
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Hint to bring the 128-byte line holding p into L2; nothing to wait for, and
// no effect on correctness.
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// One potentially blocking probe of the phase with the given parity (the
// hardware may suspend the thread for a system-dependent time while the phase
// is incomplete).
__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok;
}

// Non-blocking probe of the phase with the given parity.
__device__ __forceinline__ uint32_t mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok;
}

// Warp-uniform wait for the phase of the given parity, at most `limit` cycles
// (measured by lane 0's clock).  Returns false if the budget ran out.  The
// first probe does not suspend, so a budget shorter than the copy latency
// runs out deterministically.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned long long limit) {
    const long long t0 = clock64();
    if (__all_sync(kFullMask, mbar_test_wait(bar, parity))) return true;
    for (;;) {
        const long long dt = __shfl_sync(kFullMask, clock64() - t0, 0);
        if ((unsigned long long)dt > limit) return false;
        const uint32_t ok = mbar_try_wait(bar, parity);
        if (__all_sync(kFullMask, ok)) return true;
    }
}

}  // namespace ftlm
