// Staging a contiguous run of global memory into shared memory with the
// bulk-copy engine (cp.async.bulk, completion on an mbarrier): one thread
// issues the whole copy and the CTA waits on the barrier's phase, instead of
// every thread looping over load / store pairs.  Every wait is bounded.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace clue {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// One CTA-scope mbarrier expecting one arrival (the issuing thread's) per
// phase.  Initialised once per CTA, before its first use, by one thread;
// a __syncthreads must follow before any thread waits on it.
__device__ __forceinline__ void bulk_bar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// `src` to shared `dst`, completing the barrier's current phase.  Called by
// one thread after a __syncthreads that ends every earlier access to `dst`
// (the proxy fence orders those accesses before the engine's writes).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool bulk_bar_test(unsigned long long *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (every thread of the CTA) for the phase with the given parity to
// complete, giving up after about `limit_ns` of device time; the result is
// the same in every thread (a CTA-wide vote), false when any thread gave up.
__device__ __forceinline__ bool bulk_bar_wait(unsigned long long *bar, unsigned parity,
                                              unsigned long long limit_ns) {
    bool done = bulk_bar_test(bar, parity);
    if (!done) {
        const unsigned long long t0 = global_ns();
        while (!(done = bulk_bar_test(bar, parity)))
            if (global_ns() - t0 > limit_ns) break;
    }
    return __syncthreads_and(done) != 0;
}

}  // namespace clue
