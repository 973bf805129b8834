// Bulk asynchronous copies (the untiled TMA path, cp.async.bulk) from global into shared
// memory, completed on an mbarrier, and a bounded wait on that mbarrier.
//
// Rules the callers keep: source and destination 16-byte aligned, size a multiple of 16
// bytes; one thread arms a barrier (arrive + expected bytes) and issues the copies of one
// phase; every waiting thread passes the parity of the phase it waits for (0, 1, 0, ...).
#pragma once
#include <cstdint>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make barrier initialisation visible to the async (TMA) proxy before the first copy.
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Order this thread's generic-proxy shared-memory accesses before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Non-blocking probe of the phase of the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of the given parity; gives up (returns false) after about `cycles` SM
// clocks (2^31: about one second at 2 GHz), so a copy that never lands cannot hang the GPU.
// Limits below 2^20 cycles (diagnostics) probe with the non-blocking test_wait, whose result
// is not held back by the suspend window that try_wait may spend inside one call.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long cycles = (1ll << 31)) {
    if (cycles < (1ll << 20)) {
        const long long t0 = clock64();
        do {
            if (mbar_test_wait(bar, parity)) return true;
        } while (clock64() - t0 < cycles);
        return false;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}

// Device status word of a handle: 0 while healthy; kernels that give up a wait store a code.
#define BI_DEVSTATUS_TMA_TIMEOUT 1

// Thread 0 of a CTA whose ring of S stages (one mbarrier each, chunk c on stage c % S with
// parity (c / S) & 1) gave up waiting at chunk `first`: wait again, with the default limit of
// about one second, for the chunks still in flight so that no copy lands after the CTA has
// left, then record the failure in the status word.
__device__ __forceinline__ void bulk_give_up(uint64_t* bar, int first, int nchunks, int S, int* status) {
    if (threadIdx.x != 0) return;
    for (int c = first; c < first + S && c < nchunks; ++c) mbar_wait_bounded(&bar[c % S], (c / S) & 1);
    atomicExch(status, BI_DEVSTATUS_TMA_TIMEOUT);
}
