// bulk_copy.cuh -- inline-PTX helpers for the Blackwell bulk-copy engine
// (cp.async.bulk, TMA without a tensor map) and shared-memory mbarriers.
//
// Rules the callers follow:
//  * every address and size handed to a bulk copy is a multiple of 16 bytes;
//  * a bulk load completes on an mbarrier (transaction count in bytes);
//  * generic-proxy writes to shared memory that a bulk store will read are
//    published with fence_proxy_async_smem() by every writing thread, then a
//    CTA barrier, before the store is issued;
//  * every wait on an mbarrier is bounded (mbar_wait returns false when it
//    gives up), so a copy that never lands ends in an error status, not a hang.
#pragma once
#include <cstdint>

namespace akmc {
namespace bulk {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gmem_addr(const void* p) {
    uint64_t g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(p));
    return g;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// makes the initialised barriers visible to the bulk-copy engine
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// one arrival that also announces `bytes` of bulk-copy transactions
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Waits until the phase of parity `parity` has completed; gives up after
// `max_polls` polls (each poll may suspend the thread for a short,
// hardware-defined time) and then returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t max_polls) {
    for (uint32_t t = 0; t < max_polls; ++t) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// global -> shared, completion counted on `bar`
__device__ __forceinline__ void load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(gmem_addr(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

// shared -> global, tracked in this thread's bulk groups
__device__ __forceinline__ void store(void* dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem_addr(dst)), "r"(src),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// every committed store of this thread has finished reading shared memory
__device__ __forceinline__ void wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store of this thread is complete
__device__ __forceinline__ void wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// orders this thread's generic-proxy shared-memory writes before later
// bulk-copy (async-proxy) reads of them
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace bulk
}  // namespace akmc
