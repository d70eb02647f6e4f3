// bulk.cuh -- one-dimensional bulk copies global -> shared memory by the
// tensor memory accelerator (cp.async.bulk), completed on shared-memory
// mbarriers, as inline PTX for sm_103a.
//
// Pattern: one thread arms a barrier with the number of bytes a stage will
// receive (arrive.expect_tx), then any threads issue the copies of that
// stage (each completes its bytes on the barrier), and the consumers wait
// for the barrier's phase.  Sources and destinations must be 16-byte aligned
// and sizes multiples of 16 bytes.  A buffer that was read with ordinary
// loads is handed back to the copy engine with fence_proxy_async() (after
// the readers are done) before the next copy into it is issued.
#pragma once
#include <cstdint>

namespace ncorp {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// makes initialised barriers visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
        ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// one arrival (no bytes) on the barrier
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}"
        ::"r"(smem_addr(bar)) : "memory");
}

// true when the barrier's phase with the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// bytes from global src to shared dst, completed on bar (16-byte aligned, multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// orders earlier ordinary accesses to shared memory before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace ncorp
