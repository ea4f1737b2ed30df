// Shared-memory barriers and bulk copies (TMA) of the kernels, with bounded waits.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pat {

// TMA bulk copies global -> shared completing on an mbarrier.  Sources,
// destinations and sizes are multiples of 16 bytes.
__device__ __forceinline__ uint32_t s_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* mb, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(mb)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also announces `bytes` of copies to come
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* mb, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     s_addr(mb)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* mb) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     s_addr(dst)),
                 "l"(src), "r"(bytes), "r"(s_addr(mb))
                 : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of mb for at most limit_ns of wall time; on giving up the
// status word gets bit 1 (PAT_STATUS_WAIT of pat_status) and the caller goes on.
__device__ __forceinline__ void mbar_wait(uint64_t* mb, uint32_t parity, int* status,
                                          uint64_t limit_ns = 2000000000ull) {
    uint32_t done = 0;
    const uint64_t t0 = global_ns();
    for (;;) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(s_addr(mb)), "r"(parity)
            : "memory");
        if (done || global_ns() - t0 > limit_ns) break;
    }
    if (!done && status) atomicOr(status, 2);
}

// Wait for phase `parity` of mb for at most limit_ns of wall time; true if it completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mb, uint32_t parity, uint64_t limit_ns) {
    uint32_t done = 0;
    const uint64_t t0 = global_ns();
    for (;;) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(s_addr(mb)), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

}  // namespace pat
