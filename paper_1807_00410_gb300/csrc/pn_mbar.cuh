// mbarrier and bulk-copy (TMA) helpers shared by the TMA-staged kernels.
// Every wait is bounded: after about 2 s of %globaltimer it sets *err,
// marks the caller as failed (its later waits return at once) and returns.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pn {
namespace mbar {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// make initialised barriers visible to the copy engine
__device__ __forceinline__ void fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of `bar` to complete, for at most limit_ns of
// %globaltimer; when the limit runs out it sets *err (if not null), marks the
// caller failed (its later waits return at once) and returns.
__device__ __forceinline__ void wait_ns(uint32_t bar, uint32_t parity, unsigned int* err, bool& failed,
                                        uint64_t limit_ns) {
    if (try_wait(bar, parity) || failed) return;
    const uint64_t t0 = global_ns();
    while (!try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) {
            failed = true;
            if (err) atomicExch(err, 1u);
            return;
        }
    }
}

__device__ __forceinline__ void wait(uint32_t bar, uint32_t parity, unsigned int* err, bool& failed) {
    wait_ns(bar, parity, err, failed, 2000000000ull);
}

// 1D bulk copy global -> shared of `bytes` (a multiple of 16; both addresses
// 16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
        : "memory");
}

}  // namespace mbar
}  // namespace pn
