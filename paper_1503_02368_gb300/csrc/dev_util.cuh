// dev_util.cuh -- device helpers shared by the intersection kernels: 128-bit
// read-only loads, the bulk global->shared copy with its mbarrier, the bounded
// wait on that barrier, a lower-bound search, and the warp broadcast of a set
// descriptor.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "eh_internal.cuh"

namespace ehd {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t MBAR_SPIN_LIMIT = 1u << 24;          // bounded wait for a bulk copy: iterations
constexpr uint64_t MBAR_TIME_LIMIT_NS = 2000000000ull;  // ... and wall time (2 s)

__device__ __forceinline__ uint4 ldg4(const uint32_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completion counted on mbar (bytes % 16 == 0,
// both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true when the phase with the given parity completed within the limits
// (an iteration count and a wall-time bound, whichever comes first)
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity,
                                          uint64_t limit_ns = MBAR_TIME_LIMIT_NS) {
    uint32_t done = 0;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < MBAR_SPIN_LIMIT && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (!done && (it & 63) == 63 && global_ns() - t0 > limit_ns) break;
    }
    return done != 0;
}

// smallest index i in [lo, hi) with A[i] >= key (A sorted), or hi
__device__ __forceinline__ uint32_t lower_bound(const uint32_t *A, uint32_t lo, uint32_t hi, uint32_t key) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (A[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// descriptor held by lane `src`, broadcast to the warp (descriptors of upcoming
// pairs are loaded one per lane, in parallel, then handed out pair by pair)
__device__ __forceinline__ SetDesc bcast_desc(const SetDesc &d, int src) {
    SetDesc r;
    r.off = __shfl_sync(FULL, d.off, src);
    r.len = __shfl_sync(FULL, d.len, src);
    r.deg = __shfl_sync(FULL, d.deg, src);
    r.woff = __shfl_sync(FULL, d.woff, src);
    r.lo_word = __shfl_sync(FULL, d.lo_word, src);
    r.nwords = __shfl_sync(FULL, d.nwords, src);
    return r;
}

__device__ __forceinline__ SetDesc empty_desc() {
    SetDesc d;
    d.off = 0; d.len = 0; d.deg = 0; d.woff = 0; d.lo_word = 0; d.nwords = 0;
    return d;
}

}  // namespace ehd
