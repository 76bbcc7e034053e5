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

// ------------------------------------------------------------ load checks
//
// With EH_CHECK_LOADS defined (the checked build, libeh_check.so) every
// global load of the count kernels goes through the functions below, which
// verify that the bytes lie inside one of the arrays the kernel was given
// (registered per CTA in shared memory by chk_register at kernel start).  A
// load outside them is not made: it sets DEV_ST_BOUNDS in the kernel's status
// word and yields a harmless value (EH_PAD elements, zero words, an empty
// descriptor), so the run ends with an error status instead of a fault.
// Without the flag they are plain read-only loads.
#ifdef EH_CHECK_LOADS
constexpr int CHK_MAX = 12;
struct ChkTable {
    uintptr_t lo[CHK_MAX], hi[CHK_MAX];   // byte ranges [lo, hi)
    uint32_t *status;
    int n;
};
static __shared__ ChkTable s_chk;

// thread 0 of the CTA; the caller synchronises before the first checked load
__device__ __forceinline__ void chk_reset(uint32_t *status) {
    s_chk.n = 0;
    s_chk.status = status;
}
__device__ __forceinline__ void chk_add(const void *p, uint64_t bytes) {
    if (s_chk.n < CHK_MAX && p) {
        s_chk.lo[s_chk.n] = (uintptr_t)p;
        s_chk.hi[s_chk.n] = (uintptr_t)p + bytes;
        ++s_chk.n;
    }
}
__device__ __forceinline__ bool chk_ok(const void *p, uint32_t bytes) {
    if (!__isGlobal(p)) return true;   // shared-memory operands are indexed by construction
    const uintptr_t a = (uintptr_t)p;
    for (int i = 0; i < s_chk.n; ++i)
        if (a >= s_chk.lo[i] && a + bytes <= s_chk.hi[i]) return true;
    if (s_chk.status) atomicOr(s_chk.status, DEV_ST_BOUNDS);
    return false;
}
#endif

__device__ __forceinline__ uint4 ldg4(const uint32_t *p) {
#ifdef EH_CHECK_LOADS
    if (!chk_ok(p, 16)) return make_uint4(EH_PAD, EH_PAD, EH_PAD, EH_PAD);
#endif
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// one 32-bit element or word (a miss in the checked build reads EH_PAD)
__device__ __forceinline__ uint32_t ldg1(const uint32_t *p) {
#ifdef EH_CHECK_LOADS
    if (!chk_ok(p, 4)) return EH_PAD;
#endif
    return __ldg(p);
}

// a 32-bit element of a set that may be in shared or global memory
__device__ __forceinline__ uint32_t ld_any(const uint32_t *p) {
#ifdef EH_CHECK_LOADS
    if (!chk_ok(p, 4)) return EH_PAD;
#endif
    return *p;
}

// a set descriptor (a miss in the checked build reads an empty one)
__device__ __forceinline__ SetDesc ld_desc(const SetDesc *p) {
#ifdef EH_CHECK_LOADS
    if (!chk_ok(p, sizeof(SetDesc))) {
        SetDesc d;
        d.off = 0; d.len = 0; d.deg = 0; d.woff = 0; d.lo_word = 0; d.nwords = 0;
        return d;
    }
#endif
    return *p;
}

// the source of a bulk copy lies inside a registered array (always true
// without the checked build)
__device__ __forceinline__ bool bulk_src_ok(const void *p, uint32_t bytes) {
#ifdef EH_CHECK_LOADS
    return chk_ok(p, bytes);
#else
    (void)p; (void)bytes;
    return true;
#endif
}

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

// smallest index i in [lo, hi) with A[i] >= key (A sorted; shared or global), or hi
__device__ __forceinline__ uint32_t lower_bound(const uint32_t *A, uint32_t lo, uint32_t hi, uint32_t key) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
#ifdef EH_CHECK_LOADS
        const uint32_t am = chk_ok(&A[mid], 4) ? A[mid] : EH_PAD;
#else
        const uint32_t am = A[mid];
#endif
        if (am < key) lo = mid + 1; else hi = mid;
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
