// Inline-PTX helpers for asynchronous staging into shared memory:
// shared-memory mbarriers, 16-byte cp.async copies whose completion a
// barrier tracks, and global loads with L2 cache policies. Every wait is
// bounded: on timeout the kernel records an error in a device status word
// instead of spinning forever.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ld_common.cuh"

namespace ld {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the asynchronous copy units.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// L2 policy that keeps the copied lines resident in preference to others.
__device__ __forceinline__ uint64_t make_l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// L2 policy whose lines are evicted first (a value's last use).
__device__ __forceinline__ uint64_t make_l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Global loads with an L2 cache policy, for 32-, 16- and 64-bit storage
// words. The _now forms are volatile: the compiler keeps them where they are
// written, which is how a kernel issues a load early (before a barrier) to
// overlap its latency with other work.
#define LD_DEFINE_L2_HINT_LOADS(NAME, QUAL)                                                        \
    __device__ __forceinline__ float NAME(const float* p, uint64_t pol) {                          \
        float v;                                                                                   \
        asm QUAL("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));     \
        return v;                                                                                  \
    }                                                                                              \
    __device__ __forceinline__ double NAME(const double* p, uint64_t pol) {                        \
        double v;                                                                                  \
        asm QUAL("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));     \
        return v;                                                                                  \
    }                                                                                              \
    template <class T>                                                                             \
    __device__ __forceinline__ T NAME(const T* p, uint64_t pol) {                                  \
        static_assert(sizeof(T) == 2, "16-bit storage word");                                      \
        unsigned short bits;                                                                       \
        asm QUAL("ld.global.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(bits) : "l"(p), "l"(pol));  \
        T v;                                                                                       \
        memcpy(&v, &bits, 2);                                                                      \
        return v;                                                                                  \
    }
LD_DEFINE_L2_HINT_LOADS(ld_l2_hint, )
LD_DEFINE_L2_HINT_LOADS(ld_l2_hint_now, volatile)
#undef LD_DEFINE_L2_HINT_LOADS

// Two consecutive storage words (8- or 4-byte aligned) with an L2 policy:
// FP32 as a pair of floats, the 16-bit forms as their raw 32-bit pattern
// (low half = the lower address).
__device__ __forceinline__ float2 ld_l2_hint_pair(const float* p, uint64_t pol) {
    float2 v;
    asm("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ unsigned ld_l2_hint_pair(const void* p, uint64_t pol) {
    unsigned v;
    asm("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
// Four 16-bit values (8 bytes, 8-byte aligned) with an L2 cache policy.
__device__ __forceinline__ uint2 ld_l2_hint_quad(const void* p, uint64_t pol) {
    uint2 v;
    asm("ld.global.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}
// The same, issued where it is written (volatile), to overlap its latency.
__device__ __forceinline__ unsigned ld_l2_hint_pair_now(const void* p, uint64_t pol) {
    unsigned v;
    asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
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

// Wait for the phase with the given parity to complete; false (and the
// status bit set) if it did not within max_polls polls.
__device__ __forceinline__ bool mbar_wait_bounded_n(uint32_t bar, uint32_t parity, int* status, int max_polls) {
    for (int it = 0; it < max_polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(status, kStatusWaitTimeout);
    return false;
}

// 16-byte copy global -> this CTA's shared memory (cp.async, cached in L2
// only) with an L2 policy. Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint64_t policy) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(policy)
                 : "memory");
}

// Close the group of this thread's cp.async copies issued so far; wait until
// all of its groups have landed (a hardware wait: the copies always land).
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_group0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

}  // namespace ld
