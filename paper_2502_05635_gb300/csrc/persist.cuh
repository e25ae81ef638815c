// Building blocks of the persistent single-trajectory kernels: %globaltimer, mbarriers,
// 1D bulk copies (cp.async.bulk) into a shared-memory ring, bounded waits and a grid-wide
// barrier on a monotonic arrival counter.  Every wait has a budget in ns; on expiry the
// caller raises its CTA's abort flag and the host reports TDAGW_ERR_TIMEOUT.
#pragma once

#include "common.cuh"

namespace tdagw {
namespace persist {

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase of the given parity; false if the budget ran out or abort was raised
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_s,
                                          unsigned long long budget) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(b, parity)) return true;
        if ((i & 63) == 0) {
            if (abort_s && *abort_s) return false;
            if (gtimer() - t0 > budget) return false;
        }
    }
}
// global -> shared bulk copy completing on an mbarrier, with an L2 cache policy
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            saddr(dst)),
        "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(policy)
        : "memory");
}
// the same without a cache policy
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            saddr(dst)),
        "l"(src), "r"(bytes), "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// named barrier 1 among the first NT threads of the CTA
template <int NT> __device__ __forceinline__ void named_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Grid-wide barrier among the first NT threads of every CTA.  The arrival counter only
// grows: barrier number g (1, 2, ...) is complete once it reaches g * (gridDim.x + extra),
// so no reset is needed and arrivals are fire-and-forget reductions at L2.  The named
// barrier orders this CTA's prior stores before thread 0's release (cumulative); the
// acquire load orders the CTA's later loads after the other CTAs' releases.  Returns false
// (and raises abort) if the barrier did not complete within the budget.
template <int NT>
__device__ bool grid_sync(unsigned long long* bar_count, int* err, int extra, unsigned long long wait_ns,
                          unsigned& lgen, volatile int* abort_s) {
    named_sync<NT>();
    if (threadIdx.x == 0 && !*abort_s) {
        const unsigned long long target = (unsigned long long)(lgen + 1) * (gridDim.x + (unsigned)extra);
        red_release_add64(bar_count, 1ull);
        if (ld_acquire64(bar_count) < target) {
            const uint64_t t0 = gtimer();
            while (ld_acquire64(bar_count) < target) {
                if (gtimer() - t0 > wait_ns || *(volatile int*)err) {
                    atomicExch(err, 1);
                    *abort_s = 1;
                    break;
                }
                __nanosleep(20);
            }
        }
        lgen += 1;
    }
    named_sync<NT>();
    return !*abort_s;
}

// Position in the shared-memory ring: slot index and the parity of its current use.
struct RingPos {
    int slot;
    uint32_t phase;
    __device__ __forceinline__ void advance(int by, int ns) {
        slot += by;
        while (slot >= ns) {
            slot -= ns;
            phase ^= 1u;
        }
    }
};

// One lane waits for the slot, then the warp proceeds (bar.warp.sync orders the lanes'
// shared-memory reads after lane 0's acquire of the mbarrier phase).
__device__ __forceinline__ bool warp_wait_full(uint64_t* full, RingPos p, volatile int* abort_s,
                                               unsigned long long budget, int lane) {
    int ok = 1;
    if (lane == 0) ok = (!*abort_s && mbar_wait(full + p.slot, p.phase, abort_s, budget)) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok && lane == 0) *abort_s = 1;
    return ok != 0;
}

// Observables of one step from per-CTA partials red[3 c + {0,1,2}] (one warp; fixed order).
__device__ __forceinline__ void reduce_obs_row(const double* red, int G, double inv, double* out, int lane) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = lane; c < G; c += 32) {
        s0 += __ldcg(red + 3 * c);
        s1 += __ldcg(red + 3 * c + 1);
        s2 += __ldcg(red + 3 * c + 2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        out[0] = s0 * inv;
        out[1] = s1 * inv;
        out[2] = s2 * inv;
    }
}

}  // namespace persist
}  // namespace tdagw
