// Device helpers: bulk async copies into shared memory completed on an
// mbarrier, mbarrier waits bounded by an iteration limit (a wait that runs
// out records ERR_TIMEOUT and returns false instead of spinning forever),
// warp reductions and order-preserving keys for floats.
#pragma once

#include <stdint.h>

#include "sivf_internal.cuh"

namespace sivf {

// -------------------------------------------------------------- mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(count));
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile(
        "{\n .reg .b64 st;\n"
        " mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile(
        "{\n .reg .b64 st;\n"
        " mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// nanoseconds of the GPU's global timer
__device__ __forceinline__ uint64_t gtimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}


// Wait for phase `parity` of `bar`, giving up once `limit_ns` of global
// time has passed since the first unsuccessful poll (each try_wait itself
// suspends for a hardware-defined time; a poll count of 2^30 is a second
// limit in case the timer stalls).  Returns false and sets ERR_TIMEOUT
// when a limit is hit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint32_t *err,
                                                  uint64_t limit_ns = kWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer_ns();
    for (uint32_t it = 1; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (gtimer_ns() - t0 > limit_ns) break;
    }
    atomicOr(err, ERR_TIMEOUT);
    return false;
}

// One bulk copy global -> shared of `bytes` (multiple of 16, both addresses
// 16-byte aligned) that completes transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem,
                                         uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------- warps
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// (distance, id) lexicographic order used by every top-k
__device__ __forceinline__ bool dk_less(float a, int64_t ia, float b, int64_t ib)
{
    return a < b || (a == b && ia < ib);
}

// float -> uint32 key with the same order (for radix selection)
__device__ __forceinline__ uint32_t fkey(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float fkey_inv(uint32_t k)
{
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// Ascending (distance, id) bitonic sort of 32*E elements held E per lane
// (element i = lane + 32 e); pads are (+inf, -1).
template <int E>
__device__ __forceinline__ void warp_bitonic_sort(float (&v)[E], int64_t (&id)[E], int lane)
{
    constexpr int N = 32 * E;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1)
#pragma unroll
        for (int st = size >> 1; st > 0; st >>= 1)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane + 32 * e;
                const bool up = (i & size) == 0;
                if (st >= 32) {
                    const int pe = e ^ (st >> 5);
                    if (pe > e) {
                        const bool sw = up ? dk_less(v[pe], id[pe], v[e], id[e])
                                           : dk_less(v[e], id[e], v[pe], id[pe]);
                        if (sw) {
                            const float tv = v[e];
                            v[e] = v[pe];
                            v[pe] = tv;
                            const int64_t ti = id[e];
                            id[e] = id[pe];
                            id[pe] = ti;
                        }
                    }
                } else {
                    const float ov = __shfl_xor_sync(0xffffffffu, v[e], st);
                    const int64_t oi = __shfl_xor_sync(0xffffffffu, id[e], st);
                    const bool lower = (lane & st) == 0;
                    const bool take = (lower == up) ? dk_less(ov, oi, v[e], id[e])
                                                    : dk_less(v[e], id[e], ov, oi);
                    if (take) {
                        v[e] = ov;
                        id[e] = oi;
                    }
                }
            }
}

}  // namespace sivf
