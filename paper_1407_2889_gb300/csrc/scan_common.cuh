// scan_common.cuh -- device helpers shared by the Aho-Corasick and Wu-Manber
// scan kernels: inline PTX for mbarriers and 1-D TMA bulk copies
// (cp.async.bulk), acquire/release global accesses, a bounded spin, warp
// scans and the per-pattern counters.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pm {
namespace dev {

constexpr uint32_t kFull = 0xFFFFFFFFu;
// ~1-4 s at GB300 clocks: a wait that long means something is wrong
constexpr long long kSpinLimit = 4000000000LL;

// status word codes in the workspace header
constexpr uint32_t kErrTimeoutTma = 1;
constexpr uint32_t kErrTimeoutWait = 2;       // reserved: a bounded wait on another CTA gave up
constexpr uint32_t kErrInternal = 3;        // a consistency check failed

struct WsHeader {           // lives at the start of the workspace
    uint32_t status;        // 0 = ok, else kErr*
    uint32_t done_ctas;     // CTAs that finished (the last one finalises counts)
    uint32_t done_expand;   // expand CTAs that finished (late ids: the last one finalises counts)
    uint32_t pad0;
    unsigned long long queue;  // batched scan: next instance to take
    unsigned long long pad1[29];
};
static_assert(sizeof(WsHeader) <= kWsHeader, "workspace header too large");

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` to complete; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kSpinLimit) return false;
    }
    return true;
}

// 1-D bulk copy global -> this CTA's shared memory, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Look-back statuses carry their own "published" flag bits and every reader
// spins until those bits are set, so no other data is ordered behind them:
// relaxed (volatile) accesses suffice and avoid a memory barrier per tile.
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void set_status(WsHeader *h, uint32_t code)
{
    atomicCAS(&h->status, 0u, code);
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ void count_pattern(uint32_t r, uint32_t *s_hist, long long *g_counts)
{
    if (s_hist) atomicAdd(&s_hist[r], 1u);
    else atomicAdd(reinterpret_cast<unsigned long long *>(g_counts) + r, 1ull);
}

}  // namespace dev
}  // namespace pm
