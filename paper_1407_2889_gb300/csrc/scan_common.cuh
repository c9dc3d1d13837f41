// scan_common.cuh -- device helpers shared by the Aho-Corasick and Wu-Manber
// scan kernels: inline PTX for mbarriers and 1-D TMA bulk copies
// (cp.async.bulk), acquire/release global accesses, a bounded spin, the
// warp-level decoupled look-back that turns per-tile match counts into
// output offsets, and the per-pattern counters.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pm {
namespace dev {

constexpr uint32_t kFull = 0xFFFFFFFFu;
// ~1-4 s at GB300 clocks: a wait that long means something is wrong
constexpr long long kSpinLimit = 4000000000LL;
constexpr int kClaimBatch = 1;   // warp tiles claimed per atomic (consecutive tiles
                                 // held by one warp would serialise the look-back)

// status word codes in the workspace header
constexpr uint32_t kErrTimeoutTma = 1;
constexpr uint32_t kErrTimeoutLookback = 2;
constexpr uint32_t kErrInternal = 3;        // a consistency check failed

struct WsHeader {           // lives at the start of the workspace
    uint32_t status;        // 0 = ok, else kErr*
    uint32_t pad0;
    unsigned long long tile_ctr;   // next claim batch
    unsigned long long pad1[30];
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

__device__ __forceinline__ void set_status(WsHeader *h, uint32_t code)
{
    atomicCAS(&h->status, 0u, code);
}

// Decoupled look-back over warp tiles (one thread). Publishes the tile's
// aggregate, sums predecessors until an inclusive prefix is found, then
// publishes its own inclusive prefix. Tiles are claimed in increasing order
// by running warps, so every predecessor is eventually published.
// Returns the exclusive prefix; sets `ok` false if the wait limit ran out.
__device__ __forceinline__ unsigned long long lookback(unsigned long long *status, long long t,
                                                       unsigned long long agg, bool &ok)
{
    constexpr unsigned long long kAgg = 1ull << 62, kPre = 2ull << 62;
    constexpr unsigned long long kVal = (1ull << 62) - 1;
    ok = true;
    if (t == 0) {
        st_release(&status[0], kPre | agg);
        return 0;
    }
    st_release(&status[t], kAgg | agg);
    unsigned long long excl = 0;
    long long j = t - 1;
    long long t0 = 0;
    bool timing = false;
    while (true) {
        const unsigned long long v = ld_acquire(&status[j]);
        const unsigned long long f = v & ~kVal;
        if (f == 0) {
            if (!timing) { t0 = clock64(); timing = true; }
            else if (clock64() - t0 > kSpinLimit) { ok = false; break; }
            continue;
        }
        excl += v & kVal;
        if (f == kPre) break;
        --j;
        timing = false;
    }
    st_release(&status[t], kPre | (excl + agg));
    return excl;
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

// Claims warp tiles in batches of kClaimBatch from the workspace counter.
struct TileCursor {
    long long t = 0, end = 0;
    __device__ __forceinline__ long long claim(WsHeader *h, int lane, long long ntiles)
    {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(&h->tile_ctr, 1ull);
        b = __shfl_sync(kFull, b, 0);
        t = (long long)b * kClaimBatch;
        end = t + kClaimBatch;
        if (end > ntiles) end = ntiles;
        return t < ntiles ? t : -1;
    }
    __device__ __forceinline__ long long next(WsHeader *h, int lane, long long ntiles)
    {
        ++t;
        if (t < end) return t;
        return claim(h, lane, ntiles);
    }
};

__device__ __forceinline__ void count_pattern(uint32_t r, uint32_t *s_hist, long long *g_counts)
{
    if (s_hist) atomicAdd(&s_hist[r], 1u);
    else atomicAdd(reinterpret_cast<unsigned long long *>(g_counts) + r, 1ull);
}

}  // namespace dev
}  // namespace pm
