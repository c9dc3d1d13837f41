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

// status word codes in the workspace header
constexpr uint32_t kErrTimeoutTma = 1;
constexpr uint32_t kErrTimeoutLookback = 2;
constexpr uint32_t kErrInternal = 3;        // a consistency check failed

struct WsHeader {           // lives at the start of the workspace
    uint32_t status;        // 0 = ok, else kErr*
    uint32_t done_ctas;     // CTAs that finished (the last one finalises counts)
    unsigned long long queue;  // batched scan: next instance to take
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

// Two-level decoupled look-back over warp tiles (all 32 lanes call it).
//
// Warp tiles are grouped into super-tiles of super_tiles consecutive tiles.
// A tile publishes its aggregate (count of outputs) in its own status word
// and adds (1 << 56) | aggregate to its super-tile's word with one atomic, so
// a super-tile's sum is final once its arrival count (the top byte) reaches
// its number of tiles. A tile's exclusive prefix is (sum of all earlier
// super-tiles) + (sum of the earlier tiles of its own super-tile); earlier
// super-tiles are summed back to the nearest one with a published inclusive
// prefix, 64 per L2 round trip, and the result is published as the previous
// super-tile's inclusive prefix. A one-level look-back over tiles would
// advance the known prefixes by only one window of tiles per round trip,
// which bounds throughput at (window x tile bytes) / latency; super-tiles
// lift that bound by the super-tile size. Nothing here waits in the publish
// step; the prefix step waits (bounded) only on tiles and super-tiles that
// precede the tile, all of them claimed by resident warps.
struct LookbackRefs {
    unsigned long long *tile_st;   // per tile: 0 or kStAgg | count
    unsigned long long *super_acc; // per super-tile: (arrivals << 56) | running sum
    unsigned long long *super_pre; // per super-tile: 0 or kStPre | inclusive prefix
    long long ntiles;
    int super_tiles;               // tiles per super-tile (<= 64; divides the round size)
};

// Largest divisor of the round size (warps in the grid) not above 64: a
// super-tile then never spans two rounds of the static schedule, so
// completing it never waits for a later round.
__host__ __device__ inline int super_size_for(long long round)
{
    for (int k = 64; k > 1; --k)
        if (round % k == 0) return k;
    return 1;
}

constexpr unsigned long long kStAgg = 1ull << 62, kStPre = 2ull << 62;
constexpr unsigned long long kStVal = (1ull << 62) - 1;
constexpr unsigned long long kAccOne = 1ull << 56, kAccVal = kAccOne - 1;

// sum over lanes of the values of two statuses per lane, waiting (bounded)
// until every status selected by the masks is published
__device__ __forceinline__ bool wait_sum2(const unsigned long long *p, long long lo_idx,
                                          uint32_t need_lo, uint32_t need_hi, int lane,
                                          unsigned long long &sum)
{
    const long long t0 = clock64();
    while (true) {
        const bool want_lo = (need_lo >> lane) & 1u, want_hi = (need_hi >> lane) & 1u;
        const unsigned long long vl = want_lo ? ld_relaxed(p + lo_idx + lane) : kStAgg;
        const unsigned long long vh = want_hi ? ld_relaxed(p + lo_idx + 32 + lane) : kStAgg;
        if (__all_sync(kFull, (vl & ~kStVal) != 0 && (vh & ~kStVal) != 0)) {
            unsigned long long x = (vl & kStVal) + (vh & kStVal);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
            sum = x;
            return true;
        }
        if (clock64() - t0 > kSpinLimit) return false;
        __nanosleep(200);  // leave the issue slots to warps that have work
    }
}

__device__ __forceinline__ void tile_masks(int k, uint32_t &lo, uint32_t &hi)
{
    // the first k of 64 consecutive slots: lanes [0, min(k,32)) low, [0, k-32) high
    lo = k >= 32 ? kFull : (k <= 0 ? 0u : (kFull >> (32 - k)));
    hi = k <= 32 ? 0u : (kFull >> (64 - k));
}

// Publish step: never waits.
__device__ __forceinline__ void publish_tile(const LookbackRefs &L, long long t,
                                             unsigned long long agg, int lane)
{
    if (lane == 0) {
        st_relaxed(&L.tile_st[t], kStAgg | agg);
        atomicAdd(&L.super_acc[t / L.super_tiles], kAccOne | agg);
    }
}

__device__ __forceinline__ int tiles_in_super(const LookbackRefs &L, long long s)
{
    const long long left = L.ntiles - s * L.super_tiles;
    return left < L.super_tiles ? int(left) : L.super_tiles;
}

// Exclusive prefix of tile t (see above).
__device__ __forceinline__ unsigned long long tile_base(const LookbackRefs &L, long long t,
                                                        int lane, bool &ok)
{
    ok = true;
    const long long s = t / L.super_tiles;
    const int i = int(t - s * L.super_tiles);
    unsigned long long inpre = 0;
    if (i > 0) {
        uint32_t lo, hi;
        tile_masks(i, lo, hi);
        if (!wait_sum2(L.tile_st, s * L.super_tiles, lo, hi, lane, inpre)) { ok = false; return 0; }
    }
    if (s == 0) return inpre;
    unsigned long long excl = 0;
    long long base = s - 64;  // window: lane holds base+lane and base+32+lane
    long long t0 = clock64();
    while (true) {
        const long long jl = base + lane, jh = base + 32 + lane;
        // a super-tile's value: its inclusive prefix if published, else its
        // sum once every tile has arrived; `pre` marks the former
        unsigned long long vl = 0, vh = 0;
        bool pl_ = jl < 0, ph_ = jh < 0, rl_ = jl < 0, rh_ = jh < 0;
        if (jl >= 0) {
            const unsigned long long p = ld_relaxed(&L.super_pre[jl]);
            if (p & kStPre) { vl = p & kStVal; pl_ = rl_ = true; }
            else {
                const unsigned long long a = ld_relaxed(&L.super_acc[jl]);
                if (int(a >> 56) == tiles_in_super(L, jl)) { vl = a & kAccVal; rl_ = true; }
            }
        }
        if (jh >= 0) {
            const unsigned long long p = ld_relaxed(&L.super_pre[jh]);
            if (p & kStPre) { vh = p & kStVal; ph_ = rh_ = true; }
            else {
                const unsigned long long a = ld_relaxed(&L.super_acc[jh]);
                if (int(a >> 56) == tiles_in_super(L, jh)) { vh = a & kAccVal; rh_ = true; }
            }
        }
        const uint32_t rl = __ballot_sync(kFull, rl_), rh = __ballot_sync(kFull, rh_);
        const uint32_t pl = __ballot_sync(kFull, pl_), ph = __ballot_sync(kFull, ph_);
        uint32_t nl, nh;
        if (ph) { nh = kFull << (31 - __clz(ph)); nl = 0; }
        else if (pl) { nh = kFull; nl = kFull << (31 - __clz(pl)); }
        else { nh = kFull; nl = kFull; }
        if ((rl & nl) != nl || (rh & nh) != nh) {
            if (clock64() - t0 > kSpinLimit) { ok = false; return 0; }
            __nanosleep(200);
            continue;
        }
        unsigned long long x = (((nl >> lane) & 1u) ? vl : 0ull) + (((nh >> lane) & 1u) ? vh : 0ull);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        excl += x;
        if (ph | pl) break;
        base -= 64;
        t0 = clock64();
    }
    if (lane == 0) st_relaxed(&L.super_pre[s - 1], kStPre | excl);
    return excl + inpre;
}

// Both steps back to back (kernels that wait in place).
__device__ __forceinline__ unsigned long long lookback(const LookbackRefs &L, long long t,
                                                       unsigned long long agg, int lane, bool &ok)
{
    publish_tile(L, t, agg, lane);
    return tile_base(L, t, lane, ok);
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

// Static round-robin schedule: global warp g takes tiles g, g + G, g + 2G ...
// (G = warps in the grid). Every warp of the grid is resident at once (the
// grid is sized from the occupancy of one CTA per SM), and a tile waits only
// on tiles of earlier rounds, so the look-back cannot deadlock.
struct TileSchedule {
    long long cur, stride, ntiles;
    __device__ __forceinline__ void init(long long ntiles_)
    {
        ntiles = ntiles_;
        stride = (long long)gridDim.x * (blockDim.x >> 5);
        cur = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (cur >= ntiles) cur = -1;
    }
    __device__ __forceinline__ long long next_of(long long t) const
    {
        return t >= 0 && t + stride < ntiles ? t + stride : -1;
    }
};

__device__ __forceinline__ void count_pattern(uint32_t r, uint32_t *s_hist, long long *g_counts)
{
    if (s_hist) atomicAdd(&s_hist[r], 1u);
    else atomicAdd(reinterpret_cast<unsigned long long *>(g_counts) + r, 1ull);
}

}  // namespace dev
}  // namespace pm
