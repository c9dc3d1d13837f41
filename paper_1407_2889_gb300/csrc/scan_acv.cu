// scan_acv.cu -- Aho-Corasick scan of a pattern set whose patterns have
// their own lengths (the Section 1 definition with each pattern's length in
// place of m) on sm_103a.
//
// The DFA walk is the one of the fixed-length scan (Section 3.1, Algorithm
// 3 in its merged-table form; warp tiles staged by TMA, lane l walking the
// 80 start positions it owns plus a halo of the longest length - 1), but a
// match entry now names a state whose output set (Algorithm 2: its own
// patterns plus its supply's) can hold several patterns of different
// lengths, each starting at its own position. A lane keeps the (start, r)
// pairs whose start it owns, writes them to the tile's slot in the order
// their ends were met, and the expand kernel below puts each lane's pairs in
// (start, r) order while it writes the keys: lanes own consecutive start
// ranges, so the tile's keys are then sorted.
#include <type_traits>

#include "ac_device.cuh"

namespace pm {
namespace {

using dev::kFull;
using acdev::TableRef;
using acdev::walk_dna;
using acdev::walk_gen;
using acdev::walk_slow;

struct AcvArgs {
    const uint8_t *text;
    long long n;
    int aligned;
    const void *table_g;
    int smem_entries;
    const uint32_t *omask_g;      // one bit per row: the row's output set is not empty
    const uint32_t *orank_g;      // set bits before each word
    int nwords;
    int omask_smem;               // bitmap and ranks copied to shared memory
    const uint32_t *out_off;      // CSR of the output rows, rank order
    const uint32_t *out_ent;      // (r << 7) | len, longer first
    const uint8_t *cls_g;
    int m, lw;                    // m: longest pattern length
    uint32_t lut;
    uint32_t pad;
    long long nsub;
    int pool_cap;
    int list, hist_smem, d;
    long long *counts;
    long long *n_occ;
    dev::WsHeader *ws;
    uint32_t *tile_ent;           // list: entries (= keys) per warp tile
    uint32_t *tile_out;
    unsigned long long *seg_sum;
    long long seg_tiles;
    void *slots;                  // list: slot_stride entries per warp tile
    long long slot_stride;
    int se4;                      // 4-byte entries (start << 20 | r), else 8 (start << 32 | r)
};

__host__ __device__ constexpr long long r16v(long long x) { return (x + 15) & ~15LL; }

__host__ __device__ inline long long acv_warp_bytes(int hv, int pool_cap, int eb)
{
    // barrier | text buffer | pool (pool_cap + 1 slots per lane)
    return 16 + r16v(kWarpTile + 16 * hv) + r16v((long long)(pool_cap + 1) * 32 * eb);
}

__device__ __forceinline__ int acv_stage_bytes(const AcvArgs &a, long long t, int buf)
{
    if (!a.aligned) return 0;
    const long long avail = (a.n & ~15LL) - t * kWarpTile;
    if (avail <= 0) return 0;
    return avail >= buf ? buf : int(avail);
}

__device__ __forceinline__ void acv_stage_issue(const AcvArgs &a, long long t, uint8_t *buf,
                                                uint64_t *bar, int bufsz)
{
    const int bytes = acv_stage_bytes(a, t, bufsz);
    dev::mbar_arrive_expect_tx(bar, uint32_t(bytes));
    if (bytes > 0) dev::tma_load_1d(buf, a.text + t * kWarpTile, uint32_t(bytes), bar);
}

// launch bound 768 threads (up to 85 registers): whole-table plans run up
// to 24 warps, which measured 13 % faster than 16 on a 1,000-pattern set,
// and 16 warps lose nothing against a 512-thread build
template <typename E, int NV, int HV, bool DNA, bool PRE, bool HYB>
__global__ void __launch_bounds__(768, 1) acv_scan_kernel(const AcvArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int BUF = kWarpTile + 16 * HV;
    constexpr int HW = (NV * 16 + 31) / 32;

    // ---- shared memory carve-up (mirrors acv_smem_bytes on the host) ------
    unsigned char *p = smem;
    E *s_tab = reinterpret_cast<E *>(p);
    p += r16v((long long)a.smem_entries * sizeof(E));
    uint32_t *s_mask = a.omask_smem ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += a.omask_smem ? r16v((long long)a.nwords * 4) : 0;
    uint32_t *s_rank = a.omask_smem ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += a.omask_smem ? r16v((long long)(a.nwords + 1) * 4) : 0;
    uint32_t *s_hist = a.hist_smem ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += a.hist_smem ? r16v((long long)a.d * 4) : 0;
    uint8_t *s_cls = p;
    p += DNA ? 0 : 256;
    p += warp * acv_warp_bytes(HV, a.pool_cap, sizeof(E));
    uint64_t *bar = reinterpret_cast<uint64_t *>(p);
    uint8_t *buf = p + 16;
    E *pool = reinterpret_cast<E *>(buf + r16v(BUF));

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.table_g);
        uint4 *dst = reinterpret_cast<uint4 *>(s_tab);
        const int nvec = int(((long long)a.smem_entries * sizeof(E) + 15) / 16);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = src[i];
    }
    if (a.omask_smem) {
        for (int i = threadIdx.x; i < a.nwords; i += blockDim.x) s_mask[i] = a.omask_g[i];
        for (int i = threadIdx.x; i <= a.nwords; i += blockDim.x) s_rank[i] = a.orank_g[i];
    }
    const uint32_t *omask = a.omask_smem ? s_mask : a.omask_g;
    const uint32_t *orank = a.omask_smem ? s_rank : a.orank_g;
    if (s_hist)
        for (int i = threadIdx.x; i < a.d; i += blockDim.x) s_hist[i] = 0u;
    if (!DNA)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) s_cls[i] = a.cls_g[i];
    if (lane == 0) dev::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dev::fence_proxy_async_smem();
    __syncthreads();

    const TableRef<E, HYB> tab{s_tab, reinterpret_cast<const E *>(a.table_g), uint32_t(a.smem_entries)};
    E *pl = pool + lane;
    const uint32_t cap = uint32_t(a.pool_cap);
    const int m = a.m;
    const long long G = (long long)gridDim.x * (blockDim.x >> 5);
    const long long gwarp = (long long)blockIdx.x * (blockDim.x >> 5) + warp;

    // output set of the row an entry leads to: [first, end) of out_ent
    auto outputs = [&](uint32_t e, uint32_t &first, uint32_t &end) {
        const uint32_t row = PRE ? (e >> 2) : (e >> 1);
        const uint32_t w = row >> 5;
        const uint32_t rk = orank[w] + __popc(omask[w] & ((1u << (row & 31u)) - 1u));
        first = __ldg(a.out_off + rk);
        end = __ldg(a.out_off + rk + 1);
    };
    // every pattern of the output set that starts in this lane's chunk, in
    // the set's order (longer first, so starts ascend); f(start, r)
    auto each_start = [&](int step, uint32_t e, auto &&f) {
        uint32_t k, k1;
        outputs(e, k, k1);
        for (; k < k1; ++k) {
            const uint32_t v = __ldg(a.out_ent + k);
            const int s = step - int(v & 127u) + 1;
            if (s >= kChunk) break;   // shorter patterns start even later
            if (s >= 0) f(s, v >> 7);
        }
    };

    uint32_t phase = 0;
    bool inflight = false;
    unsigned long long my_total = 0;
    if (gwarp < a.nsub) {
        if (lane == 0) acv_stage_issue(a, gwarp, buf, bar, BUF);
        inflight = true;
    }

    for (long long st = gwarp; st < a.nsub; st += G) {
        const bool got = __all_sync(kFull, dev::mbar_wait_bounded(bar, phase));
        if (!got) {
            if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutTma);
            break;  // the copy stays in flight: waited for below
        }
        inflight = false;
        phase ^= 1u;
        const long long tile0 = st * kWarpTile;
        const int got_bytes = acv_stage_bytes(a, st, BUF);
        if (got_bytes < BUF) {  // tail of the text, or an unaligned text
            for (int b = got_bytes + lane; b < BUF; b += 32) {
                const long long g = tile0 + b;
                buf[b] = g < a.n ? a.text[g] : uint8_t(a.pad);
            }
            __syncwarp();
        }
        uint4 tv[NV];
        {
            const uint4 *bv = reinterpret_cast<const uint4 *>(buf + lane * kChunk);
#pragma unroll
            for (int v = 0; v < NV; ++v) tv[v] = bv[v];
        }
        dev::fence_proxy_async_smem();
        __syncwarp();
        if (st + G < a.nsub) {
            if (lane == 0) acv_stage_issue(a, st + G, buf, bar, BUF);
            inflight = true;
        }

        // ---- walk: the entry of every step whose state has outputs -------
        const long long g0 = tile0 + (long long)lane * kChunk;
        int steps = kChunk + m - 1;
        if (!DNA) {
            const long long left = a.n - g0;
            steps = left <= 0 ? 0 : (left < steps ? int(left) : steps);
        }
        uint32_t hw[HW];
#pragma unroll
        for (int j = 0; j < HW; ++j) hw[j] = 0u;
        uint32_t kslot = 0;
        auto rec = [&](int step, uint32_t, uint32_t e) {
            const uint32_t h = e & 1u;
            pl[kslot * 32] = E(e);
            kslot = min(kslot + h, cap);
            hw[step >> 5] += h << (step & 31);
        };
        if (DNA) walk_dna<NV, PRE>(tv, steps, a.lut, tab, rec);
        else walk_gen<NV>(tv, steps, a.lw, s_cls, tab, rec);
        uint32_t nh = 0;
#pragma unroll
        for (int j = 0; j < HW; ++j) nh += __popc(hw[j]);
        const bool ovf = nh > cap;

        // the lane's matches in end order: f(step, entry)
        auto each_hit = [&](auto &&f) {
            if (!ovf) {
                uint32_t k = 0;
#pragma unroll
                for (int j = 0; j < HW; ++j) {
                    uint32_t wj = hw[j];
                    while (wj) {
                        const int b = __ffs(int(wj)) - 1;
                        wj &= wj - 1u;
                        f(j * 32 + b, uint32_t(pl[k * 32]));
                        ++k;
                    }
                }
            } else {
                walk_slow<PRE>(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab,
                               [&](int step, uint32_t idx) { f(step, tab(idx)); });
            }
        };

        // pass 1: count (per-pattern counters and the lane's total)
        uint32_t cnt = 0;
        each_hit([&](int step, uint32_t e) {
            each_start(step, e, [&](int, uint32_t r) {
                dev::count_pattern(r, s_hist, a.counts);
                ++cnt;
            });
        });
        if (!a.list) {
            my_total += cnt;
            continue;
        }
        // pass 2: the lane's (start, r) pairs to the tile's slot
        const uint32_t o_incl = dev::warp_incl_scan(cnt, lane);
        const uint32_t o_tot = __shfl_sync(kFull, o_incl, 31);
        if ((long long)o_tot > a.slot_stride) {
            // more pairs than max_starts allows: a compiler bug, never written past the slot
            if (lane == 0) {
                dev::set_status(a.ws, dev::kErrInternal);
                a.tile_ent[st] = 0u;
                a.tile_out[st] = 0u;
            }
            continue;
        }
        const long long first = st * a.slot_stride + (o_incl - cnt);
        const uint32_t cs = uint32_t(lane * kChunk);
        uint32_t k = 0;
        each_hit([&](int step, uint32_t e) {
            each_start(step, e, [&](int s, uint32_t r) {
                if (k < cnt) {
                    if (a.se4)
                        static_cast<uint32_t *>(a.slots)[first + k] = ((cs + uint32_t(s)) << 20) | r;
                    else
                        static_cast<unsigned long long *>(a.slots)[first + k] =
                            ((unsigned long long)(cs + uint32_t(s)) << 32) | r;
                }
                ++k;
            });
        });
        if (lane == 31) {
            a.tile_ent[st] = o_tot;
            a.tile_out[st] = o_tot;
            if (o_tot) atomicAdd(&a.seg_sum[st / a.seg_tiles], (unsigned long long)o_tot);
        }
    }

    // a copy still in flight after an error exit: wait for it (bounded)
    if (inflight) (void)dev::mbar_wait_bounded(bar, phase);

    if (!a.list) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_total += __shfl_down_sync(kFull, my_total, o);
        if (lane == 0 && my_total) atomicAdd(reinterpret_cast<unsigned long long *>(a.n_occ), my_total);
    }
    __syncthreads();
    if (s_hist) {
        for (int r = threadIdx.x; r < a.d; r += blockDim.x) {
            const uint32_t c = s_hist[r];
            if (c) atomicAdd(reinterpret_cast<unsigned long long *>(a.counts) + r, (unsigned long long)c);
        }
    }
}

// ---------------------------------------------------------------------------
// List mode, step 2: a tile's entries (lane runs in lane order, each run in
// end order) become sorted keys. CTA b owns the tiles of segment b (base and
// per-tile offsets as in the fixed-length expand); a warp stages a tile of
// up to kSortCap entries in shared memory, each lane sorts its own run
// (entries whose start lies in its 80 positions) by (start, r), and the warp
// writes the keys in coalesced rows. Larger tiles are sorted in place in the
// slot.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortCap = 1024;

template <typename SE, int kShift>
__global__ void __launch_bounds__(kSortThreads)
acv_expand_kernel(SE *__restrict__ slots, long long slot_stride, const uint32_t *__restrict__ tile_ent,
                  const unsigned long long *__restrict__ seg_sum, long long seg_tiles, long long nsub,
                  unsigned long long *__restrict__ occ, long long occ_cap, long long *n_occ)
{
    extern __shared__ __align__(16) unsigned char esm[];
    constexpr int NW = kSortThreads / 32;
    SE *s_buf = reinterpret_cast<SE *>(esm);                                        // NW x kSortCap
    unsigned long long *s_off = reinterpret_cast<unsigned long long *>(s_buf + NW * kSortCap);  // seg_tiles
    __shared__ unsigned long long s_red[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long t0 = (long long)blockIdx.x * seg_tiles;
    const long long nt = min(seg_tiles, nsub - t0);
    if (nt <= 0) return;

    unsigned long long part = 0;
    for (long long q = tid; q < blockIdx.x; q += kSortThreads) part += seg_sum[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    unsigned long long seg_base = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) seg_base += s_red[w];
    __syncthreads();

    const long long per = (nt + kSortThreads - 1) / kSortThreads;
    const long long r0 = min(nt, (long long)tid * per), r1 = min(nt, r0 + per);
    unsigned long long mine = 0;
    for (long long q = r0; q < r1; ++q) {
        const uint32_t o = tile_ent[t0 + q];
        s_off[q] = o;
        mine += o;
    }
    unsigned long long inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) s_red[warp] = inc;
    __syncthreads();
    unsigned long long run = seg_base + inc - mine;
    for (int w = 0; w < warp; ++w) run += s_red[w];
    for (long long q = r0; q < r1; ++q) {
        const unsigned long long o = s_off[q];
        s_off[q] = run;
        run += o;
    }
    if (tid == kSortThreads - 1 && t0 + nt == nsub) *n_occ = (long long)run;
    __syncthreads();

    const unsigned long long cap = (unsigned long long)occ_cap;
    constexpr SE kMask = (SE(1) << kShift) - 1;
    SE *sb = s_buf + warp * kSortCap;
    for (long long q = warp; q < nt; q += NW) {
        const long long st = t0 + q;
        const uint32_t ent = tile_ent[st];
        if (ent == 0) continue;
        const unsigned long long base = s_off[q];
        const unsigned long long tile0 = (unsigned long long)st * kWarpTile;
        SE *src = slots + st * slot_stride;
        SE *v = ent <= uint32_t(kSortCap) ? sb : src;   // sort in shared memory, else in place
        if (v == sb) {
            for (uint32_t j = lane; j < ent; j += 32) sb[j] = src[j];
            __syncwarp();
        }
        // this lane's run: the entries whose start lies in [80 l, 80 l + 80)
        auto first_of = [&](uint32_t l) {
            uint32_t lo = 0, hi = ent;
            while (lo < hi) {
                const uint32_t md = (lo + hi) >> 1;
                if (uint32_t(v[md] >> kShift) / uint32_t(kChunk) < l) lo = md + 1;
                else hi = md;
            }
            return lo;
        };
        const uint32_t b0 = first_of(uint32_t(lane)), b1 = first_of(uint32_t(lane) + 1);
        for (uint32_t x = b0 + 1; x < b1; ++x) {  // insertion sort: runs are short
            const SE key = v[x];
            uint32_t y = x;
            while (y > b0 && v[y - 1] > key) {
                v[y] = v[y - 1];
                --y;
            }
            v[y] = key;
        }
        __syncwarp();
        for (uint32_t j = lane; j < ent; j += 32) {
            const SE e = v[j];
            const unsigned long long gi = base + j;
            if (gi < cap) occ[gi] = ((tile0 + (unsigned long long)(e >> kShift)) << 32) | (unsigned long long)(e & kMask);
        }
        __syncwarp();
    }
}

typedef void (*AcvKernel)(const AcvArgs);

struct AcvVariant {
    AcvKernel fn;
    int eb, hv;
    bool dna, pre;
};

// dna u16 index entries (0-2), dna u32 index entries (3-5), general u32
// (6-8), all with a table prefix in shared memory and the rest in device
// memory; dna u16 index entries with the whole table in shared memory
// (9-11); within each group HV = 1, 2, 4
const AcvVariant kAcvVariants[] = {
    {acv_scan_kernel<uint16_t, 6, 1, true, true, true>, 2, 1, true, true},
    {acv_scan_kernel<uint16_t, 7, 2, true, true, true>, 2, 2, true, true},
    {acv_scan_kernel<uint16_t, 9, 4, true, true, true>, 2, 4, true, true},
    {acv_scan_kernel<uint32_t, 6, 1, true, true, true>, 4, 1, true, true},
    {acv_scan_kernel<uint32_t, 7, 2, true, true, true>, 4, 2, true, true},
    {acv_scan_kernel<uint32_t, 9, 4, true, true, true>, 4, 4, true, true},
    {acv_scan_kernel<uint32_t, 6, 1, false, false, true>, 4, 1, false, false},
    {acv_scan_kernel<uint32_t, 7, 2, false, false, true>, 4, 2, false, false},
    {acv_scan_kernel<uint32_t, 9, 4, false, false, true>, 4, 4, false, false},
    {acv_scan_kernel<uint16_t, 6, 1, true, true, false>, 2, 1, true, true},
    {acv_scan_kernel<uint16_t, 7, 2, true, true, false>, 2, 2, true, true},
    {acv_scan_kernel<uint16_t, 9, 4, true, true, false>, 2, 4, true, true},
};

int acv_hv(int m) { return m - 1 <= 16 ? 1 : m - 1 <= 32 ? 2 : m - 1 <= 64 ? 4 : -1; }

long long acv_smem_bytes(const AcvTables &v, int eb, long long smem_entries, int warps, bool hist, int hv,
                         int pool_cap, bool omask_smem)
{
    const long long nwords = ((long long)v.ac.n_rows + 31) / 32;
    return r16v(smem_entries * eb) + (omask_smem ? r16v(nwords * 4) + r16v((nwords + 1) * 4) : 0) +
           (hist ? r16v((long long)v.ac.d * 4) : 0) + (v.ac.dna ? 0 : 256) +
           (long long)warps * acv_warp_bytes(hv, pool_cap, eb);
}

}  // namespace

// entry bytes of the device table: u16 index entries for ACGT sets of at
// most 2^14 rows, else u32 (index entries for ACGT sets)
static int acv_entry_bytes(const AcvTables &v) { return v.ac.dna && v.ac.n_rows <= (1 << 14) ? 2 : 4; }

int acv_plan(const AcvTables &v, const pm_params &opt, const DeviceProps &dp, DevAcv &dev)
{
    const int hv = acv_hv(v.ac.m);
    if (hv < 0) return PM_ETOOBIG;
    const int eb = acv_entry_bytes(v);
    const long long entries = (long long)v.ac.n_rows << v.ac.lw;
    const long long budget = (long long)dp.smem_optin - 1024;
    const int pool_cap = 40;
    const int forced = opt.warps_per_cta > 0 ? std::min(opt.warps_per_cta, 24) : 0;
    // the output-row bitmap and its ranks: shared memory up to 48 KB
    const long long nwords = ((long long)v.ac.n_rows + 31) / 32;
    const bool osm = (2 * nwords + 1) * 4 <= (48 << 10);
    bool ok = false;
    for (int pass = 0; pass < 4 && !ok; ++pass) {
        // whole table with counters, whole table, prefix with counters, prefix
        const bool hist = pass == 0 || pass == 2;
        const bool whole = pass < 2;
        // whole tables up to 24 warps; a table prefix keeps the room (16)
        for (int w = forced ? forced : (whole ? 24 : 16); w >= (forced ? forced : 8) && !ok; w -= 4) {
            const long long fixed = acv_smem_bytes(v, eb, 0, w, hist, hv, pool_cap, osm);
            if (fixed > budget) continue;
            long long se = whole ? entries : ((budget - fixed) / eb) & ~((long long)(16 / eb) - 1);
            if (se > entries) se = entries;
            if (whole && acv_smem_bytes(v, eb, se, w, hist, hv, pool_cap, osm) > budget) continue;
            if (opt.placement == PM_PLACE_GLOBAL) se = 0;
            dev.warps = w;
            dev.hist_smem = hist ? 1 : 0;
            dev.smem_entries = se;
            dev.placement = se == entries ? PM_PLACE_SMEM : (se == 0 ? PM_PLACE_GLOBAL : PM_PLACE_HYBRID);
            dev.smem_bytes = acv_smem_bytes(v, eb, se, w, hist, hv, pool_cap, osm);
            dev.omask_smem = osm ? 1 : 0;
            ok = true;
        }
    }
    if (!ok) return PM_ETOOBIG;
    dev.pool_cap = pool_cap;
    dev.hv = hv;
    dev.entry_bytes = eb;
    dev.pre = v.ac.dna ? 1 : 0;
    const bool whole_u16 = v.ac.dna && eb == 2 && dev.placement == PM_PLACE_SMEM;
    dev.variant = (whole_u16 ? 9 : v.ac.dna ? (eb == 2 ? 0 : 3) : 6) + (hv == 1 ? 0 : hv == 2 ? 1 : 2);
    return PM_OK;
}

// slots: 4-byte entries (start << 20 | r) when every id fits 20 bits, else 8
static int acv_slot_bytes(const AcvTables &v) { return v.ac.d <= (1 << 20) ? 4 : 8; }

int64_t acv_workspace_bytes(const AcvTables &v, int64_t n, bool list)
{
    return list_workspace_bytes(warp_tiles(n), list, 0, acv_slot_bytes(v) * v.K);
}

int acv_launch(const AcvTables &v, const DevAcv &dv, const uint8_t *d_text, int64_t n, bool list,
               int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
               void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long nsub = warp_tiles(n);
    const int se = acv_slot_bytes(v);
    ListParts L;
    list_workspace_parts(d_ws, nsub, 0, se * v.K, L);
    cudaError_t e = cudaMemsetAsync(d_counts, 0, size_t(v.ac.d) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_n_occ, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ws, 0, size_t(list ? L.zeroed_bytes : kWsHeader), st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (n < v.m_min || nsub == 0) return PM_OK;

    const AcvKernel fn = kAcvVariants[dv.variant].fn;
    int rc = kernel_smem_attr(reinterpret_cast<const void *>(fn), dv.smem_bytes);
    if (rc) return rc;
    DeviceProps dp;
    rc = device_props(dp);
    if (rc) return rc;
    AcvArgs a;
    a.text = d_text;
    a.n = n;
    a.aligned = (reinterpret_cast<uintptr_t>(d_text) & 15) == 0;
    a.table_g = dv.table;
    a.smem_entries = int(dv.smem_entries);
    a.omask_g = dv.omask;
    a.orank_g = dv.orank;
    a.nwords = int((v.ac.n_rows + 31) / 32);
    a.omask_smem = dv.omask_smem;
    a.out_off = dv.out_off;
    a.out_ent = dv.out_ent;
    a.cls_g = dv.cls;
    a.m = v.ac.m;
    a.lw = v.ac.lw;
    a.lut = v.ac.lut;
    {
        // a byte outside the alphabet (sends the walk to the reset row)
        uint32_t pad = 0;
        while (pad < 255 && v.ac.cls[pad] != 0xFF) ++pad;
        a.pad = pad;
    }
    a.nsub = nsub;
    a.pool_cap = dv.pool_cap;
    a.list = list ? 1 : 0;
    a.hist_smem = dv.hist_smem;
    a.d = int(v.ac.d);
    a.counts = reinterpret_cast<long long *>(d_counts);
    a.n_occ = reinterpret_cast<long long *>(d_n_occ);
    a.ws = reinterpret_cast<dev::WsHeader *>(d_ws);
    a.tile_ent = L.tile_ent;
    a.tile_out = L.tile_out;
    a.seg_sum = L.seg_sum;
    a.seg_tiles = L.seg_tiles;
    a.slots = L.slots;
    a.slot_stride = (long long)kWarpTile * v.K;
    a.se4 = se == 4 ? 1 : 0;

    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, dv.warps * 32, size_t(dv.smem_bytes));
    if (e != cudaSuccess || per_sm < 1) { set_cuda_error(int(e)); return PM_ECUDA; }
    long long grid = (long long)dp.sm_count;
    const long long want = (nsub + dv.warps - 1) / dv.warps;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    fn<<<dim3(unsigned(grid)), dim3(unsigned(dv.warps * 32)), size_t(dv.smem_bytes), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (!list) return PM_OK;

    return sorted_expand_launch(d_ws, nsub, se, v.K, d_occ, occ_cap, d_n_occ, stream);
}

int sorted_expand_launch(void *d_ws, int64_t nsub, int slot_bytes, int per_pos, uint64_t *d_occ,
                         int64_t occ_cap, int64_t *d_n_occ, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ListParts L;
    list_workspace_parts(d_ws, nsub, 0, slot_bytes * per_pos, L);
    const long long stride = (long long)kWarpTile * per_pos;
    const long long seg_tiles = L.seg_tiles;
    const long long nseg = (nsub + seg_tiles - 1) / seg_tiles;
    const size_t esmem = size_t((kSortThreads / 32) * kSortCap * slot_bytes + seg_tiles * 8);
    unsigned long long *occ = reinterpret_cast<unsigned long long *>(d_occ);
    long long *n_occ = reinterpret_cast<long long *>(d_n_occ);
    const long long cap = d_occ ? occ_cap : 0;
    const void *fn = slot_bytes == 4 ? reinterpret_cast<const void *>(acv_expand_kernel<uint32_t, 20>)
                                     : reinterpret_cast<const void *>(acv_expand_kernel<unsigned long long, 32>);
    const int rc = kernel_smem_attr(fn, int64_t(esmem));
    if (rc) return rc;
    if (slot_bytes == 4)
        acv_expand_kernel<uint32_t, 20><<<unsigned(nseg), kSortThreads, esmem, st>>>(
            static_cast<uint32_t *>(L.slots), stride, L.tile_ent, L.seg_sum, seg_tiles, nsub, occ, cap, n_occ);
    else
        acv_expand_kernel<unsigned long long, 32><<<unsigned(nseg), kSortThreads, esmem, st>>>(
            static_cast<unsigned long long *>(L.slots), stride, L.tile_ent, L.seg_sum, seg_tiles, nsub, occ, cap,
            n_occ);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    return PM_OK;
}

}  // namespace pm
