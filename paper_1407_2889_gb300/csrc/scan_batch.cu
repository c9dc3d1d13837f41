// scan_batch.cu -- many independent Aho-Corasick scans in one persistent
// launch (thousands of (text, pattern set) instances of uneven sizes).
//
// A CTA takes whole instances from a queue, largest first (the host sorts
// the descriptors by text length, which bounds the tail at the largest
// instance). For each instance it loads the set's transition table (its
// breadth-first prefix when the table is larger than the CTA's table
// budget), the canonical-terminal lookup and zeroed per-terminal counters
// into shared memory once, then its warps walk the instance's warp tiles in
// rounds: warp w takes tiles w, w + W, w + 2W ... Within a round the offsets
// of the warps' outputs come from a prefix over per-warp totals in shared
// memory, so an instance never needs a look-back across CTAs, and its
// counts are final when the CTA leaves it. Walk, resolution of matches and
// staged coalesced output are the same code as the plain kernel
// (ac_device.cuh); the launch is a plain kernel plus memsets, so it can be
// captured in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "ac_device.cuh"

namespace pm {


namespace {

using dev::kFull;
using namespace acdev;

constexpr int kBatchHV = 4;                   // halo vectors: m <= 65
constexpr int kBatchNV = 5 + kBatchHV;
constexpr int kBatchBuf = kWarpTile + 16 * kBatchHV;
constexpr int kBatchPool = 40;                  // hit pool slots per lane, u16 entries
// the pool is kBatchPool + 1 u16 slots per lane; u32 instances get half as many
constexpr int kBatchPoolBytes = (kBatchPool + 1) * 32 * 2;
constexpr int kBatchStage = 128;              // u64 entries
constexpr int kBatchMaxM = 16 * kBatchHV + 1;

struct BatchArgs {
    const BatchDesc *desc;
    int k;
    const uint8_t *text;
    long long *counts;
    unsigned long long *occ;
    long long *n_occ;
    dev::WsHeader *ws;
    unsigned long long *ccount;
    unsigned long long *spill;     // key staging of split instances' parts
    int list;
    int region_bytes;              // per-CTA shared memory for table, ids and counters
};

__host__ __device__ constexpr long long rr16(long long x) { return (x + 15) & ~15LL; }

__host__ __device__ inline long long batch_warp_bytes()
{
    return 16 + rr16(kBatchBuf) + rr16(kBatchPoolBytes) + kBatchStage * 8;
}

__device__ __forceinline__ int bstage_bytes(const uint8_t *text, long long n, long long t)
{
    if (reinterpret_cast<uintptr_t>(text) & 15) return 0;
    const long long avail = (n & ~15LL) - t * kWarpTile;
    if (avail <= 0) return 0;
    return avail >= kBatchBuf ? kBatchBuf : int(avail);
}

__device__ __forceinline__ void bstage_issue(const uint8_t *text, long long n, long long t,
                                             uint8_t *buf, uint64_t *bar)
{
    const int bytes = bstage_bytes(text, n, t);
    dev::mbar_arrive_expect_tx(bar, uint32_t(bytes));
    if (bytes > 0) dev::tma_load_1d(buf, text + t * kWarpTile, uint32_t(bytes), bar);
}

struct CtaSmem {
    unsigned char *region;          // table prefix, ids and counters of the instance
    unsigned long long *s_tot;      // per-warp totals of a round
    uint64_t *bar;
    uint8_t *buf;
    unsigned char *pool;
    unsigned long long *stage;
};

// One instance, entry type E; HYB when the table is not wholly in shared
// memory. All threads of the CTA call it.
template <typename E, bool PRE, bool HYB>
__device__ void run_instance(const BatchArgs &a, const BatchDesc &D, const CtaSmem &S,
                             uint32_t &phase, bool &failed)
{
    constexpr int NV = kBatchNV;
    constexpr int HW = (16 * NV + 31) / 32;
    constexpr uint32_t kGrp = sizeof(E) == 2 ? 0x8000u : 0x80000000u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const uint8_t *text = a.text + D.text_off;
    const long long n = D.n;

    // ---- per-instance tables into shared memory --------------------------
    E *s_tab = reinterpret_cast<E *>(S.region);
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(D.table);
        uint4 *dst = reinterpret_cast<uint4 *>(s_tab);
        const int nvec = int(((long long)D.smem_entries * sizeof(E) + 15) / 16);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = src[i];
    }
    Ids<E> ids;
    if (D.ids_off >= 0) {
        unsigned char *ip = S.region + D.ids_off;
        uint32_t *mk = reinterpret_cast<uint32_t *>(ip);
        E *rk = reinterpret_cast<E *>(ip + rr16((long long)D.nwords * 4));
        E *cn = reinterpret_cast<E *>(reinterpret_cast<unsigned char *>(rk) +
                                      rr16((long long)(D.nwords + 1) * sizeof(E)));
        for (int i = threadIdx.x; i < D.nwords; i += blockDim.x) mk[i] = D.mask[i];
        for (int i = threadIdx.x; i <= D.nwords; i += blockDim.x) rk[i] = reinterpret_cast<const E *>(D.rank)[i];
        for (int i = threadIdx.x; i < D.nterms; i += blockDim.x) cn[i] = reinterpret_cast<const E *>(D.canon)[i];
        ids.mask = mk;
        ids.rank = rk;
        ids.canon = cn;
    } else {
        ids.mask = D.mask;
        ids.rank = reinterpret_cast<const E *>(D.rank);
        ids.canon = reinterpret_cast<const E *>(D.canon);
    }
    uint32_t *s_hist = D.hist_off >= 0 ? reinterpret_cast<uint32_t *>(S.region + D.hist_off) : nullptr;
    unsigned long long *g_hist = a.ccount + D.ccount_off;
    if (s_hist)
        for (int i = threadIdx.x; i < D.nterms; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();

    const TableRef<E, HYB> tab{s_tab, reinterpret_cast<const E *>(D.table), uint32_t(D.smem_entries)};
    E *pl = reinterpret_cast<E *>(S.pool) + lane;
    const uint32_t cap = kBatchPoolBytes / (32 * sizeof(E)) - 1;  // the last slot absorbs overflow
    const int m = D.m;
    const bool split = D.nparts > 1;
    auto count_terminal = [&](uint32_t c) {
        if (s_hist) atomicAdd(&s_hist[c], 1u);
        else atomicAdd(&g_hist[c], 1ull);
    };
    auto mult_of = [&](uint32_t code) -> uint32_t {
        if (!(code & kGrp)) return 1u;
        const uint32_t g = code & ~kGrp;
        return __ldg(D.grp_off + g + 1) - __ldg(D.grp_off + g);
    };
    // where `write` puts the keys: the instance's output, or a part's staging
    unsigned long long *odst = a.occ + D.occ_off;
    unsigned long long ocap = (unsigned long long)D.occ_cap;

    // One pass over the item's warp tiles [t_lo, t_hi): warps take tiles in
    // rounds of W; `count` bumps the per-terminal counters, `write` writes
    // the keys from output offset base0 on. Returns the item's outputs.
    auto pass = [&](bool count, bool write, unsigned long long base0) -> unsigned long long {
        long long t = D.t_lo + warp;
        bool inflight = false;
        if (t < D.t_hi) {
            if (lane == 0) bstage_issue(text, n, t, S.buf, S.bar);
            inflight = true;
        }
        unsigned long long running = base0;
        const long long rounds = (D.t_hi - D.t_lo + W - 1) / W;
        for (long long rd = 0; rd < rounds; ++rd, t += W) {
            const bool active = t < D.t_hi && !failed;
            uint32_t nh = 0, cnt = 0;
            bool ovf = false;
            uint32_t hw[HW];
#pragma unroll
            for (int j = 0; j < HW; ++j) hw[j] = 0u;
            long long g0 = 0;
            if (active) {
                const bool got = __all_sync(kFull, dev::mbar_wait_bounded(S.bar, phase));
                if (!got) {
                    if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutTma);
                    failed = true;  // the copy stays in flight: waited for below
                } else {
                    inflight = false;
                    phase ^= 1u;
                    const long long tile0 = t * kWarpTile;
                    const int got_bytes = bstage_bytes(text, n, t);
                    if (got_bytes < kBatchBuf) {
                        for (int b = got_bytes + lane; b < kBatchBuf; b += 32) {
                            const long long g = tile0 + b;
                            S.buf[b] = g < n ? text[g] : uint8_t(D.pad);
                        }
                        __syncwarp();
                    }
                    uint4 tv[NV];
                    {
                        const uint4 *bv = reinterpret_cast<const uint4 *>(S.buf + lane * kChunk);
#pragma unroll
                        for (int v = 0; v < NV; ++v) tv[v] = bv[v];
                    }
                    dev::fence_proxy_async_smem();
                    __syncwarp();
                    if (t + W < D.t_hi) {
                        if (lane == 0) bstage_issue(text, n, t + W, S.buf, S.bar);
                        inflight = true;
                    }
                    g0 = tile0 + (long long)lane * kChunk;
                    const int steps = kChunk + m - 1;
                    uint32_t kslot = 0;
                    auto rec = [&](int step, uint32_t idx, uint32_t e) {
                        const uint32_t h = e & 1u;
                        if (h) pl[kslot * 32] = E(idx - D.mid_base);
                        kslot = min(kslot + h, cap);
                        hw[step >> 5] |= h << (step & 31);
                    };
                    walk_dna<NV, PRE>(tv, steps, D.lut, tab, rec);
#pragma unroll
                    for (int j = 0; j < HW; ++j) nh += __popc(hw[j]);
                    ovf = nh > cap;
                    if (!ovf) {
                        for (uint32_t k = 0; k < nh; ++k) {
                            const uint32_t c = ids.terminal(pl[k * 32]);
                            const uint32_t code = ids.code(c);
                            if (count) count_terminal(c);
                            cnt += mult_of(code);
                            pl[k * 32] = E(code);
                        }
                    } else {
                        walk_slow<PRE>(text, n, g0, kChunk + m - 1, true, D.lut, 2, nullptr, tab,
                                       [&](int, uint32_t idx) {
                                           const uint32_t c = ids.terminal(idx - D.mid_base);
                                           if (count) count_terminal(c);
                                           cnt += mult_of(ids.code(c));
                                       });
                    }
                }
            }
            // ---- offsets of this round: prefix over the warps' totals ----------
            const uint32_t incl = dev::warp_incl_scan(cnt, lane);
            const uint32_t wtot = __shfl_sync(kFull, incl, 31);
            if (lane == 0) S.s_tot[warp] = wtot;
            __syncthreads();
            unsigned long long before = 0, all = 0;
            for (int w = 0; w < W; ++w) {
                const unsigned long long v = S.s_tot[w];
                if (w < warp) before += v;
                all += v;
            }
            const unsigned long long base = running + before;
            running += all;
            if (write && active && !failed && wtot > 0) {
                const uint32_t excl = incl - cnt;
                auto put = [&](unsigned long long oi, long long pos, uint32_t r) {
                    if (oi < ocap) odst[oi] = ((unsigned long long)pos << 32) | r;
                };
                if (!__any_sync(kFull, ovf)) {
                    StepBits<HW> it;
#pragma unroll
                    for (int j = 0; j < HW; ++j) it.w[j] = hw[j];
                    it.base = 0;
                    uint32_t k = 0, my = excl;
                    bool have = false, single = true;
                    uint32_t rs = 0, glo = 0, ghi = 0;
                    long long pos = 0;
                    for (uint32_t w0 = 0; w0 < wtot; w0 += kBatchStage) {
                        const uint32_t wend = min(w0 + (uint32_t)kBatchStage, wtot);
                        const uint32_t lim = min(wend, incl);
                        while (my < lim) {
                            if (!have) {
                                const int st = it.next();
                                if (st < 0) dev::set_status(a.ws, dev::kErrInternal);
                                pos = g0 + st - (m - 1);
                                const uint32_t code = pl[k * 32];
                                ++k;
                                single = !(code & kGrp);
                                if (single) {
                                    rs = code;
                                } else {
                                    const uint32_t g = code & ~kGrp;
                                    glo = __ldg(D.grp_off + g);
                                    ghi = __ldg(D.grp_off + g + 1);
                                }
                                have = true;
                            }
                            const uint32_t r = single ? rs : __ldg(D.grp_ids + glo);
                            S.stage[my - w0] = ((unsigned long long)pos << 32) | r;
                            ++my;
                            if (single || ++glo >= ghi) have = false;
                        }
                        __syncwarp();
                        for (uint32_t q = w0 + lane; q < wend; q += 32) {
                            const unsigned long long oi = base + q;
                            if (oi < ocap) odst[oi] = S.stage[q - w0];
                        }
                        __syncwarp();
                    }
                } else {
                    unsigned long long oi = base + excl;
                    auto put_code = [&](long long pos, uint32_t code) {
                        if (code & kGrp) {
                            const uint32_t g = code & ~kGrp;
                            const uint32_t hi = __ldg(D.grp_off + g + 1);
                            for (uint32_t j = __ldg(D.grp_off + g); j < hi; ++j) put(oi++, pos, __ldg(D.grp_ids + j));
                        } else {
                            put(oi++, pos, code);
                        }
                    };
                    if (!ovf) {
                        StepBits<HW> it;
#pragma unroll
                        for (int j = 0; j < HW; ++j) it.w[j] = hw[j];
                        it.base = 0;
                        for (uint32_t k = 0; k < nh; ++k) {
                            const int st = it.next();
                            if (st < 0) dev::set_status(a.ws, dev::kErrInternal);
                            put_code(g0 + st - (m - 1), pl[k * 32]);
                        }
                    } else {
                        walk_slow<PRE>(text, n, g0, kChunk + m - 1, true, D.lut, 2, nullptr, tab,
                                       [&](int step, uint32_t idx) {
                                           put_code(g0 + step - (m - 1), ids.code(ids.terminal(idx - D.mid_base)));
                                       });
                    }
                }
            }
            __syncthreads();  // s_tot is rewritten next round
        }
        if (inflight) {  // only after a failure: let the last copy land before reuse
            (void)dev::mbar_wait_bounded(S.bar, phase);
            phase ^= 1u;
        }
        return running - base0;
    };

    long long *cnt_out = a.counts + D.count_off;
    const E *cg = reinterpret_cast<const E *>(D.canon);
    // counts[r] of the instance from per-terminal counters (shared or device)
    auto write_counts = [&](bool from_device) {
        for (int c = threadIdx.x; c < D.nterms; c += blockDim.x) {
            const unsigned long long v = from_device ? dev::ld_acquire(&g_hist[c]) : (unsigned long long)s_hist[c];
            const uint32_t code = cg[c];
            if (code & kGrp) {
                const uint32_t g = code & ~kGrp;
                for (uint32_t j = D.grp_off[g]; j < D.grp_off[g + 1]; ++j) cnt_out[D.grp_ids[j]] = (long long)v;
            } else {
                cnt_out[code] = (long long)v;
            }
        }
    };

    if (!split) {
        const unsigned long long total = pass(true, a.list != 0, 0ull);
        if (threadIdx.x == 0) a.n_occ[D.out_slot] = (long long)total;
        write_counts(s_hist == nullptr);
        __syncthreads();
        return;
    }

    // ---- a part of a split instance ----------------------------------------
    __shared__ unsigned long long s_base;
    __shared__ int s_last;
    unsigned long long *pstat = a.ccount + D.pstat_off;  // (1 << 63) | part total
    const bool staged = a.list && D.spill_cap > 0;
    if (staged) {
        odst = a.spill + D.spill_off;
        ocap = (unsigned long long)D.spill_cap;
    }
    const unsigned long long total = pass(true, staged, 0ull);
    if (threadIdx.x == 0) {
        dev::st_relaxed(&pstat[D.part], (1ull << 63) | total);
        unsigned long long base = 0;
        if (a.list) {
            // the parts before this one were taken earlier by running CTAs,
            // and publish their totals without waiting for anything
            const long long t0c = clock64();
            for (int q = 0; q < D.part; ++q) {
                unsigned long long v = dev::ld_relaxed(&pstat[q]);
                while (!(v >> 63)) {
                    if (clock64() - t0c > dev::kSpinLimit) {
                        dev::set_status(a.ws, dev::kErrTimeoutWait);
                        break;
                    }
                    __nanosleep(128);
                    v = dev::ld_relaxed(&pstat[q]);
                }
                base += v & ~(1ull << 63);
            }
        }
        s_base = base;
    }
    __syncthreads();
    if (a.list) {
        odst = a.occ + D.occ_off;
        ocap = (unsigned long long)D.occ_cap;
        const unsigned long long b0 = s_base;
        if (staged && total <= (unsigned long long)D.spill_cap) {
            // this CTA's own stores, ordered by the barrier above
            const unsigned long long *sp = a.spill + D.spill_off;
            const unsigned long long nkeep = b0 < ocap ? min(total, ocap - b0) : 0ull;
            for (unsigned long long i = threadIdx.x; i < nkeep; i += blockDim.x) odst[b0 + i] = sp[i];
        } else if (b0 < ocap) {
            (void)pass(false, true, b0);
        }
    }
    // counters into the instance's device counters; the last part writes
    // the instance's counts and its total
    if (s_hist)
        for (int c = threadIdx.x; c < D.nterms; c += blockDim.x)
            if (s_hist[c]) atomicAdd(&g_hist[c], (unsigned long long)s_hist[c]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int *done = reinterpret_cast<unsigned int *>(a.ccount + D.done_off);
        s_last = atomicAdd(done, 1u) == unsigned(D.nparts - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        write_counts(true);
        if (threadIdx.x == 0) {
            unsigned long long all = 0;
            for (int q = 0; q < D.nparts; ++q) all += dev::ld_acquire(&pstat[q]) & ~(1ull << 63);
            a.n_occ[D.out_slot] = (long long)all;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(512, 1) ac_batch_kernel(const BatchArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    __shared__ int s_next;
    __shared__ unsigned long long s_tot[32];
    CtaSmem S;
    unsigned char *p = smem;
    S.region = p;
    p += a.region_bytes;
    p += warp * batch_warp_bytes();
    S.bar = reinterpret_cast<uint64_t *>(p);
    S.buf = p + 16;
    S.pool = S.buf + rr16(kBatchBuf);
    S.stage = reinterpret_cast<unsigned long long *>(S.pool + rr16(kBatchPoolBytes));
    S.s_tot = s_tot;
    (void)W;
    if (lane == 0) dev::mbar_init(S.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dev::fence_proxy_async_smem();
    __syncthreads();

    uint32_t phase = 0;
    bool failed = false;
    while (true) {
        if (threadIdx.x == 0) {
            const unsigned long long j = atomicAdd(&a.ws->queue, 1ull);
            s_next = j < (unsigned long long)a.k ? int(j) : -1;
        }
        __syncthreads();
        const int j = s_next;
        __syncthreads();
        if (j < 0) break;
        const BatchDesc D = a.desc[j];
        // u16 tables wholly in shared memory skip the bounds check of every
        // lookup; u32 tables are always partly in device memory
        if (D.eb == 2) {
            if (D.resident) {
                if (D.pre) run_instance<uint16_t, true, false>(a, D, S, phase, failed);
                else run_instance<uint16_t, false, false>(a, D, S, phase, failed);
            } else {
                if (D.pre) run_instance<uint16_t, true, true>(a, D, S, phase, failed);
                else run_instance<uint16_t, false, true>(a, D, S, phase, failed);
            }
        } else {
            if (D.pre) run_instance<uint32_t, true, true>(a, D, S, phase, failed);
            else run_instance<uint32_t, false, true>(a, D, S, phase, failed);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
constexpr int kBatchWarpChoices[] = {8, 12, 16};   // autotuner candidates
constexpr long long kSpillBytes = 32;               // text bytes per staged key of a part
constexpr int kBatchMaxWarps = 16;

struct InstLayout {
    int smem_entries, ids_off, hist_off;
};

// Where an instance's tables go inside the region. Everything when it fits;
// otherwise counters and ids stay in shared memory only while each takes at
// most a quarter of the region, and the table gets the rest (its
// breadth-first prefix: the rows a walk visits most).
static InstLayout layout_of(const AcTables &t, int region, int policy)
{
    const int eb = t.entry_bytes;
    const long long entries = (long long)t.n_rows << t.lw;
    const long long nw = (long long)t.flag_mask.size(), nt = (long long)t.canon.size();
    const long long tb = rr16(entries * eb);
    const long long ib = rr16(nw * 4) + rr16((nw + 1) * eb) + rr16(nt * eb);
    const long long hb = rr16(nt * 4);
    InstLayout L;
    if (tb + ib + hb <= region) {
        L.smem_entries = int(entries);
        L.ids_off = int(tb);
        L.hist_off = int(tb + ib);
        return L;
    }
    long long off = region;
    L.hist_off = L.ids_off = -1;
    if (policy == 0 && hb <= region / 4) { off -= hb; L.hist_off = int(off); }
    if (policy == 0 && ib <= region / 4) { off -= ib; L.ids_off = int(off); }
    long long se = off / eb;
    se &= ~((long long)(16 / eb) - 1);
    L.smem_entries = int(std::min(entries, se));
    return L;
}

// Per-CTA shared memory: one block of per-warp buffers, the rest is the
// instance region (table prefix, ids, counters).
int batch_shape(int warps, BatchShape &out)
{
    if (warps < 1 || warps > kBatchMaxWarps) return PM_EINVAL;
    DeviceProps dp;
    const int rc = device_props(dp);
    if (rc) return rc;
    out.warps = warps;
    const long long budget = (long long)dp.smem_optin - 2048;   // static shared memory and slack
    long long room = budget - (long long)warps * batch_warp_bytes();
    if (room < 4096) room = 4096;
    out.region_bytes = int(room & ~15LL);
    out.smem_bytes = (long long)out.region_bytes + (long long)warps * batch_warp_bytes();
    out.sm_count = dp.sm_count;
    return PM_OK;
}

bool batch_supports(const pm_set *s)
{
    return s && !s->host_only && s->algo == PM_ALGO_AC && s->ac.dna && s->ac.m <= kBatchMaxM;
}

// The descriptor of one instance (or of its part p of P, tiles [t_lo, t_hi)).
static void fill_desc(const BatchInst &I, const InstLayout &L, long long coff, BatchDesc &D)
{
    const AcTables &t = I.set->ac;
    const DevAc &dv = I.set->dac;
    std::memset(&D, 0, sizeof(D));
    D.text_off = I.text_off;
    D.n = I.text_len;
    D.count_off = I.count_off;
    D.occ_off = I.occ_off;
    D.occ_cap = I.occ_cap;
    D.ccount_off = coff;
    D.out_slot = I.out_slot;
    D.table = dv.table;
    D.mask = dv.flag_mask;
    D.rank = dv.flag_rank;
    D.canon = dv.canon;
    D.grp_off = dv.grp_off;
    D.grp_ids = dv.grp_ids;
    D.eb = t.entry_bytes;
    D.smem_entries = L.smem_entries;
    D.resident = L.smem_entries >= ((long long)t.n_rows << t.lw) ? 1 : 0;
    D.ids_off = L.ids_off;
    D.hist_off = L.hist_off;
    D.m = t.m;
    D.nwords = int(t.flag_mask.size());
    D.nterms = int(t.canon.size());
    D.d = int(t.d);
    D.mid_base = uint32_t(t.d0_row << t.lw);
    D.lut = t.lut;
    D.pre = uint32_t(dv.pre);
    D.pad = 0;
    for (uint32_t x = 0; x < 256; ++x)  // a byte outside the alphabet
        if (t.cls[x] == 0xFF) { D.pad = x; break; }
    D.t_lo = 0;
    D.t_hi = (I.text_len + kWarpTile - 1) / kWarpTile;
    D.part = 0;
    D.nparts = 1;
}

int64_t batch_fill(const BatchInst *inst, int k, const BatchShape &sh, BatchDesc *out)
{
    int64_t ccount = 0;
    for (int q = 0; q < k; ++q) {
        const BatchInst &I = inst[q];
        const AcTables &t = I.set->ac;
        const InstLayout L = layout_of(t, sh.region_bytes, sh.policy);
        const int64_t nt = int64_t(t.canon.size());
        const int64_t coff = ccount;
        if (L.hist_off < 0) ccount += nt;
        if (out) fill_desc(I, L, coff, out[q]);
    }
    return ccount;
}

int64_t batch_items(const BatchInst *inst, int k, const BatchShape &sh, bool list, std::vector<BatchDesc> &out,
                    int64_t *spill_words)
{
    out.clear();
    if (spill_words) *spill_words = 0;
    if (k <= 0) return 0;
    std::vector<InstLayout> lay(static_cast<size_t>(k));
    std::vector<double> cost(static_cast<size_t>(k));
    double total = 0.0;
    for (int q = 0; q < k; ++q) {
        const AcTables &t = inst[q].set->ac;
        lay[size_t(q)] = layout_of(t, sh.region_bytes, sh.policy);
        // a table read partly through L2 costs several times more per byte;
        // every instance also pays for loading its tables
        const long long entries = (long long)t.n_rows << t.lw;
        const double w = lay[size_t(q)].smem_entries >= entries ? 1.0 : 4.0;
        cost[size_t(q)] = double(inst[q].text_len) * w + 4.0 * double(lay[size_t(q)].smem_entries * t.entry_bytes);
        total += cost[size_t(q)];
    }
    std::vector<int> order(static_cast<size_t>(k));
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[size_t(x)] > cost[size_t(y)]; });
    // about four items per CTA: an instance above that share is split
    const double share = total / (4.0 * double(std::max(sh.sm_count, 1)));
    int64_t ccount = 0, spill = 0;
    for (const int q : order) {
        const BatchInst &I = inst[q];
        const InstLayout &L = lay[size_t(q)];
        const int64_t nt = int64_t(I.set->ac.canon.size());
        const long long ntiles = (I.text_len + kWarpTile - 1) / kWarpTile;
        long long parts = 1;
        if (cost[size_t(q)] > share && share > 0.0) {
            parts = (long long)std::ceil(cost[size_t(q)] / share);
            parts = std::min(parts, ntiles / (2LL * sh.warps));  // at least two rounds of tiles each
            parts = std::max(parts, 1LL);
        }
        int64_t coff = ccount;
        if (L.hist_off < 0 || parts > 1) ccount += nt;  // parts add into device counters
        int64_t pstat = 0, done = 0;
        if (parts > 1) {
            pstat = ccount;
            ccount += parts;
            done = ccount;
            ccount += 1;
        }
        for (long long p = 0; p < parts; ++p) {
            BatchDesc D;
            fill_desc(I, L, coff, D);
            D.t_lo = ntiles * p / parts;
            D.t_hi = ntiles * (p + 1) / parts;
            D.part = int(p);
            D.nparts = int(parts);
            D.pstat_off = pstat;
            D.done_off = done;
            if (parts > 1 && list) {
                // one key per kSpillBytes text bytes, at most the instance's capacity
                const long long bytes = std::min(D.t_hi * kWarpTile, (long long)I.text_len) - D.t_lo * kWarpTile;
                D.spill_off = spill;
                D.spill_cap = std::min<long long>((bytes + kSpillBytes - 1) / kSpillBytes, I.occ_cap);
                spill += D.spill_cap;
            }
            out.push_back(D);
        }
    }
    if (spill_words) *spill_words = spill;
    return ccount;
}

int64_t batch_words_bound(const BatchInst &I, const BatchShape &sh, bool list)
{
    const AcTables &t = I.set->ac;
    const InstLayout L = layout_of(t, sh.region_bytes, sh.policy);
    const long long ntiles = (I.text_len + kWarpTile - 1) / kWarpTile;
    const long long parts = std::max(1LL, ntiles / (2LL * std::max(sh.warps, 1)));
    int64_t w = (L.hist_off < 0 || parts > 1) ? int64_t(t.canon.size()) : 0;
    if (parts > 1) {
        w += parts + 1;
        if (list) w += std::min<int64_t>(parts * I.occ_cap, (I.text_len + kSpillBytes - 1) / kSpillBytes + parts);
    }
    return w;
}

static int ensure_batch_attr(long long smem_bytes)
{
    static std::mutex mu;
    static long long attr[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) { set_cuda_error(int(e)); return PM_ECUDA; }
    std::lock_guard<std::mutex> lk(mu);
    if (attr[dev] < smem_bytes) {
        e = cudaFuncSetAttribute(ac_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes));
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        attr[dev] = smem_bytes;
    }
    return PM_OK;
}

int batch_prepare_launch(const BatchShape &sh) { return ensure_batch_attr(sh.smem_bytes); }

// A memset of the queue, status and global counters, then the persistent
// kernel. Nothing else touches the host, so the pair can be captured in a
// graph (batch_prepare_launch must have run for the shape).
int batch_launch_raw(const BatchDesc *d_desc, int k, const uint8_t *text, int64_t *counts,
                     uint64_t *occ, int64_t *n_occ, void *ws, int64_t ccount_total,
                     const BatchShape &sh, bool list, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(ws, 0, size_t(batch_ws_bytes(ccount_total)), st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (k == 0) return PM_OK;
    BatchArgs a;
    a.desc = d_desc;
    a.k = k;
    a.text = text;
    a.counts = reinterpret_cast<long long *>(counts);
    a.occ = reinterpret_cast<unsigned long long *>(occ);
    a.n_occ = reinterpret_cast<long long *>(n_occ);
    a.ws = reinterpret_cast<dev::WsHeader *>(ws);
    a.ccount = reinterpret_cast<unsigned long long *>(static_cast<char *>(ws) + kWsHeader);
    a.spill = a.ccount + ccount_total;
    a.list = list ? 1 : 0;
    a.region_bytes = sh.region_bytes;
    const int grid = std::min(sh.sm_count, k);
    ac_batch_kernel<<<dim3(unsigned(grid)), dim3(unsigned(sh.warps * 32)), size_t(sh.smem_bytes), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    return PM_OK;
}

}  // namespace pm

// The prepared batch of the C ABI.
struct pm_batch {
    int32_t k = 0;
    std::vector<int64_t> occ_off, count_off;
    std::vector<pm::BatchInst> inst;  // as given
    int32_t n_items = 0;              // queue items (instances, or parts of large ones)
    int64_t desc_cap = 0;             // descriptors the device array holds
    pm::BatchDesc *d_desc = nullptr;
    int64_t ccount_total = 0;
    int64_t ws_bytes = 0;             // enough for every candidate shape
    int64_t d_total = 0;
    pm::BatchShape shape;
    uint32_t flags = 0;
    cudaGraphExec_t graph = nullptr;  // captured launch, see pm_batch_capture
};

namespace pm {

// Lay the batch out for `warps` warps per CTA and upload the descriptors
// (into the existing device array once there is one).
static int apply_plan(pm_batch *b, int warps, int policy)
{
    int rc = batch_shape(warps, b->shape);
    if (rc) return rc;
    b->shape.policy = policy;
    std::vector<BatchDesc> h;
    b->ccount_total = batch_items(b->inst.data(), b->k, b->shape, !(b->flags & PM_COUNTS_ONLY), h, nullptr);
    b->n_items = int32_t(h.size());
    if (h.empty()) return PM_OK;
    cudaError_t e = cudaSuccess;
    if (b->desc_cap < int64_t(h.size())) {
        if (b->d_desc) cudaFree(b->d_desc);
        b->d_desc = nullptr;
        b->desc_cap = 0;
        e = cudaMalloc(&b->d_desc, h.size() * sizeof(BatchDesc));
        if (e == cudaSuccess) b->desc_cap = int64_t(h.size());
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->d_desc, h.data(), h.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA;
    }
    return PM_OK;
}

struct BatchBufs {
    const uint8_t *text;
    int64_t *counts;
    uint64_t *occ;
    int64_t *n_occ;
    void *ws;
};

static int batch_enqueue(const pm_batch *b, const BatchBufs &o, cudaStream_t st)
{
    return batch_launch_raw(b->d_desc, b->n_items, o.text, o.counts, o.occ, o.n_occ, o.ws, b->ccount_total,
                            b->shape, !(b->flags & PM_COUNTS_ONLY), st);
}

static int batch_check(const pm_batch *b, const BatchBufs &o, int64_t ws_bytes)
{
    if (!b) return PM_EINVAL;
    if (b->k > 0 && (!o.text || !o.n_occ || !o.ws || (b->d_total > 0 && !o.counts))) return PM_EINVAL;
    if (!(b->flags & PM_COUNTS_ONLY) && b->occ_off[size_t(b->k)] > 0 && !o.occ) return PM_EINVAL;
    if (ws_bytes < b->ws_bytes) return PM_EINVAL;
    return PM_OK;
}

static void drop_graph(pm_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

}  // namespace pm

using namespace pm;

extern "C" {

int pm_batch_prepare(const pm_set *const *sets, int32_t k, const int64_t *text_off,
                     const int64_t *text_len, const int64_t *occ_off, uint32_t flags,
                     pm_batch **out)
{
    if (!out || k < 0 || (k > 0 && (!sets || !text_off || !text_len || !occ_off))) return PM_EINVAL;
    if (flags & ~(PM_DEVICE_TEXT | PM_COUNTS_ONLY)) return PM_EINVAL;
    if (k > 0 && occ_off[0] < 0) return PM_EINVAL;
    for (int32_t j = 0; j < k; ++j) {
        if (!batch_supports(sets[j])) return PM_EINVAL;
        if (text_off[j] < 0 || text_len[j] < 0 || occ_off[j + 1] < occ_off[j]) return PM_EINVAL;
        if (text_len[j] >= (int64_t(1) << 32)) return PM_ETOOBIG;
    }
    pm_batch *b = new (std::nothrow) pm_batch();
    if (!b) return PM_ENOMEM;
    try {
        b->k = k;
        b->flags = flags;
        b->occ_off.assign(occ_off, occ_off + k + 1);
        b->count_off.assign(size_t(k) + 1, 0);
        for (int32_t j = 0; j < k; ++j)
            b->count_off[size_t(j) + 1] = b->count_off[size_t(j)] + sets[j]->ac.d;
        b->d_total = b->count_off[size_t(k)];
        b->inst.resize(size_t(k));
        for (int32_t j = 0; j < k; ++j)
            b->inst[size_t(j)] = BatchInst{sets[j], text_off[j], text_len[j], b->count_off[size_t(j)],
                                           occ_off[j], occ_off[j + 1] - occ_off[j], j};
        // the workspace must hold the counters and part words of every
        // warp count the tuner may pick
        int rc = PM_OK;
        b->ws_bytes = 0;
        for (int w : kBatchWarpChoices)
            for (int policy : {0, 1}) {
                BatchShape sh;
                rc = batch_shape(w, sh);
                if (rc) { delete b; return rc; }
                sh.policy = policy;
                std::vector<BatchDesc> tmp;
                int64_t spill = 0;
                const int64_t cw = batch_items(b->inst.data(), k, sh, !(flags & PM_COUNTS_ONLY), tmp, &spill);
                b->ws_bytes = std::max<int64_t>(b->ws_bytes, batch_ws_bytes(cw) + 8 * spill);
            }
        rc = apply_plan(b, 12, 0);
        if (rc) { pm_batch_free(b); return rc; }
    } catch (const std::bad_alloc &) {
        pm_batch_free(b);
        return PM_ENOMEM;
    }
    *out = b;
    return PM_OK;
}

void pm_batch_free(pm_batch *b)
{
    if (!b) return;
    drop_graph(b);
    if (b->d_desc) cudaFree(b->d_desc);
    delete b;
}

int64_t pm_batch_workspace_bytes(const pm_batch *b) { return b ? b->ws_bytes : -1; }

int64_t pm_batch_counts_total(const pm_batch *b) { return b ? b->d_total : -1; }

int32_t pm_batch_warps(const pm_batch *b) { return b ? b->shape.warps : -1; }

int pm_batch_set_warps(pm_batch *b, int32_t warps)
{
    if (!b || warps < 1 || warps > kBatchMaxWarps) return PM_EINVAL;
    drop_graph(b);
    return apply_plan(b, warps, b->shape.policy);
}

int32_t pm_batch_placement(const pm_batch *b) { return b ? b->shape.policy : -1; }

int pm_batch_set_placement(pm_batch *b, int32_t placement)
{
    if (!b || placement < 0 || placement > 1) return PM_EINVAL;
    drop_graph(b);
    return apply_plan(b, b->shape.warps, placement);
}

int pm_batch_scan_device(const pm_batch *b, const uint8_t *d_text, int64_t *d_counts,
                         uint64_t *d_occ, int64_t *d_n_occ, void *d_workspace,
                         int64_t workspace_bytes, void *stream)
{
    const BatchBufs o{d_text, d_counts, d_occ, d_n_occ, d_workspace};
    int rc = batch_check(b, o, workspace_bytes);
    if (rc) return rc;
    rc = batch_prepare_launch(b->shape);
    if (rc) return rc;
    return batch_enqueue(b, o, static_cast<cudaStream_t>(stream));
}

int pm_batch_tune(pm_batch *b, const uint8_t *d_text, int64_t *d_counts, uint64_t *d_occ,
                  int64_t *d_n_occ, void *d_workspace, int64_t workspace_bytes, int32_t reps,
                  void *stream, float *best_ms)
{
    const BatchBufs o{d_text, d_counts, d_occ, d_n_occ, d_workspace};
    int rc = batch_check(b, o, workspace_bytes);
    if (rc) return rc;
    if (reps < 1) reps = 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    drop_graph(b);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        if (e0) cudaEventDestroy(e0);
        return PM_ECUDA;
    }
    int best_w = b->shape.warps, best_p = b->shape.policy;
    float best = -1.0f;
    for (int w : kBatchWarpChoices)
    for (int policy : {0, 1}) {
        rc = apply_plan(b, w, policy);
        if (!rc) rc = batch_prepare_launch(b->shape);
        if (!rc) rc = batch_enqueue(b, o, st);  // warm-up
        if (!rc) {
            e = cudaEventRecord(e0, st);
            for (int r = 0; r < reps && !rc && e == cudaSuccess; ++r) rc = batch_enqueue(b, o, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) { set_cuda_error(int(e)); rc = PM_ECUDA; }
            if (!rc && pm_scan_status(d_workspace, stream) != PM_OK) rc = PM_ETIMEOUT;
            if (!rc && (best < 0.0f || ms < best)) { best = ms; best_w = w; best_p = policy; }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best_ms) *best_ms = best / float(reps);
    return apply_plan(b, best_w, best_p);
}

int pm_batch_capture(pm_batch *b, const uint8_t *d_text, int64_t *d_counts, uint64_t *d_occ,
                     int64_t *d_n_occ, void *d_workspace, int64_t workspace_bytes)
{
    const BatchBufs o{d_text, d_counts, d_occ, d_n_occ, d_workspace};
    int rc = batch_check(b, o, workspace_bytes);
    if (!rc) rc = batch_prepare_launch(b->shape);
    if (rc) return rc;
    drop_graph(b);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = batch_enqueue(b, o, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (!rc && e2 != cudaSuccess) e = e2;
    }
    if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (!rc && e != cudaSuccess) {
        set_cuda_error(int(e));
        cudaGetLastError();
        b->graph = nullptr;
        rc = PM_ECUDA;
    }
    return rc;
}

int pm_batch_replay(const pm_batch *b, void *stream)
{
    if (!b || !b->graph) return PM_EINVAL;
    const cudaError_t e = cudaGraphLaunch(b->graph, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    return PM_OK;
}

}  // extern "C"
