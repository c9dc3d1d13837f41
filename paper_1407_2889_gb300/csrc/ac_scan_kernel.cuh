// ac_scan_kernel.cuh -- the plain Aho-Corasick scan kernel (one character
// per lookup) and its launch arguments, shared by the three translation units
// that instantiate it: scan_ac.cu (512-thread launch bound, up to 16 warps
// per CTA and 128 registers), scan_ac_wide.cu (768 threads, up to 24 warps
// and 85 registers) and scan_ac_wide_counts.cu (the 768-thread ones for
// counts-only scans). The work decomposition and the walk are described at
// the top of scan_ac.cu.
#pragma once

#include <cstdint>
#include <type_traits>

#include "ac_device.cuh"

namespace pm {

struct AcArgs {
    const uint8_t *text;
    long long n;
    int aligned;
    const void *table_g;
    int smem_entries;
    uint32_t mid_base;            // first table index of the match rows
    const uint32_t *mask_g;       // match-entry bitmap words
    const void *rank_g;           // E: set bits before each word
    const void *canon_g;          // E: pattern id or group flag per terminal
    const uint32_t *tmul_g;       // late ids: 2 bits per terminal, min(multiplicity - 1, 3)
    const uint32_t *emul_g;       // late ids: 2 bits per match entry, the same for the terminal it enters
    int nwords, nterms;
    const uint32_t *grp_off;
    const uint32_t *grp_ids;
    const uint8_t *cls_g;
    int m, lw;
    uint32_t lut;
    uint32_t pad;
    long long nsub;               // warp tiles (2560 text bytes each)
    int pool_cap;
    int list, hist_smem, ids_smem, d;
    int late;                     // list mode with late ids: slots carry match-entry offsets, no counting here
    long long *counts;
    long long *n_occ;
    dev::WsHeader *ws;
    unsigned long long *ccount;   // per-terminal totals
    uint32_t *tile_ent;           // list: entries (one per matching position) per warp tile
    uint32_t *tile_out;           // list: outputs (keys, groups expanded) per warp tile
    unsigned long long *seg_sum;  // list: outputs per segment of seg_tiles warp tiles
    long long seg_tiles;
    void *slots;                  // list: kWarpTile entries per warp tile
};

typedef void (*AcKernel)(const AcArgs);

struct Variant {
    AcKernel fn;
    int eb, hv;
    bool dna, hyb;
};

// The 768-thread instances (scan_ac_wide.cu), indexed by wide group x 3 +
// HV slot (HV = 1, 2, 4). Wide groups 0-4 are the ACGT groups of the
// 512-thread table (u16 whole table, u16 hybrid, u16 whole table with index
// entries, u16 hybrid with index entries, u32 hybrid with index entries),
// 5-9 their late-ids forms. kWideCountsVariants (scan_ac_wide_counts.cu)
// are the same kernels for counts-only scans, which record no step bits.
constexpr int kWideGroups = 10;
extern const Variant kWideVariants[kWideGroups * 3];
extern const Variant kWideCountsVariants[kWideGroups * 3];

namespace {

using dev::kFull;
using namespace acdev;

__host__ __device__ constexpr long long r16(long long x) { return (x + 15) & ~15LL; }

__host__ __device__ inline long long ac_warp_bytes(int hv, int pool_cap, int eb)
{
    // barrier | text buffer | pool (pool_cap + 1 slots per lane)
    return 16 + r16(kWarpTile + 16 * hv) + r16((long long)(pool_cap + 1) * 32 * eb);
}

__device__ __forceinline__ int stage_bytes(const AcArgs &a, long long t, int buf)
{
    if (!a.aligned) return 0;
    const long long avail = (a.n & ~15LL) - t * kWarpTile;
    if (avail <= 0) return 0;
    return avail >= buf ? buf : int(avail);
}

__device__ __forceinline__ void stage_issue(const AcArgs &a, long long t, uint8_t *buf,
                                            uint64_t *bar, int bufsz)
{
    const int bytes = stage_bytes(a, t, bufsz);
    dev::mbar_arrive_expect_tx(bar, uint32_t(bytes));
    if (bytes > 0) dev::tma_load_1d(buf, a.text + t * kWarpTile, uint32_t(bytes), bar);
}

// MAXT: the launch bound, 512 threads (up to 128 registers) or 768 (up to
// 85, for plans of more than 16 warps). CO: an instance for counts-only
// scans, whose walk records no step bits (a lane's hit count is its pool
// counter, and a full pool counts as an overflow).
template <typename E, int NV, int HV, bool DNA, bool HYB, bool PRE, bool LATE, int MAXT, bool CO = false>
__global__ void __launch_bounds__(MAXT, 1) ac_scan_kernel(const AcArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int BUF = kWarpTile + 16 * HV;
    constexpr int HW = (16 * NV + 31) / 32;
    constexpr uint32_t kGrp = sizeof(E) == 2 ? 0x8000u : 0x80000000u;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    // ---- shared memory carve-up (mirrors ac_smem_bytes on the host) -------
    unsigned char *p = smem;
    E *s_tab = reinterpret_cast<E *>(p);
    p += r16((long long)a.smem_entries * sizeof(E));
    Ids<E> ids;
    uint32_t *s_tmul = nullptr;  // late ids, counts mode: the terminals' multiplicities
    uint32_t *s_emul = nullptr;  // late ids, list mode: the match entries' multiplicities
    const bool late_list = LATE && a.late;
    if (late_list) {
        // only the multiplicities; the id structure stays in device memory
        // for groups of four or more equal patterns (ids keeps the places
        // of its counts-mode layout, unread here, so that its loads stay
        // shared-memory loads there)
        ids.mask = reinterpret_cast<const uint32_t *>(p);
        ids.rank = reinterpret_cast<const E *>(p);
        ids.canon = reinterpret_cast<const E *>(a.canon_g);
        s_emul = reinterpret_cast<uint32_t *>(p);
        p += r16((long long)a.nwords * 8);
    } else if (LATE || a.ids_smem) {
        ids.mask = reinterpret_cast<const uint32_t *>(p);
        p += r16((long long)a.nwords * 4);
        ids.rank = reinterpret_cast<const E *>(p);
        p += r16((long long)(a.nwords + 1) * sizeof(E));
        if (!LATE) {
            ids.canon = reinterpret_cast<const E *>(p);
            p += r16((long long)a.nterms * sizeof(E));
        } else {
            ids.canon = reinterpret_cast<const E *>(a.canon_g);
            s_tmul = reinterpret_cast<uint32_t *>(p);
            p += r16((long long)(a.nterms + 15) / 16 * 4);
        }
    } else {
        ids.mask = a.mask_g;
        ids.rank = reinterpret_cast<const E *>(a.rank_g);
        ids.canon = reinterpret_cast<const E *>(a.canon_g);
    }
    // per-terminal counters: 32-bit (hist_smem 1) or two 16-bit halves per
    // word (hist_smem 2) in shared memory, else 64-bit in the workspace
    uint32_t *s_hist = a.hist_smem ? reinterpret_cast<uint32_t *>(p) : nullptr;
    const long long hist_words = a.hist_smem == 2 ? (a.nterms + 1) / 2 : a.nterms;
    p += a.hist_smem ? r16(hist_words * 4) : 0;
    uint8_t *s_cls = p;
    p += DNA ? 0 : 256;
    p += warp * ac_warp_bytes(HV, a.pool_cap, sizeof(E));
    uint64_t *bar = reinterpret_cast<uint64_t *>(p);
    uint8_t *buf = p + 16;
    E *pool = reinterpret_cast<E *>(buf + r16(BUF));

    {   // table prefix -> shared memory (16-byte vectors; the global copy is padded)
        const uint4 *src = reinterpret_cast<const uint4 *>(a.table_g);
        uint4 *dst = reinterpret_cast<uint4 *>(s_tab);
        const int nvec = int(((long long)a.smem_entries * sizeof(E) + 15) / 16);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = src[i];
    }
    if (late_list) {
        for (int i = threadIdx.x; i < 2 * a.nwords; i += blockDim.x) s_emul[i] = a.emul_g[i];
    } else if (LATE || a.ids_smem) {
        uint32_t *mk = const_cast<uint32_t *>(ids.mask);
        for (int i = threadIdx.x; i < a.nwords; i += blockDim.x) mk[i] = a.mask_g[i];
        E *rk = const_cast<E *>(ids.rank);
        const E *rg = reinterpret_cast<const E *>(a.rank_g);
        for (int i = threadIdx.x; i <= a.nwords; i += blockDim.x) rk[i] = rg[i];
        if (!LATE) {
            E *cn = const_cast<E *>(ids.canon);
            const E *cg = reinterpret_cast<const E *>(a.canon_g);
            for (int i = threadIdx.x; i < a.nterms; i += blockDim.x) cn[i] = cg[i];
        } else {
            for (int i = threadIdx.x; i < (a.nterms + 15) / 16; i += blockDim.x) s_tmul[i] = a.tmul_g[i];
        }
    }
    if (s_hist)
        for (int i = threadIdx.x; i < hist_words; i += blockDim.x) s_hist[i] = 0u;
    if (!DNA)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) s_cls[i] = a.cls_g[i];
    if (lane == 0) dev::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dev::fence_proxy_async_smem();
    __syncthreads();

    const TableRef<E, HYB> tab{s_tab, reinterpret_cast<const E *>(a.table_g),
                               uint32_t(a.smem_entries)};
    E *pl = pool + lane;  // this lane's pool column (stride 32 entries)
    const uint32_t cap = uint32_t(a.pool_cap);
    const int m = a.m;

    auto count_terminal = [&](uint32_t c) {
        if (a.hist_smem == 1) {
            atomicAdd(&s_hist[c], 1u);
        } else if (a.hist_smem == 2) {
            // the add that takes a half to 0x8000 moves 0x8000 to the global
            // counter, so a half never wraps (it would take 0x8000 more adds
            // between that add and the move)
            const uint32_t sh = (c & 1u) << 4;
            const uint32_t old = atomicAdd(&s_hist[c >> 1], 1u << sh);
            if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
                atomicSub(&s_hist[c >> 1], 0x8000u << sh);
                atomicAdd(&a.ccount[c], 0x8000ull);
            }
        } else {
            atomicAdd(&a.ccount[c], 1ull);
        }
    };
    // offset of a recorded table index among the match rows' entries (in
    // 16-bit arithmetic for u16 tables, whose match rows span < 65536 entries)
    auto match_off = [&](E v) -> uint32_t {
        return sizeof(E) == 2 ? uint32_t(uint16_t(v - E(a.mid_base))) : uint32_t(v) - a.mid_base;
    };
    // multiplicity of a pattern code (1, or the size of its group)
    auto mult_of = [&](uint32_t code) -> uint32_t {
        if (!(code & kGrp)) return 1u;
        const uint32_t g = code & ~kGrp;
        return __ldg(a.grp_off + g + 1) - __ldg(a.grp_off + g);
    };
    // what a terminal's hit contributes: its outputs, and the slot value (its
    // pattern code; in the counts mode of late ids the terminal id itself,
    // whose multiplicity comes from the 2-bit table, and through canon in
    // device memory only for groups of four or more equal patterns)
    auto resolve = [&](uint32_t c, uint32_t &mult) -> uint32_t {
        if (LATE) {
            const uint32_t v = (s_tmul[c >> 4] >> ((c & 15u) << 1)) & 3u;
            mult = v < 3u ? v + 1u : mult_of(uint32_t(__ldg(ids.canon + c)));
            return c;
        }
        const uint32_t code = ids.code(c);
        mult = mult_of(code);
        return code;
    };
    // late ids in list mode: the outputs of a match entry (offset o among
    // the match rows' entries) from its 2-bit multiplicity; the id structure
    // in device memory names the group of four or more
    auto entry_mult = [&](uint32_t o) -> uint32_t {
        const uint32_t v = (s_emul[o >> 4] >> ((o & 15u) << 1)) & 3u;
        if (v < 3u) return v + 1u;
        const uint32_t w = o >> 5;
        const uint32_t c = uint32_t(__ldg(reinterpret_cast<const E *>(a.rank_g) + w)) +
                           __popc(__ldg(a.mask_g + w) & ((1u << (o & 31u)) - 1u));
        return mult_of(uint32_t(__ldg(reinterpret_cast<const E *>(a.canon_g) + c)));
    };

    // slot entries: (start offset in the tile, pattern code or, with late
    // ids, match-entry offset)
    typedef typename std::conditional<sizeof(E) == 2, uint32_t, unsigned long long>::type SE;
    constexpr int kOffShift = sizeof(E) == 2 ? 16 : 32;
    const long long G = (long long)gridDim.x * (blockDim.x >> 5);
    const long long gwarp = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    SE *slots = reinterpret_cast<SE *>(a.slots);

    uint32_t phase = 0;
    bool inflight = false;
    bool failed = false;
    unsigned long long my_total = 0;

    if (gwarp < a.nsub) {
        if (lane == 0) stage_issue(a, gwarp, buf, bar, BUF);
        inflight = true;
    }

    for (long long st = gwarp; st < a.nsub && !failed; st += G) {
        const bool got = __all_sync(kFull, dev::mbar_wait_bounded(bar, phase));
        if (!got) {
            if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutTma);
            failed = true;  // the copy stays in flight: waited for below
            break;
        }
        inflight = false;
        phase ^= 1u;
        const long long tile0 = st * kWarpTile;
        const int got_bytes = stage_bytes(a, st, BUF);
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
            if (lane == 0) stage_issue(a, st + G, buf, bar, BUF);
            inflight = true;
        }

        // ---- walk: a step that enters a terminal stores its table index ----
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
        // pool slot `cap` absorbs the stores of an overflowing lane
        auto rec = [&](int step, uint32_t idx, uint32_t e) {
            const uint32_t h = e & 1u;
            if (h) pl[kslot * 32] = E(idx);  // the match-row base is subtracted when resolving
            kslot = min(kslot + h, cap);
            if (!CO) hw[step >> 5] += h << (step & 31);
        };
        if (DNA) walk_dna<NV, PRE>(tv, steps, a.lut, tab, rec);
        else walk_gen<NV>(tv, steps, a.lw, s_cls, tab, rec);
        uint32_t nh = 0;  // exact even when the pool overflowed (CO: up to cap)
        if (CO) {
            nh = kslot;
        } else {
#pragma unroll
            for (int j = 0; j < HW; ++j) nh += __popc(hw[j]);
        }
        const bool ovf = CO ? kslot >= cap : nh > cap;

        // ---- resolve: match entry -> terminal -> pattern code ---------------
        // (late ids in list mode: no resolve; the compaction below adds up the
        // multiplicities)
        uint32_t cnt = 0;
        if (!late_list && !ovf) {
            for (uint32_t k0 = 0; k0 < nh; k0 += 4) {
                uint32_t c4[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    c4[j] = ids.terminal(k0 + j < nh ? match_off(pl[(k0 + j) * 32]) : 0u);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (k0 + j < nh) {
                        uint32_t mult;
                        const uint32_t val = resolve(c4[j], mult);
                        count_terminal(c4[j]);
                        cnt += mult;
                        pl[(k0 + j) * 32] = E(val);
                    }
                }
            }
        } else if (!late_list) {
            walk_slow<PRE>(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab,
                      [&](int, uint32_t idx) {
                          const uint32_t c = ids.terminal(idx - a.mid_base);
                          uint32_t mult;
                          (void)resolve(c, mult);
                          count_terminal(c);
                          cnt += mult;
                      });
        }

        if (CO || !a.list) {
            my_total += cnt;
            continue;
        }

        // ---- this tile's matches -> its slot, in text order -----------------
        const uint32_t e_incl = dev::warp_incl_scan(nh, lane);
        const uint32_t e_excl = e_incl - nh;
        SE *dst = slots + st * kWarpTile + e_excl;
        // start offset (in the tile) of a match whose last byte is `step`
        const uint32_t off0 = uint32_t(lane * kChunk - (m - 1));
        if (late_list && !ovf) {
            // slot values: match-entry offsets (the expand kernel takes the
            // terminal ids, codes and counts from them)
            uint32_t k = 0;
            bool big = false;  // a group of four or more equal patterns
#pragma unroll
            for (int j = 0; j < HW; ++j) {
                uint32_t wj = hw[j];
                while (wj) {
                    const uint32_t b = uint32_t(__ffs(int(wj))) - 1u;
                    wj &= wj - 1u;
                    const uint32_t o = match_off(pl[k * 32]);
                    const uint32_t v = (s_emul[o >> 4] >> ((o & 15u) << 1)) & 3u;
                    cnt += v + 1u;
                    big |= v == 3u;
                    dst[k] = ((SE)(off0 + uint32_t(j * 32) + b) << kOffShift) | (SE)o;
                    ++k;
                }
            }
            if (big) {  // rare: those hits' true multiplicities instead of 4
                for (uint32_t q = 0; q < nh; ++q) {
                    const uint32_t o = match_off(pl[q * 32]);
                    if (((s_emul[o >> 4] >> ((o & 15u) << 1)) & 3u) == 3u) cnt += entry_mult(o) - 4u;
                }
            }
        } else if (late_list) {
            uint32_t k = 0;
            walk_slow<PRE>(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab,
                      [&](int step, uint32_t idx) {
                          const uint32_t o = idx - a.mid_base;
                          cnt += entry_mult(o);
                          if (k < nh) dst[k] = ((SE)(off0 + uint32_t(step)) << kOffShift) | (SE)o;
                          ++k;
                      });
        } else if (!ovf) {
            // the lane's match steps in order, word by word of its step mask
            uint32_t k = 0;
#pragma unroll
            for (int j = 0; j < HW; ++j) {
                uint32_t wj = hw[j];
                while (wj) {
                    const uint32_t b = uint32_t(__ffs(int(wj))) - 1u;
                    wj &= wj - 1u;
                    dst[k] = ((SE)(off0 + uint32_t(j * 32) + b) << kOffShift) | (SE)pl[k * 32];
                    ++k;
                }
            }
        } else {
            uint32_t k = 0;
            walk_slow<PRE>(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab,
                      [&](int step, uint32_t idx) {
                          uint32_t mult;
                          const uint32_t val = resolve(ids.terminal(idx - a.mid_base), mult);
                          if (k < nh) dst[k] = ((SE)(off0 + uint32_t(step)) << kOffShift) | (SE)val;
                          ++k;
                      });
        }
        uint32_t o_tot = cnt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) o_tot += __shfl_xor_sync(kFull, o_tot, o);
        if (lane == 31) {
            a.tile_ent[st] = e_incl;
            a.tile_out[st] = o_tot;
            if (o_tot) atomicAdd(&a.seg_sum[st / a.seg_tiles], (unsigned long long)o_tot);
        }
    }

    // a copy still in flight after an error exit: wait for it (bounded) so
    // it is not still writing this CTA's shared memory when the CTA exits
    if (inflight) (void)dev::mbar_wait_bounded(bar, phase);

    if (CO || !a.list) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_total += __shfl_down_sync(kFull, my_total, o);
        if (lane == 0 && my_total)
            atomicAdd(reinterpret_cast<unsigned long long *>(a.n_occ), my_total);
    }

    // ---- per-terminal counters -> global; the last CTA writes counts[r] ----
    __syncthreads();
    if (s_hist) {
        for (int c = threadIdx.x; c < a.nterms; c += blockDim.x) {
            const uint32_t v = a.hist_smem == 2 ? (s_hist[c >> 1] >> ((c & 1) << 4)) & 0xFFFFu : s_hist[c];
            if (v) atomicAdd(&a.ccount[c], (unsigned long long)v);
        }
    }
    __threadfence();
    __syncthreads();
    if (LATE && a.late) return;  // the expand kernel counts and writes counts[r]
    __shared__ int s_last;
    if (threadIdx.x == 0) s_last = atomicAdd(&a.ws->done_ctas, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        const E *cg = reinterpret_cast<const E *>(a.canon_g);
        for (int c = threadIdx.x; c < a.nterms; c += blockDim.x) {
            const unsigned long long v = dev::ld_acquire(&a.ccount[c]);
            const uint32_t code = cg[c];
            if (code & kGrp) {
                const uint32_t g = code & ~kGrp;
                for (uint32_t j = a.grp_off[g]; j < a.grp_off[g + 1]; ++j)
                    a.counts[a.grp_ids[j]] = (long long)v;
            } else {
                a.counts[code] = (long long)v;
            }
        }
    }
}

}  // namespace
}  // namespace pm
