// scan_ac.cu -- Aho-Corasick DFA scan on sm_103a.
//
// Work decomposition (the paper's data-parallel strategy, Section 4.2.1 and
// Algorithms 6 and 8, re-planned for GB300): the text is cut into warp
// tiles of 32 x 80 bytes. Lane l of a warp owns the 80 start positions
// [tile + 80 l, tile + 80 l + 80) and walks the DFA from the root over those
// bytes plus the m-1 that follow (the paper's m-1 overlap), so every start
// position belongs to exactly one lane and a match is reported by the lane
// that owns its start. A warp claims tiles from a global counter in
// increasing order, stages each tile (plus halo) into its own shared-memory
// buffer with one 1-D TMA bulk copy, loads its 80+16*HV bytes into
// registers, and immediately prefetches the next tile into the same buffer.
//
// The transition table (Section 3.1, goto and supply merged) is loaded into
// shared memory once per CTA; with hybrid placement only its breadth-first
// prefix is, and deeper rows are read through L1/L2. For an ACGT-like
// alphabet the byte->class map is arithmetic, ((b>>1)^(b>>2))&3, checked
// against a 4-byte table; bytes outside the alphabet select row 0, whose
// entries all lead to the root.
//
// The walk records, without branches, a bit per step that entered a
// terminal state and the table index of that transition (pool, shared
// memory). Afterwards each match is resolved to its terminal's canonical id
// (the rank of its table entry among match entries, from a bitmap with
// prefix counts) and to the pattern id, per-terminal counters are bumped,
// per-lane offsets come from a warp scan and the tile's global offset from a
// two-level decoupled look-back, and the sorted (i, r) keys leave through a
// shared-memory staging window so global stores are coalesced (the paper's
// coalesced writes, GPU-CW).
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "ac_device.cuh"

namespace pm {
namespace {

using dev::kFull;
using namespace acdev;

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
    int nwords, nterms;
    const uint32_t *grp_off;
    const uint32_t *grp_ids;
    const uint8_t *cls_g;
    int m, lw;
    uint32_t lut;
    uint32_t pad;
    long long ntiles;             // look-back tiles of ksub warp tiles each
    long long nsub;               // warp tiles (2560 text bytes each)
    int ksub;
    int pool_cap, stage_cap;
    int list, hist_smem, ids_smem, d;
    long long *counts;
    unsigned long long *occ;
    long long occ_cap;
    long long *n_occ;
    dev::WsHeader *ws;
    unsigned long long *ccount;   // per-terminal totals
    dev::LookbackRefs lb;
    void *scratch;                // list mode: 2 slots of ksub * kWarpTile entries per warp
};

__host__ __device__ constexpr long long r16(long long x) { return (x + 15) & ~15LL; }

__host__ __device__ inline long long ac_warp_bytes(int hv, int pool_cap, int eb, int stage_cap)
{
    // barrier | text buffer | pool (pool_cap + 1 slots per lane) | staging
    return 16 + r16(kWarpTile + 16 * hv) + r16((long long)(pool_cap + 1) * 32 * eb) +
           (long long)stage_cap * 8;
}

__host__ __device__ inline long long ac_ids_bytes(int nwords, int nterms, int eb)
{
    return r16((long long)nwords * 4) + r16((long long)(nwords + 1) * eb) + r16((long long)nterms * eb);
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

template <typename E, int NV, int HV, bool DNA, bool HYB>
__global__ void __launch_bounds__(512, 1) ac_scan_kernel(const AcArgs a)
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
    if (a.ids_smem) {
        ids.mask = reinterpret_cast<const uint32_t *>(p);
        p += r16((long long)a.nwords * 4);
        ids.rank = reinterpret_cast<const E *>(p);
        p += r16((long long)(a.nwords + 1) * sizeof(E));
        ids.canon = reinterpret_cast<const E *>(p);
        p += r16((long long)a.nterms * sizeof(E));
    } else {
        ids.mask = a.mask_g;
        ids.rank = reinterpret_cast<const E *>(a.rank_g);
        ids.canon = reinterpret_cast<const E *>(a.canon_g);
    }
    uint32_t *s_hist = a.hist_smem ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += a.hist_smem ? r16((long long)a.nterms * 4) : 0;
    uint8_t *s_cls = p;
    p += DNA ? 0 : 256;
    p += warp * ac_warp_bytes(HV, a.pool_cap, sizeof(E), a.stage_cap);
    uint64_t *bar = reinterpret_cast<uint64_t *>(p);
    uint8_t *buf = p + 16;
    E *pool = reinterpret_cast<E *>(buf + r16(BUF));
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(
        reinterpret_cast<unsigned char *>(pool) + r16((long long)(a.pool_cap + 1) * 32 * sizeof(E)));

    {   // table prefix -> shared memory (16-byte vectors; the global copy is padded)
        const uint4 *src = reinterpret_cast<const uint4 *>(a.table_g);
        uint4 *dst = reinterpret_cast<uint4 *>(s_tab);
        const int nvec = int(((long long)a.smem_entries * sizeof(E) + 15) / 16);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = src[i];
    }
    if (a.ids_smem) {
        uint32_t *mk = const_cast<uint32_t *>(ids.mask);
        for (int i = threadIdx.x; i < a.nwords; i += blockDim.x) mk[i] = a.mask_g[i];
        E *rk = const_cast<E *>(ids.rank);
        const E *rg = reinterpret_cast<const E *>(a.rank_g);
        for (int i = threadIdx.x; i <= a.nwords; i += blockDim.x) rk[i] = rg[i];
        E *cn = const_cast<E *>(ids.canon);
        const E *cg = reinterpret_cast<const E *>(a.canon_g);
        for (int i = threadIdx.x; i < a.nterms; i += blockDim.x) cn[i] = cg[i];
    }
    if (s_hist)
        for (int i = threadIdx.x; i < a.nterms; i += blockDim.x) s_hist[i] = 0u;
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
        if (s_hist) atomicAdd(&s_hist[c], 1u);
        else atomicAdd(&a.ccount[c], 1ull);
    };
    // multiplicity of a pattern code (1, or the size of its group)
    auto mult_of = [&](uint32_t code) -> uint32_t {
        if (!(code & kGrp)) return 1u;
        const uint32_t g = code & ~kGrp;
        return __ldg(a.grp_off + g + 1) - __ldg(a.grp_off + g);
    };

    // scratch entries: (start offset in the tile, pattern code)
    typedef typename std::conditional<sizeof(E) == 2, uint32_t, unsigned long long>::type SE;
    constexpr int kOffShift = sizeof(E) == 2 ? 16 : 32;
    const int K = a.ksub;
    const long long slot_len = (long long)K * kWarpTile;
    const long long gwarp = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    SE *slots = reinterpret_cast<SE *>(a.scratch) + gwarp * 2 * slot_len;
    SE *sstage = reinterpret_cast<SE *>(stage);  // staging window, SE entries
    const uint32_t S = uint32_t(a.stage_cap) * 8u / sizeof(SE);

    dev::TileSchedule sch;
    sch.init(a.ntiles);
    uint32_t phase = 0;
    bool inflight = false;
    bool failed = false;
    unsigned long long my_total = 0;
    // the tile whose output is written one round later (list mode)
    long long prev = -1;
    uint32_t prev_entries = 0, prev_slot = 0, cur_slot = 0;
    unsigned long long prev_outputs = 0;
    bool prev_group = false;

    // Emits tile u from its scratch slot once its offset is known.
    auto emit_deferred = [&](long long u, uint32_t entries, unsigned long long outputs,
                             bool group, uint32_t slot) -> bool {
        bool ok;
        const unsigned long long B = dev::tile_base(a.lb, u, lane, ok);
        if (!ok) return false;
        const long long tile0 = u * slot_len;
        const SE *sl = slots + (long long)slot * slot_len;
        if (!group) {
            // coalesced copy with 16 independent scratch loads in flight per lane
            constexpr int U = sizeof(SE) == 4 ? 16 : 8;
            const unsigned long long cap_occ = (unsigned long long)a.occ_cap;
            for (uint32_t j0 = 0; j0 < entries; j0 += 32 * U) {
                SE v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t j = j0 + u * 32 + lane;
                    v[u] = j < entries ? __ldcg(sl + j) : (SE)0;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t j = j0 + u * 32 + lane;
                    const unsigned long long gi = B + j;
                    if (j < entries && gi < cap_occ)
                        a.occ[gi] = ((unsigned long long)(tile0 + (long long)(v[u] >> kOffShift)) << 32) |
                                    (uint32_t)(v[u] & (((SE)1 << kOffShift) - 1));
                }
            }
        } else {
            unsigned long long run = 0;
            for (uint32_t w0 = 0; w0 < entries; w0 += 32) {
                const uint32_t j = w0 + lane;
                SE v = 0;
                uint32_t mult = 0, code = 0, lo = 0;
                if (j < entries) {
                    v = sl[j];
                    code = uint32_t(v & (((SE)1 << kOffShift) - 1));
                    if (code & kGrp) {
                        const uint32_t g = code & ~kGrp;
                        lo = __ldg(a.grp_off + g);
                        mult = __ldg(a.grp_off + g + 1) - lo;
                    } else {
                        mult = 1;
                    }
                }
                const uint32_t inc = dev::warp_incl_scan(mult, lane);
                const unsigned long long key_hi =
                    (unsigned long long)(tile0 + (long long)(v >> kOffShift)) << 32;
                for (uint32_t k = 0; k < mult; ++k) {
                    const uint32_t r = (code & kGrp) ? __ldg(a.grp_ids + lo + k) : code;
                    const unsigned long long gi = B + run + (inc - mult) + k;
                    if (gi < (unsigned long long)a.occ_cap) a.occ[gi] = key_hi | r;
                }
                run += __shfl_sync(kFull, inc, 31);
            }
        }
        if (lane == 0 && u == a.ntiles - 1) *a.n_occ = (long long)(B + outputs);
        return true;
    };

    if (sch.cur >= 0) {
        if (lane == 0) stage_issue(a, sch.cur * K, buf, bar, BUF);
        inflight = true;
    }

    for (long long t = sch.cur; t >= 0 && !failed; t = sch.next_of(t)) {
        const long long tn = sch.next_of(t);
        uint32_t e_base = 0;           // entries of this tile written so far
        unsigned long long o_sum = 0;  // outputs of this tile (with multiplicity)
        bool grp_tile = false;
        SE *slot = slots + (long long)cur_slot * slot_len;

        for (int sub = 0; sub < K; ++sub) {
            const long long stile = t * K + sub;  // warp tile index
            if (stile >= a.nsub) break;
            const bool got = __all_sync(kFull, dev::mbar_wait_bounded(bar, phase));
            if (!got) {
                if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutTma);
                inflight = false;  // the copy never completed; nothing to wait for
                failed = true;
                break;
            }
            inflight = false;
            phase ^= 1u;
            const long long tile0 = stile * kWarpTile;
            const int got_bytes = stage_bytes(a, stile, BUF);
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
            const long long snext =
                (sub + 1 < K && stile + 1 < a.nsub) ? stile + 1 : (tn >= 0 ? tn * K : -1);
            if (snext >= 0) {
                if (lane == 0) stage_issue(a, snext, buf, bar, BUF);
                inflight = true;
            }

            // ---- walk: branch-free recording of match steps ----------------
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
                pl[kslot * 32] = E(idx - a.mid_base);
                kslot = min(kslot + h, cap);
                hw[step >> 5] |= h << (step & 31);
            };
            if (DNA) walk_dna<NV>(tv, steps, a.lut, tab, rec);
            else walk_gen<NV>(tv, steps, a.lw, s_cls, tab, rec);
            uint32_t nh = 0;
#pragma unroll
            for (int j = 0; j < HW; ++j) nh += __popc(hw[j]);
            const bool ovf = nh > cap;

            // ---- resolve: match entry -> terminal -> pattern code -----------
            uint32_t cnt = 0;
            bool grp = false;
            if (!ovf) {
                for (uint32_t k0 = 0; k0 < nh; k0 += 4) {
                    uint32_t c4[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        c4[j] = ids.terminal(k0 + j < nh ? uint32_t(pl[(k0 + j) * 32]) : 0u);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (k0 + j < nh) {
                            const uint32_t code = ids.code(c4[j]);
                            count_terminal(c4[j]);
                            grp |= (code & kGrp) != 0;
                            cnt += mult_of(code);
                            pl[(k0 + j) * 32] = E(code);
                        }
                    }
                }
            } else {
                walk_slow(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab,
                          [&](int, uint32_t idx) {
                              const uint32_t c = ids.terminal(idx - a.mid_base);
                              const uint32_t code = ids.code(c);
                              count_terminal(c);
                              grp |= (code & kGrp) != 0;
                              cnt += mult_of(code);
                          });
            }

            if (!a.list) {
                my_total += cnt;
                continue;
            }

            // ---- entries of this warp tile -> scratch slot, in text order ---
            const uint32_t e_incl = dev::warp_incl_scan(nh, lane);
            const uint32_t e_excl = e_incl - nh;
            const uint32_t e_tot = __shfl_sync(kFull, e_incl, 31);
            unsigned long long o_tot = cnt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) o_tot += __shfl_xor_sync(kFull, o_tot, o);
            grp_tile |= __any_sync(kFull, grp);
            SE *dst = slot + e_base;
            // start offset (in the tile) of a match whose last byte is `step`
            const uint32_t off0 = uint32_t(sub * kWarpTile + lane * kChunk - (m - 1));
            if (!__any_sync(kFull, ovf)) {
                StepBits<HW> it;
#pragma unroll
                for (int j = 0; j < HW; ++j) it.w[j] = hw[j];
                it.base = 0;
                uint32_t k = 0, my = e_excl;
                for (uint32_t w0 = 0; w0 < e_tot; w0 += S) {
                    const uint32_t wend = min(w0 + S, e_tot);
                    const uint32_t lim = min(wend, e_incl);  // this lane's entries in the window
                    while (my < lim) {
                        const int stp = it.next();
                        if (stp < 0) dev::set_status(a.ws, dev::kErrInternal);
                        sstage[my - w0] = ((SE)(off0 + uint32_t(stp)) << kOffShift) | (SE)pl[k * 32];
                        ++k;
                        ++my;
                    }
                    __syncwarp();
                    for (uint32_t qq = w0 + lane; qq < wend; qq += 32) dst[qq] = sstage[qq - w0];
                    __syncwarp();
                }
            } else {
                // a lane overflowed its pool: every lane writes its entries directly
                uint32_t j = e_excl;
                if (!ovf) {
                    StepBits<HW> it;
#pragma unroll
                    for (int jj = 0; jj < HW; ++jj) it.w[jj] = hw[jj];
                    it.base = 0;
                    for (uint32_t k = 0; k < nh; ++k) {
                        const int stp = it.next();
                        if (stp < 0) dev::set_status(a.ws, dev::kErrInternal);
                        dst[j++] = ((SE)(off0 + uint32_t(stp)) << kOffShift) | (SE)pl[k * 32];
                    }
                } else {
                    walk_slow(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab,
                              [&](int step, uint32_t idx) {
                                  const uint32_t code = ids.code(ids.terminal(idx - a.mid_base));
                                  dst[j++] = ((SE)(off0 + uint32_t(step)) << kOffShift) | (SE)code;
                              });
                }
                __syncwarp();
            }
            e_base += e_tot;
            o_sum += o_tot;
        }
        if (failed || !a.list) continue;

        dev::publish_tile(a.lb, t, o_sum, lane);
        // ---- output of the previous tile, whose predecessors are done -------
        if (prev >= 0 && !emit_deferred(prev, prev_entries, prev_outputs, prev_group, prev_slot)) {
            if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutLookback);
            failed = true;
            break;
        }
        prev = t;
        prev_entries = e_base;
        prev_outputs = o_sum;
        prev_group = grp_tile;
        prev_slot = cur_slot;
        cur_slot ^= 1u;
    }
    if (!failed && prev >= 0 &&
        !emit_deferred(prev, prev_entries, prev_outputs, prev_group, prev_slot)) {
        if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutLookback);
    }

    // a prefetch issued before an error exit: wait for it (bounded) so no
    // copy is still writing this CTA's shared memory when it exits
    if (inflight) (void)dev::mbar_wait_bounded(bar, phase);

    if (!a.list) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_total += __shfl_down_sync(kFull, my_total, o);
        if (lane == 0 && my_total)
            atomicAdd(reinterpret_cast<unsigned long long *>(a.n_occ), my_total);
    }

    // ---- per-terminal counters -> global; the last CTA writes counts[r] ----
    __syncthreads();
    if (s_hist) {
        for (int c = threadIdx.x; c < a.nterms; c += blockDim.x) {
            const uint32_t v = s_hist[c];
            if (v) atomicAdd(&a.ccount[c], (unsigned long long)v);
        }
    }
    __threadfence();
    __syncthreads();
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

typedef void (*AcKernel)(const AcArgs);

struct Variant {
    AcKernel fn;
    int eb, hv;
    bool dna, hyb;
};

// variant ids: dna u16 smem (0-2), dna u16 hybrid (3-5), dna u32 hybrid
// (6-8), general u32 hybrid (9-11); within each group HV = 1, 2, 4.
const Variant kVariants[] = {
    {ac_scan_kernel<uint16_t, 6, 1, true, false>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true>, 2, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, true, true>, 4, 1, true, true},
    {ac_scan_kernel<uint32_t, 7, 2, true, true>, 4, 2, true, true},
    {ac_scan_kernel<uint32_t, 9, 4, true, true>, 4, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, false, true>, 4, 1, false, true},
    {ac_scan_kernel<uint32_t, 7, 2, false, true>, 4, 2, false, true},
    {ac_scan_kernel<uint32_t, 9, 4, false, true>, 4, 4, false, true},
};

int hv_for_m(int m)
{
    if (m - 1 <= 16) return 1;
    if (m - 1 <= 32) return 2;
    if (m - 1 <= 64) return 4;
    return -1;
}

int hv_slot(int hv) { return hv == 1 ? 0 : hv == 2 ? 1 : 2; }

struct Layout {
    long long smem_entries;
    int warps, hist, ids, stage;
};

long long ac_smem_bytes(const AcTables &t, int eb, const Layout &L, int hv, int pool_cap)
{
    const int nwords = int(t.flag_mask.size());
    const int nterms = int(t.canon.size());
    return r16(L.smem_entries * eb) + (L.ids ? ac_ids_bytes(nwords, nterms, eb) : 0) +
           (L.hist ? r16((long long)nterms * 4) : 0) + (t.dna ? 0 : 256) +
           (long long)L.warps * ac_warp_bytes(hv, pool_cap, eb, L.stage);
}

}  // namespace

int ac_plan(const AcTables &t, const pm_params &opt, const DeviceProps &dp, DevAc &dev)
{
    const int hv = hv_for_m(t.m);
    if (hv < 0) return PM_ETOOBIG;
    const int eb = t.dna ? t.entry_bytes : 4;
    const long long entries = (long long)t.n_rows << t.lw;
    const long long budget = (long long)dp.smem_optin - 1024;
    const int pool_cap = 40;
    const int place = opt.placement;
    const int forced_warps = opt.warps_per_cta > 0 ? std::min(opt.warps_per_cta, 16) : 0;
    dev.pool_cap = pool_cap;
    dev.hv = hv;
    dev.nv = 5 + hv;
    dev.ctas_per_sm = opt.ctas_per_sm > 0 ? opt.ctas_per_sm : 1;
    auto fits = [&](const Layout &L) {
        const long long need = ac_smem_bytes(t, eb, L, hv, pool_cap);
        return need <= budget &&
               need * dev.ctas_per_sm + 1024LL * dev.ctas_per_sm <= (long long)dp.smem_per_sm;
    };

    Layout best{0, 0, 0, 0, 0};
    bool chosen = false;
    if ((place == PM_PLACE_AUTO || place == PM_PLACE_SMEM) &&
        (opt.smem_table_bytes <= 0 || entries * eb <= opt.smem_table_bytes)) {
        // whole table in shared memory; prefer the id structure and the
        // counters there too, then the most warps (at least 12 if possible)
        const int ids_hist[3][2] = {{1, 1}, {1, 0}, {0, 0}};
        for (int minw : {12, 4}) {
            for (int o = 0; o < 3 && !chosen; ++o) {
                for (int stage : {128, 64}) {
                    const int hi = forced_warps ? forced_warps : 16;
                    const int lo = forced_warps ? forced_warps : minw;
                    for (int w = hi; w >= lo; --w) {
                        Layout L{entries, w, ids_hist[o][1], ids_hist[o][0], stage};
                        if (fits(L)) { best = L; chosen = true; break; }
                    }
                    if (chosen) break;
                }
            }
            if (chosen) break;
        }
        if (!chosen && place == PM_PLACE_SMEM) return PM_ETOOBIG;
        if (chosen) dev.placement = PM_PLACE_SMEM;
    }
    if (!chosen) {
        // hybrid / global: breadth-first prefix of rows in shared memory
        const int w = forced_warps ? forced_warps : 16;
        Layout L{0, w, 0, 0, 128};
        const long long fixed = ac_smem_bytes(t, eb, L, hv, pool_cap);
        long long room = budget - fixed;
        if (dev.ctas_per_sm > 1)
            room = std::min(room, (long long)dp.smem_per_sm / dev.ctas_per_sm - 1024 - fixed);
        if (opt.smem_table_bytes > 0) room = std::min<long long>(room, opt.smem_table_bytes);
        if (place == PM_PLACE_GLOBAL) room = 0;
        long long se = room > 0 ? room / eb : 0;
        se &= ~((long long)(16 / eb) - 1);   // whole 16-byte vectors
        if (se > entries) se = entries;
        L.smem_entries = se;
        best = L;
        dev.placement = place == PM_PLACE_GLOBAL ? PM_PLACE_GLOBAL : PM_PLACE_HYBRID;
    }
    dev.warps = best.warps;
    dev.hist_smem = best.hist;
    dev.ids_smem = best.ids;
    dev.stage_cap = best.stage;
    dev.smem_entries = best.smem_entries;
    const bool hyb = dev.smem_entries < entries || !t.dna || eb == 4;
    int group;
    if (!t.dna) group = 3;
    else if (eb == 4) group = 2;
    else group = hyb ? 1 : 0;
    dev.variant = group * 3 + hv_slot(hv);
    dev.smem_bytes = ac_smem_bytes(t, eb, best, hv, pool_cap);
    dev.max_warps = (long long)dp.sm_count * dev.ctas_per_sm * dev.warps;
    dev.ksub = 8;
    return PM_OK;
}

int ac_ksub_for(const DevAc &dv, int64_t n)
{
    const long long nsub = warp_tiles(n);
    int k = dv.ksub < 1 ? 1 : dv.ksub;
    while (k > 1 && (nsub + k - 1) / k < dv.max_warps) k >>= 1;
    return k;
}

int ac_launch(const AcTables &t, const DevAc &dv, const uint8_t *d_text, int64_t n, bool list,
              int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
              void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const long long nsub = warp_tiles(n);
    const int K = ac_ksub_for(dv, n);
    const long long ntiles = (nsub + K - 1) / K;
    const long long nterms = (long long)t.canon.size();
    e = cudaMemsetAsync(d_counts, 0, size_t(t.d) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_n_occ, 0, sizeof(int64_t), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_ws, 0, size_t(zeroed_workspace_bytes(ntiles, list, nterms)), st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (n < t.m || nsub == 0) return PM_OK;

    const Variant &v = kVariants[dv.variant];
    static int attr_bytes[sizeof(kVariants) / sizeof(kVariants[0])] = {};
    if (attr_bytes[dv.variant] < dv.smem_bytes) {
        e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dv.smem_bytes));
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        attr_bytes[dv.variant] = int(dv.smem_bytes);
    }
    DeviceProps dp;
    int rc = device_props(dp);
    if (rc) return rc;

    AcArgs a;
    a.text = d_text;
    a.n = n;
    a.aligned = (reinterpret_cast<uintptr_t>(d_text) & 15) == 0;
    a.table_g = dv.table;
    a.smem_entries = int(dv.smem_entries);
    a.mid_base = uint32_t(t.d0_row << t.lw);
    a.mask_g = dv.flag_mask;
    a.rank_g = dv.flag_rank;
    a.canon_g = dv.canon;
    a.nwords = int(t.flag_mask.size());
    a.nterms = int(nterms);
    a.grp_off = dv.grp_off;
    a.grp_ids = dv.grp_ids;
    a.cls_g = dv.cls;
    a.m = t.m;
    a.lw = t.lw;
    a.lut = t.lut;
    a.pad = 0;
    if (t.dna) {
        // a byte outside the alphabet: position n onward never matches
        for (uint32_t b = 0; b < 256; ++b)
            if (t.cls[b] == 0xFF) { a.pad = b; break; }
    }
    a.ntiles = ntiles;
    a.nsub = nsub;
    a.ksub = K;
    a.pool_cap = dv.pool_cap;
    a.stage_cap = dv.stage_cap;
    a.list = list ? 1 : 0;
    a.hist_smem = dv.hist_smem;
    a.ids_smem = dv.ids_smem;
    a.d = int(t.d);
    a.counts = reinterpret_cast<long long *>(d_counts);
    a.occ = reinterpret_cast<unsigned long long *>(d_occ);
    a.occ_cap = list ? occ_cap : 0;
    a.n_occ = reinterpret_cast<long long *>(d_n_occ);
    char *w = static_cast<char *>(d_ws);
    a.ws = reinterpret_cast<dev::WsHeader *>(w);
    a.ccount = reinterpret_cast<unsigned long long *>(w + kWsHeader);
    char *after = w + kWsHeader + r16(nterms * 8);
    a.lb.tile_st = reinterpret_cast<unsigned long long *>(after);
    a.lb.super_acc = reinterpret_cast<unsigned long long *>(after + ntiles * 8);
    a.lb.super_pre = reinterpret_cast<unsigned long long *>(after + ntiles * 16);
    a.lb.ntiles = ntiles;
    a.scratch = after + r16(ntiles * 24);

    // the static tile schedule needs every CTA of the grid resident at once
    const int threads = dv.warps * 32;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fn, threads, size_t(dv.smem_bytes));
    if (e != cudaSuccess || per_sm < 1) { set_cuda_error(int(e)); return PM_ECUDA; }
    long long grid = (long long)dp.sm_count * std::min(per_sm, dv.ctas_per_sm);
    const long long want = (ntiles + dv.warps - 1) / dv.warps;  // look-back tiles
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    if (grid * dv.warps > dv.max_warps) grid = dv.max_warps / dv.warps;
    a.lb.super_tiles = dev::super_size_for(grid * dv.warps);
    v.fn<<<dim3(unsigned(grid)), dim3(unsigned(threads)), size_t(dv.smem_bytes), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    return PM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free scan (pm_scan_device_noalloc).
//
// Some callers cannot allocate device memory when they scan: a host
// application that owns the GPU allocator (a plugin must not add cudaMalloc
// calls it cannot account for), or a latency-bound loop that reserved all
// of its memory up front and must not call cudaMalloc, which can block on
// the device and fail once memory is fragmented. For them the scratch of
// the Aho-Corasick scan lives in one fixed array inside the library. The
// array is reserved on every GPU that loads the library and stays reserved
// until the process exits. Every call uses the same array and it keeps the
// last call's contents, so the launcher clears what must start at zero, and
// two calls whose work overlaps on the GPU (different streams, or host
// threads) race on it. To keep the array modest the scan runs with one warp
// tile per look-back tile (the per-warp output slots then need only two
// warp tiles of entries).
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {};

// Device address of the scratch array on the current device. The first call
// on a device looks it up (host code cannot use the array's name as an
// address); later calls reuse it.
int noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        set_cuda_error(int(e));
        cudaGetLastError();
        return PM_ENODEV;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_cuda_error(int(e));
            cudaGetLastError();
            return PM_ECUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return PM_OK;
}
}  // namespace

int64_t ac_noalloc_limit_bytes() { return int64_t(kNoAllocScratchBytes); }

int ac_launch_noalloc(const AcTables &t, const DevAc &dv, const uint8_t *d_text, int64_t n,
                      bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap,
                      int64_t *d_n_occ, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const int K = 1;
    const long long nsub = warp_tiles(n);
    const long long ntiles = nsub;
    const long long nterms = (long long)t.canon.size();
    const Variant &v = kVariants[dv.variant];
    DeviceProps dp;
    int rc = device_props(dp);
    if (rc) return rc;

    // the grid the launch will use decides the size of the output slots
    static int attr_bytes_na[sizeof(kVariants) / sizeof(kVariants[0])] = {};
    if (attr_bytes_na[dv.variant] < dv.smem_bytes) {
        e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dv.smem_bytes));
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        attr_bytes_na[dv.variant] = int(dv.smem_bytes);
    }
    const int threads = dv.warps * 32;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fn, threads, size_t(dv.smem_bytes));
    if (e != cudaSuccess || per_sm < 1) { set_cuda_error(int(e)); return PM_ECUDA; }
    long long grid = (long long)dp.sm_count * std::min(per_sm, dv.ctas_per_sm);
    const long long want = (ntiles + dv.warps - 1) / dv.warps;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    if (grid * dv.warps > dv.max_warps) grid = dv.max_warps / dv.warps;

    const long long se = sizeof(uint32_t) * ((t.dna ? t.entry_bytes : 4) == 2 ? 1 : 2);
    const long long zeroed = zeroed_workspace_bytes(ntiles, list, nterms);
    const long long slots = list ? r16(grid * dv.warps * 2LL * K * kWarpTile * se) : 0;
    if (zeroed + slots > (long long)kNoAllocScratchBytes) return PM_ETOOBIG;

    void *ws = nullptr;
    rc = noalloc_scratch(&ws);
    if (rc) return rc;
    e = cudaMemsetAsync(d_counts, 0, size_t(t.d) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_n_occ, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, size_t(zeroed), st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (n < t.m || nsub == 0) return PM_OK;

    AcArgs a;
    a.text = d_text;
    a.n = n;
    a.aligned = (reinterpret_cast<uintptr_t>(d_text) & 15) == 0;
    a.table_g = dv.table;
    a.smem_entries = int(dv.smem_entries);
    a.mid_base = uint32_t(t.d0_row << t.lw);
    a.mask_g = dv.flag_mask;
    a.rank_g = dv.flag_rank;
    a.canon_g = dv.canon;
    a.nwords = int(t.flag_mask.size());
    a.nterms = int(nterms);
    a.grp_off = dv.grp_off;
    a.grp_ids = dv.grp_ids;
    a.cls_g = dv.cls;
    a.m = t.m;
    a.lw = t.lw;
    a.lut = t.lut;
    a.pad = 0;
    if (t.dna) {
        for (uint32_t b = 0; b < 256; ++b)
            if (t.cls[b] == 0xFF) { a.pad = b; break; }
    }
    a.ntiles = ntiles;
    a.nsub = nsub;
    a.ksub = K;
    a.pool_cap = dv.pool_cap;
    a.stage_cap = dv.stage_cap;
    a.list = list ? 1 : 0;
    a.hist_smem = dv.hist_smem;
    a.ids_smem = dv.ids_smem;
    a.d = int(t.d);
    a.counts = reinterpret_cast<long long *>(d_counts);
    a.occ = reinterpret_cast<unsigned long long *>(d_occ);
    a.occ_cap = list ? occ_cap : 0;
    a.n_occ = reinterpret_cast<long long *>(d_n_occ);
    char *w = static_cast<char *>(ws);
    a.ws = reinterpret_cast<dev::WsHeader *>(w);
    a.ccount = reinterpret_cast<unsigned long long *>(w + kWsHeader);
    char *after = w + kWsHeader + r16(nterms * 8);
    a.lb.tile_st = reinterpret_cast<unsigned long long *>(after);
    a.lb.super_acc = reinterpret_cast<unsigned long long *>(after + ntiles * 8);
    a.lb.super_pre = reinterpret_cast<unsigned long long *>(after + ntiles * 16);
    a.lb.ntiles = ntiles;
    a.lb.super_tiles = dev::super_size_for(grid * dv.warps);
    a.scratch = after + r16(ntiles * 24);
    v.fn<<<dim3(unsigned(grid)), dim3(unsigned(threads)), size_t(dv.smem_bytes), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    return PM_OK;
}

}  // namespace pm
