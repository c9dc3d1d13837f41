// scan_ac.cu -- Aho-Corasick DFA scan on sm_103a.
//
// Work decomposition (the paper's data-parallel strategy, Section 4.2.1 and
// Algorithms 6 and 8, re-planned for GB300): the text is cut into warp
// tiles of 32 x 80 bytes. Lane l of a warp owns the 80 start positions
// [tile + 80 l, tile + 80 l + 80) and walks the DFA from the root over those
// bytes plus the m-1 that follow (the paper's m-1 overlap), so every start
// position belongs to exactly one lane and a match is reported by the lane
// that owns its start. Warp w of the grid takes tiles w, w + G, w + 2G ...,
// stages each tile (plus halo) into its own shared-memory buffer with one
// 1-D TMA bulk copy, loads its 80+16*HV bytes into registers, and
// immediately prefetches its next tile into the same buffer.
//
// The transition table (Section 3.1, goto and supply merged) is loaded into
// shared memory once per CTA; with hybrid placement only its breadth-first
// prefix is, and deeper rows are read through L1/L2. For an ACGT-like
// alphabet the byte->class map is arithmetic, ((b>>1)^(b>>2))&3, checked
// against a 4-byte table; bytes outside the alphabet select row 0, whose
// entries all lead to the root.
//
// The walk records, without branches, a bit per step that entered a
// terminal state, and the table index of such a step in the lane's hit pool
// (shared memory). Afterwards each match is resolved to its terminal's
// canonical id (the rank of its table entry among match entries, from a
// bitmap with prefix counts) and to the pattern code, and per-terminal
// counters are bumped; the last CTA turns them into counts[r]. With late ids
// in list mode the scan keeps the match entry's offset and only adds up its
// outputs (a 2-bit multiplicity per match entry); the expand kernel does the
// rest.
//
// List mode writes the output in two launches, so that no warp ever waits
// for another: the scan writes each warp tile's matches, in text order, to
// that tile's own slot of kWarpTile entries (at most one distinct pattern
// string starts at a position) with the tile's totals and its segment's
// sum; an expand kernel with many resident warps turns the totals into
// offsets and copies the slots to the sorted (i, r) keys, one key per
// pattern of a group of equal patterns (the paper's coalesced writes,
// GPU-CW).
//
// The kernel itself is in ac_scan_kernel.cuh: this file instantiates it with
// a 512-thread launch bound, scan_ac_wide.cu and scan_ac_wide_counts.cu
// (counts-only scans) with 768 threads.
#include <cstddef>
#include <cstdio>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "ac_scan_kernel.cuh"

namespace pm {
namespace {

using dev::kFull;
using namespace acdev;


// Workspace carve-up shared by the launchers and the workspace size:
//   [header][per-terminal counters][list: segment sums u64] -- zeroed by every scan
//   list mode: [tile_ent u32][tile_out u32][slots]
struct AcWsLayout {
    long long seg_sum, zeroed, tile_ent, tile_out, slots, total;
};

// Output segments of the list mode: one expand CTA per segment of
// consecutive warp tiles (two CTAs per SM, at least 64 tiles each).
inline long long ac_segments(long long nsub, int sm_count)
{
    long long b = 2LL * (sm_count > 0 ? sm_count : 1);
    const long long most = (nsub + 63) / 64;
    if (most < b) b = most;
    return b < 1 ? 1 : b;
}


AcWsLayout ac_ws_layout(long long nsub, bool list, long long nterms, int slot_entry_bytes, int sm_count)
{
    AcWsLayout L;
    L.seg_sum = kWsHeader + r16(nterms * 8);
    L.zeroed = L.seg_sum + (list ? r16(ac_segments(nsub, sm_count) * 8) : 0);
    L.tile_ent = L.zeroed;
    L.tile_out = L.tile_ent + (list ? r16(nsub * 4) : 0);
    L.slots = L.tile_out + (list ? r16(nsub * 4) : 0);
    L.total = L.slots + (list ? r16(nsub * kWarpTile * (long long)slot_entry_bytes) : 0);
    return L;
}

__host__ __device__ inline long long ac_ids_bytes(int nwords, int nterms, int eb)
{
    return r16((long long)nwords * 4) + r16((long long)(nwords + 1) * eb) + r16((long long)nterms * eb);
}

// late ids, counts mode: match bitmap, ranks and the terminals' 2-bit
// multiplicities
__host__ __device__ inline long long ac_ids_late_bytes(int nwords, int nterms, int eb)
{
    return r16((long long)nwords * 4) + r16((long long)(nwords + 1) * eb) + r16((long long)(nterms + 15) / 16 * 4);
}

// late ids, list mode: the match entries' 2-bit multiplicities
__host__ __device__ inline long long ac_emul_bytes(int nwords) { return r16((long long)nwords * 8); }


// ---------------------------------------------------------------------------
// List mode, step 2: slots -> sorted keys ((i << 32) | r). CTA b owns the
// warp tiles of segment b: its output base is the sum of the earlier
// segments' totals (added up by the scan), each tile's offset inside the
// segment comes from a block scan of the tiles' totals kept in shared
// memory, and its warps then copy one tile at a time in rows of 32 entries
// (lane l takes entry l of a row, ten rows loaded together), so slot loads
// and key stores are both coalesced. A row that names a group of equal
// patterns takes a warp prefix over the entries' multiplicities instead. The
// CTA that owns the last tile writes the total.
// With late ids the entries carry match-entry offsets: each is mapped to
// its terminal id (rank of the entry in the match bitmap) and through canon
// to its pattern code and counted per terminal (in shared memory when the id
// structure and the counters fit there), the counters go to the workspace
// when the CTA is done, and the last CTA to finish writes counts[r].
// CM, the counter mode: 0 no late ids; late ids with canon and 32-bit (1) or
// 16-bit (2) counters in shared memory, or both in device memory (3). GS:
// the group tables are in shared memory. Both are template parameters so
// that every table load is a plain shared or global load.
// ---------------------------------------------------------------------------
constexpr int kExpandThreads = 512;

struct ExpandLateArgs {
    const void *canon;            // u16 (4-byte slots) or u32 per terminal
    const uint32_t *mask;         // match-entry bitmap
    const void *rank;             // set bits before each bitmap word (type of canon)
    long long nterms, nwords;
    int smem;                     // canon and counters in shared memory: 1 32-bit, 2 16-bit counters; 0 neither
    unsigned long long *ccount;   // per-terminal counters (workspace)
    long long *counts;
    dev::WsHeader *ws;
};

template <typename SE, int kOffShift, uint32_t kGrp, int CM, bool GS>
__global__ void __launch_bounds__(kExpandThreads)
expand_kernel(const SE *__restrict__ slots, const uint32_t *__restrict__ tile_ent,
              const uint32_t *__restrict__ tile_out, const unsigned long long *__restrict__ seg_sum,
              long long nseg, long long seg_tiles, long long nsub,
              const uint32_t *__restrict__ grp_off, const uint32_t *__restrict__ grp_ids,
              unsigned long long *__restrict__ occ, long long occ_cap, long long *n_occ,
              const unsigned long long *occ_base, unsigned long long pos_base, long long ngo, long long ngi,
              const ExpandLateArgs late)
{
    typedef typename std::conditional<sizeof(SE) == 4, uint16_t, uint32_t>::type CE;
    constexpr bool LATE = CM != 0;
    extern __shared__ __align__(16) unsigned char esm[];
    unsigned long long *s_off = reinterpret_cast<unsigned long long *>(esm);  // seg_tiles + 1
    uint32_t *s_ent = reinterpret_cast<uint32_t *>(s_off + seg_tiles + 1);
    __shared__ unsigned long long s_red[kExpandThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kExpandThreads / 32;
    const long long seg = blockIdx.x;
    const long long t0 = seg * seg_tiles;
    const long long nt = max(0LL, min(seg_tiles, nsub - t0));
    if (nt == 0 && !LATE) return;

    // base of the segment: sum of the earlier segments
    unsigned long long part = 0;
    for (long long q = tid; q < seg; q += kExpandThreads) part += seg_sum[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    // a chunk of a longer scan writes after the keys of the chunks before it
    unsigned long long seg_base = occ_base ? *occ_base : 0ull;
#pragma unroll
    for (int w = 0; w < NW; ++w) seg_base += s_red[w];
    __syncthreads();

    // per-tile offsets: each thread scans a run of consecutive tiles
    const long long per = (nt + kExpandThreads - 1) / kExpandThreads;
    const long long r0 = min(nt, (long long)tid * per), r1 = min(nt, r0 + per);
    unsigned long long mine = 0;
    for (long long q = r0; q < r1; ++q) {
        const uint32_t o = tile_out[t0 + q];
        s_ent[q] = min(tile_ent[t0 + q], uint32_t(kWarpTile));
        s_off[q] = o;  // the tile's own total, replaced by its offset below
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
    if (tid == kExpandThreads - 1 && nt > 0 && t0 + nt == nsub) *n_occ = (long long)run;  // the last tile's CTA
    // small group tables move to shared memory (GS): their loads sit on a
    // row's critical path
    uint32_t *s_grp = s_ent + seg_tiles;
    if (GS) {
        for (long long i = tid; i < ngo; i += kExpandThreads) s_grp[i] = grp_off[i];
        for (long long i = tid; i < ngi; i += kExpandThreads) s_grp[ngo + i] = grp_ids[i];
    }
    const uint32_t *s_go = s_grp, *s_gid = s_grp + ngo;
    auto grp_first = [&](uint32_t g) -> uint32_t { return GS ? s_go[g] : __ldg(grp_off + g); };
    auto grp_id = [&](uint32_t j) -> uint32_t { return GS ? s_gid[j] : __ldg(grp_ids + j); };
    // late ids: canon, match bitmap, ranks and per-terminal counters (in
    // shared memory for CM 1, 2)
    const CE *canon_g = static_cast<const CE *>(late.canon);
    const CE *rank_g = static_cast<const CE *>(late.rank);
    unsigned char *lq = reinterpret_cast<unsigned char *>(s_grp + (GS ? ngo + ngi : 0));
    CE *s_canon = reinterpret_cast<CE *>(lq);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(lq + r16(late.nterms * (long long)sizeof(CE)));
    CE *s_rank = reinterpret_cast<CE *>(reinterpret_cast<unsigned char *>(s_mask) + r16(late.nwords * 4));
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(s_rank) +
                                                   r16((late.nwords + 1) * (long long)sizeof(CE)));
    if (CM == 1 || CM == 2) {
        const long long words = CM == 2 ? (late.nterms + 1) / 2 : late.nterms;
        for (long long i = tid; i < late.nterms; i += kExpandThreads) s_canon[i] = canon_g[i];
        for (long long i = tid; i < late.nwords; i += kExpandThreads) s_mask[i] = late.mask[i];
        for (long long i = tid; i <= late.nwords; i += kExpandThreads) s_rank[i] = rank_g[i];
        for (long long i = tid; i < words; i += kExpandThreads) s_cnt[i] = 0u;
    }
    // terminal id of match-entry offset o: its rank among the bitmap's set bits
    auto terminal_of = [&](uint32_t o) -> uint32_t {
        const uint32_t w = o >> 5;
        const uint32_t mw = CM == 3 ? __ldg(late.mask + w) : s_mask[w];
        const uint32_t rw = uint32_t(CM == 3 ? __ldg(rank_g + w) : s_rank[w]);
        return rw + __popc(mw & ((1u << (o & 31u)) - 1u));
    };
    __syncthreads();

    const unsigned long long cap = (unsigned long long)occ_cap;
    constexpr int R = 10;  // rows of 32 entries loaded together; lane l takes entry 32 u + l of a row
    constexpr uint32_t kMask = (uint32_t)((((SE)1) << kOffShift) - 1);
    // The warp's work items are (tile q, first entry g0) in order; the slot
    // loads of the next item are in flight while the current one is written.
    auto load = [&](SE (&x)[R], long long qq, uint32_t gg) {
        const uint32_t ent = s_ent[qq];
        const SE *src = slots + (t0 + qq) * kWarpTile;
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const uint32_t j = gg + u * 32 + lane;
            x[u] = j < ent ? __ldcs(src + j) : (SE)0;
        }
    };
    long long q = warp;
    while (q < nt && s_ent[q] == 0) q += NW;
    uint32_t g0 = 0;
    SE v[R];
    if (q < nt) load(v, q, 0);
    // keys of the current tile go to out[0 .. room): 32-bit offsets from the
    // tile's base, clipped to the capacity left after it
    unsigned long long *out = occ;
    uint32_t room = 0, pos = 0;
    auto enter = [&](long long qq) {
        const unsigned long long b = s_off[qq];
        out = occ + b;
        room = b < cap ? uint32_t(min(cap - b, 0xFFFFFFFFull)) : 0u;
        pos = 0;
    };
    if (q < nt) enter(q);
    const uint32_t lt = (1u << lane) - 1u;
    while (q < nt) {
        const uint32_t ent = s_ent[q];
        long long qn = q;
        uint32_t gn = g0 + R * 32;
        if (gn >= ent) {
            gn = 0;
            qn += NW;
            while (qn < nt && s_ent[qn] == 0) qn += NW;
        }
        SE w[R];
        if (qn < nt) {
            load(w, qn, gn);
        } else {
#pragma unroll
            for (int u = 0; u < R; ++u) w[u] = (SE)0;
        }
        const uint32_t tile0 = uint32_t(pos_base + (unsigned long long)(t0 + q) * kWarpTile);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const uint32_t row = g0 + u * 32;
            if (row >= ent) break;
            const uint32_t cnt = min(ent - row, 32u);
            const bool valid = uint32_t(lane) < cnt;   // the valid lanes are 0 .. cnt-1
            uint32_t code = uint32_t(v[u] & kMask);
            if (LATE && valid) {  // a match entry: count its terminal, take its pattern code
                code = terminal_of(code);
                if (CM == 3) {
                    atomicAdd(&late.ccount[code], 1ull);
                    code = uint32_t(__ldg(canon_g + code));
                } else {
                    if (CM == 1) {
                        atomicAdd(&s_cnt[code], 1u);
                    } else {
                        // 16-bit halves: the add that takes a half to 0x8000 moves
                        // 0x8000 to the workspace counter, so a half never wraps
                        const uint32_t sh = (code & 1u) << 4;
                        const uint32_t old = atomicAdd(&s_cnt[code >> 1], 1u << sh);
                        if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
                            atomicSub(&s_cnt[code >> 1], 0x8000u << sh);
                            atomicAdd(&late.ccount[code], 0x8000ull);
                        }
                    }
                    code = uint32_t(s_canon[code]);
                }
            }
            const unsigned long long key_hi = (unsigned long long)(tile0 + uint32_t(v[u] >> kOffShift)) << 32;
            const bool grp = valid && (code & kGrp);
            if (!__any_sync(kFull, grp)) {
                // one key per entry: consecutive lanes write consecutive keys
                const uint32_t o = pos + lane;
                if (valid && o < room) out[o] = key_hi | code;
                pos += cnt;
                continue;
            }
            // a row naming a group of equal patterns: exclusive prefix over
            // the multiplicities (from ballots while every group adds at most 3)
            uint32_t lo = code, mult = valid ? 1u : 0u;
            if (grp) {
                const uint32_t g = code & ~kGrp;
                lo = grp_first(g);
                mult = grp_first(g + 1) - lo;
            }
            const uint32_t extra = grp ? mult - 1u : 0u;
            uint32_t excl, tot;
            bool pairs = false;  // every group in the row is a pair
            if (__all_sync(kFull, extra < 4u)) {
                const uint32_t e0 = __ballot_sync(kFull, extra & 1u);
                const uint32_t e1 = __ballot_sync(kFull, extra & 2u);
                pairs = e1 == 0u;
                excl = uint32_t(lane) + __popc(e0 & lt) + 2u * __popc(e1 & lt);
                tot = cnt + __popc(e0) + 2u * __popc(e1);
            } else {
                const uint32_t incl = dev::warp_incl_scan(mult, lane);
                excl = incl - mult;
                tot = __shfl_sync(kFull, incl, 31);
            }
            const uint32_t o0 = pos + excl;
            if (pairs) {
                // the first key of every entry, then the second of each pair
                if (valid && o0 < room) out[o0] = key_hi | (grp ? grp_id(lo) : code);
                if (extra && o0 + 1u < room) out[o0 + 1u] = key_hi | grp_id(lo + 1u);
            } else {
                for (uint32_t k = 0; k < mult; ++k) {
                    const uint32_t id = grp ? grp_id(lo + k) : code;
                    if (o0 + k < room) out[o0 + k] = key_hi | id;
                }
            }
            pos += tot;
        }
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = w[u];
        if (qn != q && qn < nt) enter(qn);
        q = qn;
        g0 = gn;
    }
    if (!LATE) return;

    // ---- late ids: counters -> workspace; the last CTA writes counts[r] ----
    __syncthreads();
    if (CM == 1 || CM == 2)
        for (long long c = tid; c < late.nterms; c += kExpandThreads) {
            const uint32_t v = CM == 2 ? (s_cnt[c >> 1] >> ((c & 1) << 4)) & 0xFFFFu : s_cnt[c];
            if (v) atomicAdd(&late.ccount[c], (unsigned long long)v);
        }
    __threadfence();
    __syncthreads();
    __shared__ int s_last;
    if (tid == 0) s_last = atomicAdd(&late.ws->done_expand, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const CE *cg = static_cast<const CE *>(late.canon);
    for (long long c = tid; c < late.nterms; c += kExpandThreads) {
        const unsigned long long n = dev::ld_acquire(&late.ccount[c]);
        const uint32_t code = cg[c];
        if (code & kGrp) {
            const uint32_t g = code & ~kGrp;
            for (uint32_t j = grp_off[g]; j < grp_off[g + 1]; ++j) late.counts[grp_ids[j]] = (long long)n;
        } else {
            late.counts[code] = (long long)n;
        }
    }
}

// ---------------------------------------------------------------------------
// PFAC scan: one walk per start position along goto edges only (Lin et al.'s
// failure-less Aho-Corasick; the table is the merged one with every
// non-goto entry 0). A warp takes its warp tile (staged like the DFA scan)
// in 80 rounds of 32 consecutive positions, lane l walking position
// 32 r + l from the root over at most m bytes; a walk that reaches depth m
// is a match, one that meets a dead entry or a byte outside the alphabet
// stops. A round's matches are compacted by ballot in position order into
// the tile's slot, so the expand kernel of the DFA scan finishes the list.
// ---------------------------------------------------------------------------
template <typename E, bool DNA, bool HYB>
__global__ void __launch_bounds__(768, 1) pfac_scan_kernel(const AcArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr uint32_t kGrp = sizeof(E) == 2 ? 0x8000u : 0x80000000u;
    typedef typename std::conditional<sizeof(E) == 2, uint32_t, unsigned long long>::type SE;
    constexpr int kOffShift = sizeof(E) == 2 ? 16 : 32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int hv = a.m - 1 <= 16 ? 1 : a.m - 1 <= 32 ? 2 : 4;
    const int BUF = kWarpTile + 16 * hv;

    // ---- shared memory carve-up (the same as the DFA scan's) ----------------
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
    const long long hist_words = a.hist_smem == 2 ? (a.nterms + 1) / 2 : a.nterms;
    p += a.hist_smem ? r16(hist_words * 4) : 0;
    uint8_t *s_cls = p;
    p += DNA ? 0 : 256;
    p += warp * ac_warp_bytes(hv, a.pool_cap, sizeof(E));
    uint64_t *bar = reinterpret_cast<uint64_t *>(p);
    uint8_t *buf = p + 16;

    {
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
        for (int i = threadIdx.x; i < hist_words; i += blockDim.x) s_hist[i] = 0u;
    if (!DNA)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) s_cls[i] = a.cls_g[i];
    if (lane == 0) dev::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dev::fence_proxy_async_smem();
    __syncthreads();

    const TableRef<E, HYB> tab{s_tab, reinterpret_cast<const E *>(a.table_g), uint32_t(a.smem_entries)};
    const int m = a.m;
    auto count_terminal = [&](uint32_t c) {
        if (a.hist_smem == 1) {
            atomicAdd(&s_hist[c], 1u);
        } else if (a.hist_smem == 2) {
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
    auto mult_of = [&](uint32_t code) -> uint32_t {
        if (!(code & kGrp)) return 1u;
        const uint32_t g = code & ~kGrp;
        return __ldg(a.grp_off + g + 1) - __ldg(a.grp_off + g);
    };

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
            failed = true;
            break;
        }
        inflight = false;
        phase ^= 1u;
        const long long tile0 = st * kWarpTile;
        const int got_bytes = stage_bytes(a, st, BUF);
        if (got_bytes < BUF) {
            for (int b = got_bytes + lane; b < BUF; b += 32) {
                const long long g = tile0 + b;
                buf[b] = g < a.n ? a.text[g] : uint8_t(a.pad);
            }
        }
        __syncwarp();
        SE *dst = slots + st * kWarpTile;
        uint32_t ent = 0, outs = 0;
        for (int r = 0; r < kChunk; ++r) {
            const int q = r * 32 + lane;  // start offset in the tile
            bool hit = false;
            uint32_t hidx = 0;
            if (tile0 + q + m <= a.n) {
                uint32_t e = 2u;  // root (row 1)
                for (int j = 0; j < m; ++j) {
                    const uint32_t b = buf[q + j];
                    uint32_t c;
                    if (DNA) {
                        c = ((b >> 1) ^ (b >> 2)) & 3u;
                        if (((a.lut >> (8 * c)) & 0xFFu) != b) break;
                    } else {
                        c = s_cls[b];
                        if (c == 0xFFu) break;
                    }
                    const uint32_t idx = ((e >> 1) << a.lw) | c;
                    e = tab(idx);
                    if (e & 1u) { hit = true; hidx = idx; break; }
                    if (e == 0u) break;
                }
            }
            const uint32_t bal = __ballot_sync(kFull, hit);
            if (hit) {
                const uint32_t c = ids.terminal(hidx - a.mid_base);
                const uint32_t code = ids.code(c);
                count_terminal(c);
                outs += mult_of(code);
                if (a.list) dst[ent + __popc(bal & ((1u << lane) - 1u))] = ((SE)q << kOffShift) | (SE)code;
            }
            ent += __popc(bal);
        }
        // the buffer is free: stage this warp's next tile
        dev::fence_proxy_async_smem();
        __syncwarp();
        if (st + G < a.nsub) {
            if (lane == 0) stage_issue(a, st + G, buf, bar, BUF);
            inflight = true;
        }
        if (!a.list) {
            my_total += outs;
            continue;
        }
        uint32_t o_tot = outs;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) o_tot += __shfl_xor_sync(kFull, o_tot, o);
        if (lane == 31) {
            a.tile_ent[st] = ent;
            a.tile_out[st] = o_tot;
            if (o_tot) atomicAdd(&a.seg_sum[st / a.seg_tiles], (unsigned long long)o_tot);
        }
    }
    if (inflight) (void)dev::mbar_wait_bounded(bar, phase);

    if (!a.list) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_total += __shfl_down_sync(kFull, my_total, o);
        if (lane == 0 && my_total)
            atomicAdd(reinterpret_cast<unsigned long long *>(a.n_occ), my_total);
    }
    __syncthreads();
    if (s_hist) {
        for (int c = threadIdx.x; c < a.nterms; c += blockDim.x) {
            const uint32_t v = a.hist_smem == 2 ? (s_hist[c >> 1] >> ((c & 1) << 4)) & 0xFFFFu : s_hist[c];
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


// variant ids: dna u16 smem (0-2), dna u16 hybrid (3-5), dna u16 smem with
// index entries (6-8), dna u16 hybrid with index entries (9-11), dna u32
// hybrid with index entries (12-14), general u32 hybrid (15-17), then the
// late-ids forms of the five ACGT groups (18-32); within each group HV = 1,
// 2, 4.
const Variant kVariants[] = {
    {ac_scan_kernel<uint16_t, 6, 1, true, false, false, false, 512>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, false, false, 512>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, false, false, 512>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, false, false, 512>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, false, false, 512>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, false, false, 512>, 2, 4, true, true},
    {ac_scan_kernel<uint16_t, 6, 1, true, false, true, false, 512>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, true, false, 512>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, true, false, 512>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, true, false, 512>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, true, false, 512>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, true, false, 512>, 2, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, true, true, true, false, 512>, 4, 1, true, true},
    {ac_scan_kernel<uint32_t, 7, 2, true, true, true, false, 512>, 4, 2, true, true},
    {ac_scan_kernel<uint32_t, 9, 4, true, true, true, false, 512>, 4, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, false, true, false, false, 512>, 4, 1, false, true},
    {ac_scan_kernel<uint32_t, 7, 2, false, true, false, false, 512>, 4, 2, false, true},
    {ac_scan_kernel<uint32_t, 9, 4, false, true, false, false, 512>, 4, 4, false, true},

    {ac_scan_kernel<uint16_t, 6, 1, true, false, false, true, 512>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, false, true, 512>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, false, true, 512>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, false, true, 512>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, false, true, 512>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, false, true, 512>, 2, 4, true, true},
    {ac_scan_kernel<uint16_t, 6, 1, true, false, true, true, 512>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, true, true, 512>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, true, true, 512>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, true, true, 512>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, true, true, 512>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, true, true, 512>, 2, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, true, true, true, true, 512>, 4, 1, true, true},
    {ac_scan_kernel<uint32_t, 7, 2, true, true, true, true, 512>, 4, 2, true, true},
    {ac_scan_kernel<uint32_t, 9, 4, true, true, true, true, 512>, 4, 4, true, true},
};

constexpr int kWideWarps = 24;   // warps per CTA of the 768-thread instances
constexpr int kWideBase = 100;   // variant ids from here index kWideVariants


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
    int warps, hist, ids;
    int lst;  // the list-mode layout of late ids (multiplicities per match entry only)
};

long long ac_hist_bytes(int hist, long long nterms)
{
    return hist == 1 ? r16(nterms * 4) : hist == 2 ? r16((nterms + 1) / 2 * 4) : 0;
}

long long ac_smem_bytes(const AcTables &t, int eb, const Layout &L, int hv, int pool_cap)
{
    const int nwords = int(t.flag_mask.size());
    const int nterms = int(t.canon.size());
    const long long ids = L.ids == 1 ? ac_ids_bytes(nwords, nterms, eb)
                        : L.ids == 2 ? (L.lst ? ac_emul_bytes(nwords) : ac_ids_late_bytes(nwords, nterms, eb))
                                     : 0;
    return r16(L.smem_entries * eb) + ids + ac_hist_bytes(L.hist, nterms) + (t.dna ? 0 : 256) +
           (long long)L.warps * ac_warp_bytes(hv, pool_cap, eb);
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
    // more than 16 warps: the 768-thread kernels of ACGT tables (one CTA per
    // SM); the PFAC kernel is one of them
    const bool wide_ok = t.dna && (opt.ctas_per_sm <= 1);
    const int max_w = wide_ok ? kWideWarps : 16;
    const int forced_warps = opt.warps_per_cta > 0 ? std::min(opt.warps_per_cta, max_w) : 0;
    dev.pool_cap = pool_cap;
    dev.hv = hv;
    dev.nv = 5 + hv;
    dev.ctas_per_sm = opt.ctas_per_sm > 0 ? opt.ctas_per_sm : 1;
    // pm_params.counters: 0 auto, 1 32-bit shared, 2 16-bit shared, 3 global;
    // pm_params.ids_place: 0 auto, 1 shared, 2 global, 3 late (Layout::ids
    // 1, 0 and 2)
    auto hist_ok = [&](int h) {
        return opt.counters == 0 || (opt.counters == 3 ? h == 0 : h == opt.counters);
    };
    auto ids_ok = [&](int i) {
        if (i == 2 && (t.goto_only || !t.dna)) return false;
        if (opt.ids_place == 0) return true;
        return i == (opt.ids_place == 1 ? 1 : opt.ids_place == 2 ? 0 : 2);
    };
    auto fits = [&](const Layout &L) {
        const long long need = ac_smem_bytes(t, eb, L, hv, pool_cap);
        return need <= budget &&
               need * dev.ctas_per_sm + 1024LL * dev.ctas_per_sm <= (long long)dp.smem_per_sm;
    };

    Layout best{0, 0, 0, 0};
    Layout list_layout{0, 0, 0, 0};
    bool chosen = false;
    if ((place == PM_PLACE_AUTO || place == PM_PLACE_SMEM) &&
        (opt.smem_table_bytes <= 0 || entries * eb <= opt.smem_table_bytes)) {
        // whole table in shared memory; prefer the id structure and the
        // counters there too (32-bit, else 16-bit), then late ids (whose
        // list mode keeps only the multiplicities there; counts mode adds
        // the counters that still fit), then the most warps (at least 12 if
        // possible; PFAC, whose walks hide latency only by having more of
        // them in flight, the most warps first); pm_params can pin either
        // choice
        const int ids_hist[7][2] = {{1, 1}, {1, 2}, {2, -1}, {0, 1}, {0, 2}, {1, 0}, {0, 0}};
        // A first pass (unless the warps are pinned) wants at least 20
        // warps with the whole id structure and 32-bit counters, else late
        // ids: a 768-thread kernel pays for its 80-register cap only from
        // about 20 warps on (d=8000, m=8: 17 warps with everything shared
        // ran 562 GB/s in list mode, late ids at 24 warps 784).
        const int first_minw = forced_warps ? 0 : t.goto_only ? max_w : 20;
        for (int minw : {first_minw, 12, 4}) {
            if (minw == 0) continue;
            for (int o = 0; o < 7 && !chosen; ++o) {
                const int ids = ids_hist[o][0], hist = ids_hist[o][1];
                if (!ids_ok(ids) || (hist >= 0 && !hist_ok(hist))) continue;
                if (minw == first_minw && !t.goto_only && o != 0 && o != 2) continue;
                const int hi = forced_warps ? forced_warps : max_w;
                const int lo = forced_warps ? forced_warps : minw;
                for (int w = hi; w >= lo && !chosen; --w) {
                    Layout L{entries, w, hist < 0 ? 0 : hist, ids, hist < 0 ? 1 : 0};
                    if (!fits(L)) continue;
                    Layout C = L;
                    if (hist < 0) {
                        // counts mode (id structure in shared memory): the
                        // most warps (down to lo) that still hold shared
                        // counters, else device counters
                        bool any = false;
                        for (int wc = w; wc >= lo && !any; --wc)
                            for (int h : {1, 2}) {
                                Layout D{entries, wc, h, ids, 0};
                                if (hist_ok(h) && fits(D)) { C = D; any = true; break; }
                            }
                        for (int wc = w; wc >= lo && !any && hist_ok(0); --wc) {
                            Layout D{entries, wc, 0, ids, 0};
                            if (fits(D)) { C = D; any = true; }
                        }
                        if (!any) continue;
                    }
                    best = C;
                    list_layout = L;
                    chosen = true;
                }
            }
            if (chosen) break;
        }
        if (!chosen && place == PM_PLACE_SMEM) return PM_ETOOBIG;
        if (chosen) dev.placement = PM_PLACE_SMEM;
    }
    if (!chosen) {
        // hybrid / global: breadth-first prefix of rows in shared memory;
        // 16 warps, or 24 for PFAC, whose walks hide latency only by
        // having more of them in flight
        const int w = forced_warps ? forced_warps : (t.goto_only && wide_ok) ? kWideWarps : 16;
        // counters / ids only when pinned by pm_params (the table prefix
        // gets the room otherwise)
        Layout L{0, w, opt.counters == 1 ? 1 : opt.counters == 2 ? 2 : 0,
                 opt.ids_place == 1 ? 1 : (opt.ids_place == 3 && ids_ok(2)) ? 2 : 0, 0};
        Layout LL = L;  // list mode: late ids keep no counters and only the multiplicities
        if (L.ids == 2) { LL.hist = 0; LL.lst = 1; }
        const long long fixed = std::max(ac_smem_bytes(t, eb, L, hv, pool_cap), ac_smem_bytes(t, eb, LL, hv, pool_cap));
        if (fixed > budget) return PM_ETOOBIG;
        long long room = budget - fixed;
        if (dev.ctas_per_sm > 1)
            room = std::min(room, (long long)dp.smem_per_sm / dev.ctas_per_sm - 1024 - fixed);
        if (opt.smem_table_bytes > 0) room = std::min<long long>(room, opt.smem_table_bytes);
        if (place == PM_PLACE_GLOBAL) room = 0;
        long long se = room > 0 ? room / eb : 0;
        se &= ~((long long)(16 / eb) - 1);   // whole 16-byte vectors
        if (se > entries) se = entries;
        L.smem_entries = se;
        LL.smem_entries = se;
        best = L;
        list_layout = LL;
        dev.placement = place == PM_PLACE_GLOBAL ? PM_PLACE_GLOBAL : PM_PLACE_HYBRID;
    }
    dev.warps = best.warps;
    dev.hist_smem = best.hist;
    dev.ids_smem = best.ids;
    dev.smem_entries = best.smem_entries;
    const bool hyb = dev.smem_entries < entries || !t.dna || eb == 4;
    // ACGT tables whose entries fit as next-row indices: u32, or u16 with
    // fewer than 2^14 rows
    dev.pre = t.dna && (eb == 4 || t.n_rows <= (1 << 14)) ? 1 : 0;
    int group;
    if (!t.dna) group = 5;
    else if (eb == 4) group = 4;
    else group = (hyb ? 1 : 0) + (dev.pre ? 2 : 0);
    if (best.ids == 2) group += 6;   // late ids (ACGT groups only)
    // variant ids >= kWideBase index kWideVariants: ACGT groups 0-4 and
    // their late-ids forms 6-10 are wide groups 0-9
    auto variant_for = [&](int warps) {
        if (warps <= 16) return group * 3 + hv_slot(hv);
        const int wg = group >= 6 ? group - 1 : group;
        return kWideBase + wg * 3 + hv_slot(hv);
    };
    dev.variant = variant_for(best.warps);
    dev.smem_bytes = ac_smem_bytes(t, eb, best, hv, pool_cap);
    if (list_layout.warps == 0) list_layout = best;
    dev.warps_list = list_layout.warps;
    dev.variant_list = variant_for(list_layout.warps);
    dev.smem_bytes_list = ac_smem_bytes(t, eb, list_layout, hv, pool_cap);
    dev.max_warps = (long long)dp.sm_count * dev.ctas_per_sm * std::max(dev.warps, dev.warps_list);
    return PM_OK;
}

namespace {

int slot_entry_bytes(const AcTables &t) { return (t.dna ? t.entry_bytes : 4) == 2 ? 4 : 8; }

// Enqueue a whole scan on `st` with workspace `d_ws` (laid out by ac_ws_layout).
AcKernel pfac_kernel_for(const AcTables &t, const DevAc &dv)
{
    const bool hyb = dv.smem_entries < ((long long)t.n_rows << t.lw);
    const int eb = t.dna ? t.entry_bytes : 4;
    if (!t.dna) return hyb ? pfac_scan_kernel<uint32_t, false, true> : pfac_scan_kernel<uint32_t, false, false>;
    if (eb == 2) return hyb ? pfac_scan_kernel<uint16_t, true, true> : pfac_scan_kernel<uint16_t, true, false>;
    return hyb ? pfac_scan_kernel<uint32_t, true, true> : pfac_scan_kernel<uint32_t, true, false>;
}

// first: this scan starts a result (counts, totals and per-terminal counters
// start at zero); later chunks of a longer scan keep adding to them, write
// their keys after occ_base keys and shift positions by pos_base.
int ac_enqueue(const AcTables &t, const DevAc &dv, const uint8_t *d_text, int64_t n, bool list,
               int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
               cudaStream_t st, bool pfac = false, bool first = true,
               const unsigned long long *occ_base = nullptr, unsigned long long pos_base = 0)
{
    cudaError_t e;
    const long long nsub = warp_tiles(n);
    const long long nterms = (long long)t.canon.size();
    const int se = slot_entry_bytes(t);
    DeviceProps dp;
    int rc = device_props(dp);
    if (rc) return rc;
    const AcWsLayout L = ac_ws_layout(nsub, list, nterms, se, dp.sm_count);
    // every segment non-empty: at most ac_segments() of them
    const long long seg_tiles = (nsub + ac_segments(nsub, dp.sm_count) - 1) / ac_segments(nsub, dp.sm_count);
    if (first) {
        e = cudaMemsetAsync(d_counts, 0, size_t(t.d) * sizeof(int64_t), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_n_occ, 0, sizeof(int64_t), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_ws, 0, size_t(L.zeroed), st);
    } else {
        // keep the status word and the per-terminal counters
        static_assert(offsetof(dev::WsHeader, done_expand) == offsetof(dev::WsHeader, done_ctas) + 4,
                      "done counters side by side");
        e = cudaMemsetAsync(static_cast<char *>(d_ws) + offsetof(dev::WsHeader, done_ctas), 0, 8, st);
        if (e == cudaSuccess && L.zeroed > L.seg_sum)
            e = cudaMemsetAsync(static_cast<char *>(d_ws) + L.seg_sum, 0, size_t(L.zeroed - L.seg_sum), st);
    }
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (n < t.m || nsub == 0) {
        // nothing to scan in this piece: the key total stays that of the pieces before
        if (list && occ_base && !first) e = cudaMemcpyAsync(d_n_occ, occ_base, 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        return PM_OK;
    }

    // list mode has its own layout (with late ids: no counters, maybe more warps)
    const bool late = list && !pfac && dv.ids_smem == 2;
    const int var = list ? dv.variant_list : dv.variant;
    const int warps = list ? dv.warps_list : dv.warps;
    const AcKernel fn = pfac ? pfac_kernel_for(t, dv)
                             : var >= kWideBase ? (list ? kWideVariants : kWideCountsVariants)[var - kWideBase].fn
                                                : kVariants[var].fn;
    const long long smem = list ? dv.smem_bytes_list : dv.smem_bytes;
    rc = kernel_smem_attr(reinterpret_cast<const void *>(fn), smem);
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
    a.tmul_g = dv.tmul;
    a.emul_g = dv.emul;
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
    a.nsub = nsub;
    a.pool_cap = dv.pool_cap;
    a.list = list ? 1 : 0;
    a.hist_smem = late ? 0 : dv.hist_smem;
    a.ids_smem = dv.ids_smem;
    a.late = late ? 1 : 0;
    a.d = int(t.d);
    a.counts = reinterpret_cast<long long *>(d_counts);
    a.n_occ = reinterpret_cast<long long *>(d_n_occ);
    char *w = static_cast<char *>(d_ws);
    a.ws = reinterpret_cast<dev::WsHeader *>(w);
    a.ccount = reinterpret_cast<unsigned long long *>(w + kWsHeader);
    a.tile_ent = reinterpret_cast<uint32_t *>(w + L.tile_ent);
    a.tile_out = reinterpret_cast<uint32_t *>(w + L.tile_out);
    a.seg_sum = reinterpret_cast<unsigned long long *>(w + L.seg_sum);
    a.seg_tiles = seg_tiles;
    a.slots = w + L.slots;

    const int threads = warps * 32;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, size_t(smem));
    if (e != cudaSuccess || per_sm < 1) { set_cuda_error(int(e)); return PM_ECUDA; }
    long long grid = (long long)dp.sm_count * std::min(per_sm, dv.ctas_per_sm);
    const long long want = (nsub + warps - 1) / warps;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    fn<<<dim3(unsigned(grid)), dim3(unsigned(threads)), size_t(smem), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (!list) return PM_OK;

    ExpandLate xl;
    if (late) {
        xl.canon = dv.canon;
        xl.mask = dv.flag_mask;
        xl.rank = dv.flag_rank;
        xl.nterms = nterms;
        xl.nwords = (int64_t)t.flag_mask.size();
        xl.counts = d_counts;
    }
    return expand_launch(d_ws, nsub, nterms, se, dv.grp_off, dv.grp_ids, (int64_t)t.grp_off.size(),
                         (int64_t)t.grp_ids.size(), d_occ, occ_cap, d_n_occ, occ_base, pos_base, st,
                         late ? &xl : nullptr);
}

}  // namespace

int64_t list_workspace_bytes(int64_t nsub, bool list, int64_t nterms, int slot_entry_bytes)
{
    DeviceProps dp;
    if (device_props(dp)) dp.sm_count = 1024;  // an upper bound on the segments
    return ac_ws_layout(nsub, list, nterms, slot_entry_bytes, dp.sm_count).total;
}

void list_workspace_parts(void *d_ws, int64_t nsub, int64_t nterms, int slot_entry_bytes, ListParts &out)
{
    DeviceProps dp;
    if (device_props(dp)) dp.sm_count = 1;
    const AcWsLayout L = ac_ws_layout(nsub, true, nterms, slot_entry_bytes, dp.sm_count);
    char *w = static_cast<char *>(d_ws);
    out.zeroed_bytes = L.zeroed;
    out.seg_sum = reinterpret_cast<unsigned long long *>(w + L.seg_sum);
    out.tile_ent = reinterpret_cast<uint32_t *>(w + L.tile_ent);
    out.tile_out = reinterpret_cast<uint32_t *>(w + L.tile_out);
    out.slots = w + L.slots;
    const long long segs = ac_segments(nsub, dp.sm_count);
    out.seg_tiles = (nsub + segs - 1) / segs;
}

int expand_launch(void *d_ws, int64_t nsub, int64_t nterms, int slot_entry_bytes, const uint32_t *grp_off,
                  const uint32_t *grp_ids, int64_t n_grp_off, int64_t n_grp_ids, uint64_t *d_occ,
                  int64_t occ_cap, int64_t *d_n_occ, const unsigned long long *occ_base,
                  unsigned long long pos_base, void *stream, const ExpandLate *late)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ListParts P;
    list_workspace_parts(d_ws, nsub, nterms, slot_entry_bytes, P);
    const long long seg_tiles = P.seg_tiles;
    const long long nseg = (nsub + seg_tiles - 1) / seg_tiles;
    // shared memory of the expand kernel: 12 bytes per tile of a segment
    // (above 48 KB only for texts of more than about 3 GB), then, while two
    // CTAs still fit an SM: with late ids canon, the match bitmap and its
    // ranks and 32-bit (else 16-bit) per-terminal counters, and the group
    // tables (offsets and ids)
    unsigned long long *occ = reinterpret_cast<unsigned long long *>(d_occ);
    const long long cap = d_occ ? occ_cap : 0;
    DeviceProps dp;
    int rc = device_props(dp);
    if (rc) return rc;
    const long long per_cta = std::min<long long>((long long)dp.smem_per_sm / 2 - 2048, dp.smem_optin - 1024);
    long long esmem = (seg_tiles + 1) * 8 + seg_tiles * 4;
    const bool se4 = slot_entry_bytes == 4;
    ExpandLateArgs la{};
    const bool is_late = late && late->canon;
    if (is_late) {
        la.canon = late->canon;
        la.mask = late->mask;
        la.rank = late->rank;
        la.nterms = late->nterms;
        la.nwords = late->nwords;
        la.ccount = reinterpret_cast<unsigned long long *>(static_cast<char *>(d_ws) + kWsHeader);
        la.counts = reinterpret_cast<long long *>(late->counts);
        la.ws = static_cast<dev::WsHeader *>(d_ws);
        const int ceb = se4 ? 2 : 4;
        const long long cb = r16(late->nterms * ceb) + r16(late->nwords * 4) + r16((late->nwords + 1) * ceb);
        const long long x32 = cb + r16(late->nterms * 4), x16 = cb + r16((late->nterms + 1) / 2 * 4);
        la.smem = esmem + x32 <= per_cta ? 1 : esmem + x16 <= per_cta ? 2 : 0;
        esmem += la.smem == 1 ? x32 : la.smem == 2 ? x16 : 0;
    }
    const long long grp_bytes = (n_grp_off + n_grp_ids) * 4;
    const bool grp_smem = n_grp_off > 0 && (grp_bytes <= (16 << 10) || esmem + grp_bytes <= per_cta);
    const long long ngo = grp_smem ? n_grp_off : 0, ngi = grp_smem ? n_grp_ids : 0;
    esmem += (ngo + ngi) * 4;
    long long *n_occ = reinterpret_cast<long long *>(d_n_occ);
    auto go = [&](auto kern, const auto *slots) -> cudaError_t {
        if (esmem > (48 << 10)) {
            const cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(esmem));
            if (ea != cudaSuccess) return ea;
        }
        kern<<<unsigned(nseg), kExpandThreads, size_t(esmem), st>>>(slots, P.tile_ent, P.tile_out, P.seg_sum, nseg,
                                                                   seg_tiles, nsub, grp_off, grp_ids, occ, cap, n_occ,
                                                                   occ_base, pos_base, ngo, ngi, la);
        return cudaGetLastError();
    };
    const int cm = !is_late ? 0 : la.smem == 1 ? 1 : la.smem == 2 ? 2 : 3;
    // one instance per slot width, counter mode and group-table placement
    auto pick = [&](auto se_tag) -> cudaError_t {
        typedef decltype(se_tag) SE;
        constexpr int sh = sizeof(SE) == 4 ? 16 : 32;
        constexpr uint32_t grp = sizeof(SE) == 4 ? 0x8000u : 0x80000000u;
        const SE *sl = static_cast<const SE *>(P.slots);
        switch (cm * 2 + (grp_smem ? 1 : 0)) {
            case 0: return go(expand_kernel<SE, sh, grp, 0, false>, sl);
            case 1: return go(expand_kernel<SE, sh, grp, 0, true>, sl);
            case 2: return go(expand_kernel<SE, sh, grp, 1, false>, sl);
            case 3: return go(expand_kernel<SE, sh, grp, 1, true>, sl);
            case 4: return go(expand_kernel<SE, sh, grp, 2, false>, sl);
            case 5: return go(expand_kernel<SE, sh, grp, 2, true>, sl);
            case 6: return go(expand_kernel<SE, sh, grp, 3, false>, sl);
            default: return go(expand_kernel<SE, sh, grp, 3, true>, sl);
        }
    };
    const cudaError_t e = se4 ? pick(uint32_t(0)) : pick(0ull);
    if (e != cudaSuccess) { set_cuda_error(int(e)); cudaGetLastError(); return PM_ECUDA; }
    return PM_OK;
}

int64_t ac_workspace_bytes(const AcTables &t, int64_t n, bool list)
{
    DeviceProps dp;
    if (device_props(dp)) dp.sm_count = 1024;  // an upper bound on the segments
    return ac_ws_layout(warp_tiles(n), list, (long long)t.canon.size(), slot_entry_bytes(t), dp.sm_count).total;
}

int ac_launch(const AcTables &t, const DevAc &dv, const uint8_t *d_text, int64_t n, bool list,
              int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
              void *stream)
{
    return ac_enqueue(t, dv, d_text, n, list, d_counts, d_occ, occ_cap, d_n_occ, d_ws,
                      static_cast<cudaStream_t>(stream));
}

int ac_launch_piece(const AcTables &t, const DevAc &dv, bool pfac, const uint8_t *d_text, int64_t n,
                    bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ,
                    void *d_ws, void *stream, bool first, const unsigned long long *occ_base,
                    unsigned long long pos_base)
{
    return ac_enqueue(t, dv, d_text, n, list, d_counts, d_occ, occ_cap, d_n_occ, d_ws,
                      static_cast<cudaStream_t>(stream), pfac, first, occ_base, pos_base);
}

int pfac_launch(const AcTables &t, const DevAc &dv, const uint8_t *d_text, int64_t n, bool list,
                int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
                void *stream)
{
    return ac_enqueue(t, dv, d_text, n, list, d_counts, d_occ, occ_cap, d_n_occ, d_ws,
                      static_cast<cudaStream_t>(stream), true);
}

// ---------------------------------------------------------------------------
// Allocation-free scan (pm_scan_device_noalloc).
//
// Some callers cannot allocate device memory when they scan: a host
// application that owns the GPU allocator (a plugin must not add cudaMalloc
// calls it cannot account for), or a latency-bound loop that reserved all
// of its memory up front and must not call cudaMalloc, which can block on
// the device and fail once memory is fragmented. For them the workspace of
// the Aho-Corasick scan lives in one fixed array inside the library. The
// array is reserved on every GPU that loads the library and stays reserved
// until the process exits. Every call uses the same array and it keeps the
// last call's contents, so the launcher clears what must start at zero, and
// two calls whose work overlaps on the GPU (different streams, or host
// threads) race on it. List mode needs 4 or 8 bytes of the array per text
// byte (one slot entry per start position), so list-mode texts are limited
// to a few MiB.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
// Device address of the scratch array on the current device. Host code
// cannot use the array's name as an address; the lookup allocates nothing
// and is repeated on every call, so it stays right after a device reset
// (which may move the array when the module loads again).
int noalloc_scratch(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_cuda_error(int(e));
        cudaGetLastError();
        return e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ? PM_ENODEV : PM_ECUDA;
    }
    *out = p;
    return PM_OK;
}
}  // namespace

int64_t ac_noalloc_limit_bytes() { return int64_t(kNoAllocScratchBytes); }

int ac_launch_noalloc(const AcTables &t, const DevAc &dv, const uint8_t *d_text, int64_t n,
                      bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap,
                      int64_t *d_n_occ, void *stream)
{
    if (ac_workspace_bytes(t, n, list) > (int64_t)kNoAllocScratchBytes) return PM_ETOOBIG;
    void *ws = nullptr;
    const int rc = noalloc_scratch(&ws);
    if (rc) return rc;
    return ac_enqueue(t, dv, d_text, n, list, d_counts, d_occ, occ_cap, d_n_occ, ws,
                      static_cast<cudaStream_t>(stream));
}

int ac_noalloc_status(void *stream)
{
    void *ws = nullptr;
    const int rc = noalloc_scratch(&ws);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, ws, sizeof(status), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        return PM_ECUDA;
    }
    return status ? PM_ETIMEOUT : PM_OK;
}

}  // namespace pm
