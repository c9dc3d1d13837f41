// scan_wm.cu -- Wu-Manber block scan on sm_103a (Section 3.2, Algorithm 5,
// parallelised as in Section 4.2.1 / Algorithms 7 and 9).
//
// Same warp-tile decomposition as the Aho-Corasick kernel: lane l owns the
// windows that start in [tile + 80 l, tile + 80 l + 80), i.e. window ends
// from its chunk start + m - 1 on, and runs Algorithm 5 over them: hash the
// B-byte block ending at the window end, jump by SHIFT when it is non-zero,
// else hash the B'-byte window prefix, take the run of HASH[h] whose PREFIX
// equals it and verify its candidates. Equal patterns enter the tables once
// (a group code), so a window matches at most one candidate and the walk
// stops at the first. ACGT-like sets with m <= 32 walk the lane's text from
// registers with the exact 2-bit codes as h1 / h2 (the next tile's copy is
// in flight meanwhile); other sets read the staged tile byte by byte. Matches
// go through the lane's pool into the tile's slot, and the expand kernel of
// the Aho-Corasick scan writes the sorted keys (list mode).
#include <type_traits>

#include "scan_common.cuh"

namespace pm {
namespace {

using dev::kFull;

struct WmArgs {
    const uint8_t *text;
    long long n;
    int aligned;
    const uint8_t *shift_g;
    int hbits;
    const uint32_t *hoff;
    const uint32_t *hids;
    const uint32_t *hcode;
    const uint16_t *hpfx;
    const uint8_t *pats;
    const long long *poff;        // mixed lengths: pattern r is pats[poff[r] .. poff[r+1])
    int m, B, Bp;                 // mixed lengths: m is the shortest length
    int mbuf;                     // length that sizes the staged halo (the longest)
    long long ntiles;
    int pool_cap, buf;
    int list, hist_smem, d;
    long long *counts;
    long long *n_occ;
    dev::WsHeader *ws;
    const uint32_t *grp_off;      // groups of equal patterns (kWmGroup codes)
    const uint32_t *grp_ids;
    uint32_t *tile_ent;           // list: entries per warp tile
    uint32_t *tile_out;           // list: keys per warp tile (groups expanded)
    unsigned long long *seg_sum;  // list: keys per segment of seg_tiles warp tiles
    long long seg_tiles;
    void *slots;                  // list: slot_stride entries per warp tile
    long long slot_stride;
    int se4;                      // 4-byte entries, else 8
    // exact-code tables (ACGT-like sets, m <= 32)
    uint32_t lut;
    const uint8_t *shift2_g;
    const uint32_t *dir_g;
    const unsigned long long *ccode;
    const uint32_t *cr;
    const unsigned long long *fcode;  // mixed lengths: whole packed pattern of each candidate
    const uint8_t *flen;              // and its length
    int nkey;                     // 4^(B + B')
};

__host__ __device__ constexpr int r16w(long long x) { return int((x + 15) & ~15LL); }

__host__ __device__ inline int wm_buf_bytes(int m) { return kWarpTile + r16w(m - 1 > 0 ? m - 1 : 0); }

// register text of the exact-code walk: chunk + halo in 16-byte vectors
__host__ __device__ inline int wm_nv(int m) { return m - 1 <= 16 ? 6 : 7; }

// staged bytes per warp tile: the windows' bytes, and for the exact-code
// walk every byte the last lane loads into registers
__host__ __device__ inline int wm_tile_buf(int m, bool dna)
{
    const int b = wm_buf_bytes(m), r = (kLane - 1) * kChunk + 16 * wm_nv(m);
    return dna && r > b ? r : b;
}

__host__ __device__ inline int wm_warp_bytes(int m, int pool_cap, bool dna)
{
    return 16 + r16w(wm_tile_buf(m, dna)) + r16w((long long)pool_cap * 32 * 4);
}

__device__ __forceinline__ uint32_t block_hash(const uint8_t *s, int len)
{
    uint32_t h = 0;
    for (int k = 0; k < len; ++k) h = (h << 5) | (s[k] & 31u);
    return h;
}

__device__ __forceinline__ int wm_stage_bytes(const WmArgs &a, long long t)
{
    if (!a.aligned) return 0;
    const long long avail = (a.n & ~15LL) - t * kWarpTile;
    if (avail <= 0) return 0;
    return avail >= a.buf ? a.buf : int(avail);
}

__device__ __forceinline__ void wm_stage_issue(const WmArgs &a, long long t, uint8_t *buf,
                                               uint64_t *bar)
{
    const int bytes = wm_stage_bytes(a, t);
    dev::mbar_arrive_expect_tx(bar, uint32_t(bytes));
    if (bytes > 0) dev::tma_load_1d(buf, a.text + t * kWarpTile, uint32_t(bytes), bar);
}

// Algorithm 5 over one lane's windows; hit(start_offset, code) per match,
// in ascending start (at most one distinct pattern matches a window).
template <bool SHIFT_SMEM, class F>
__device__ __forceinline__ void wm_walk(const WmArgs &a, const uint8_t *s_shift,
                                        const uint8_t *w, int lim, F &&hit)
{
    const int m = a.m, B = a.B, Bp = a.Bp;
    int i = m - 1;
    while (i < lim) {
        const uint32_t h = block_hash(w + i - B + 1, B);
        const uint32_t sh = SHIFT_SMEM ? uint32_t(s_shift[h]) : uint32_t(__ldg(a.shift_g + h));
        if (sh > 0) {
            i += int(sh);
            continue;
        }
        const uint8_t *win = w + i - m + 1;
        const uint16_t hp = uint16_t(block_hash(win, Bp));
        uint32_t lo = __ldg(a.hoff + h);
        const uint32_t end = __ldg(a.hoff + h + 1);
        uint32_t hi = end;
        while (lo < hi) {  // first entry with PREFIX >= h'
            const uint32_t md = (lo + hi) >> 1;
            if (__ldg(a.hpfx + md) < hp) lo = md + 1;
            else hi = md;
        }
        for (uint32_t k = lo; k < end && __ldg(a.hpfx + k) == hp; ++k) {
            const uint8_t *pp = a.pats + (size_t)__ldg(a.hids + k) * m;
            int j = 0;
            while (j < m && __ldg(pp + j) == win[j]) ++j;
            if (j == m) {
                hit(i - (m - 1), __ldg(a.hcode + k));
                break;
            }
        }
        ++i;
    }
}

// Algorithm 5 over the windows of the shortest length m of a mixed-length
// set; a candidate (the HASH run with the window's PREFIX, in ascending r)
// matches when its whole pattern, of its own length, equals the text from
// the window start (avail bytes of text from the lane's chunk start).
// hit(start_offset, r) in ascending (start, r).
template <bool SHIFT_SMEM, class F>
__device__ __forceinline__ void wmv_walk(const WmArgs &a, const uint8_t *s_shift, const uint8_t *w,
                                         int lim, long long avail, F &&hit)
{
    const int m = a.m, B = a.B, Bp = a.Bp;
    int i = m - 1;
    while (i < lim) {
        const uint32_t h = block_hash(w + i - B + 1, B);
        const uint32_t sh = SHIFT_SMEM ? uint32_t(s_shift[h]) : uint32_t(__ldg(a.shift_g + h));
        if (sh > 0) {
            i += int(sh);
            continue;
        }
        const int start = i - (m - 1);
        const uint8_t *win = w + start;
        const uint16_t hp = uint16_t(block_hash(win, Bp));
        uint32_t lo = __ldg(a.hoff + h);
        const uint32_t end = __ldg(a.hoff + h + 1);
        uint32_t hi = end;
        while (lo < hi) {  // first entry with PREFIX >= h'
            const uint32_t md = (lo + hi) >> 1;
            if (__ldg(a.hpfx + md) < hp) lo = md + 1;
            else hi = md;
        }
        for (uint32_t k = lo; k < end && __ldg(a.hpfx + k) == hp; ++k) {
            const uint32_t r = __ldg(a.hids + k);
            const long long p0 = __ldg(a.poff + r);
            const int len = int(__ldg(a.poff + r + 1) - p0);
            if (start + len > avail) continue;
            const uint8_t *pp = a.pats + p0;
            int j = 0;
            while (j < len && __ldg(pp + j) == win[j]) ++j;
            if (j == len) hit(start, r);
        }
        ++i;
    }
}

// Algorithm 5 over the windows of the shortest length m of a mixed-length
// ACGT-like set, with the exact-code tables, over the staged bytes: the
// rolling code of the window's m characters picks the candidates of its
// (block, prefix) run with the same code (the run is sorted by (code, r));
// a longer candidate extends that code with the next len - m bytes and
// compares it with its whole packed pattern. hit(start_offset, r) in
// ascending (start, r).
template <class F>
__device__ __forceinline__ void wmv_walk_dna(const WmArgs &a, const uint8_t *s_shift2, const uint2 *s_run,
                                             const uint8_t *w, int lim, long long avail, F &&hit)
{
    const int m = a.m, B = a.B, Bp = a.Bp;
    const unsigned long long mask = m >= 32 ? ~0ull : ((1ull << (2 * m)) - 1ull);
    const uint32_t bmask = (1u << (2 * B)) - 1u;
    const int pshift = 2 * (m - Bp);
    auto cls = [](uint32_t b) { return ((b >> 1) ^ (b >> 2)) & 3u; };
    auto ok = [&](uint32_t b) { return ((a.lut >> (8 * cls(b))) & 0xFFu) == b; };
    unsigned long long code = 0;
    int bad = -1;       // last offset holding a byte outside the alphabet
    int next = m - 1;   // next window end to examine
    for (int i = 0; i < lim; ++i) {
        const uint32_t b = w[i];
        if (!ok(b)) bad = i;
        code = ((code << 2) | cls(b)) & mask;
        if (i < next) continue;
        const uint32_t blk = uint32_t(code) & bmask;
        uint32_t sh = s_shift2[blk];
        if (bad > i - B) sh = uint32_t(m - B + 1);
        if (sh > 0) {
            next = i + int(sh);
            continue;
        }
        next = i + 1;
        if (bad > i - m) continue;
        const uint2 run = s_run[(blk << (2 * Bp)) | uint32_t(code >> pshift)];
        const int start = i - (m - 1);
        // four candidates per step; the run is sorted, so it stops at the
        // first code above the window's
        for (uint32_t k0 = run.x; k0 < run.y; k0 += 4) {
            unsigned long long cc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) cc[u] = k0 + u < run.y ? __ldg(a.ccode + k0 + u) : 0ull;
            bool stop = false;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t k = k0 + u;
                const bool in = k < run.y;
                stop |= in && cc[u] > code;
                if (!in || cc[u] != code) continue;
                const int len = __ldg(a.flen + k);
                if (start + len > avail) continue;
                unsigned long long ext = code;
                bool good = true;
                for (int j = i + 1; j < start + len && good; ++j) {
                    const uint32_t bj = w[j];
                    good = ok(bj);
                    ext = (ext << 2) | cls(bj);
                }
                if (good && ext == __ldg(a.fcode + k)) hit(start, __ldg(a.cr + k));
            }
            if (stop) break;
        }
    }
}

// Algorithm 5 over one lane's windows on an ACGT-like set, with h1 and h2
// the exact 2-bit codes of the block and the prefix, over the lane's bytes
// held in registers (NV vectors: chunk + halo). The lane keeps the packed
// code of its last m characters (first character in the high bits), the
// offset of its last byte outside the alphabet and the next window end
// Algorithm 5 examines; the window ends visited are the same as with the
// byte hash (a block holding a byte outside the alphabet occurs in no
// pattern: SHIFT m-B+1). A run of candidates is sorted by packed code, so
// its scan stops at the first code not below the window's. Bytes past the
// text are 0, outside every ACGT-like alphabet.
template <int NV, bool WIDE, class F>
__device__ __forceinline__ void wm_walk_dna(const WmArgs &a, const uint8_t *s_shift2,
                                            const uint2 *s_run, const uint4 (&tv)[NV], F &&hit)
{
    // packed codes: 32 bits for m <= 16, else 64
    typedef typename std::conditional<WIDE, unsigned long long, uint32_t>::type CT;
    const int m = a.m, B = a.B, Bp = a.Bp;
    const CT mask = m >= int(4 * sizeof(CT)) ? ~CT(0) : CT((CT(1) << (2 * m)) - 1);
    const uint32_t bmask = (1u << (2 * B)) - 1u;
    const int pshift = 2 * (m - Bp);
    const int lim = kChunk + m - 1;   // window ends at offsets < lim
    CT code = 0;
    int bad = -1;                     // last offset holding a byte outside the alphabet
    int next = m - 1;                 // next window end to examine
    // one 16-byte vector per iteration (a rolled loop keeps the code small;
    // the vector is picked from the registers by predicated moves)
#pragma unroll 1
    for (int v = 0; v < NV && v * 16 < lim; ++v) {
        uint4 tx = tv[0];
#pragma unroll
        for (int u = 1; u < NV; ++u)
            if (v == u) tx = tv[u];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t w = q == 0 ? tx.x : q == 1 ? tx.y : q == 2 ? tx.z : tx.w;
            const uint32_t a4 = ((w >> 1) ^ (w >> 2)) & 0x03030303u;
            const uint32_t sel = __byte_perm(a4 | (a4 >> 4), 0u, 0x4420);
            const uint32_t x = w ^ __byte_perm(a.lut, 0u, sel);  // zero byte = in the alphabet
            const uint32_t y = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = v * 16 + q * 4 + k;
                if (i < lim) {
                    code = ((code << 2) | CT((a4 >> (8 * k)) & 3u)) & mask;
                    if (!((y >> (8 * k + 7)) & 1u)) bad = i;
                    if (i >= next) {
                        const uint32_t blk = uint32_t(code) & bmask;
                        uint32_t sh = s_shift2[blk];
                        if (bad > i - B) sh = uint32_t(m - B + 1);
                        if (sh > 0) {
                            next = i + int(sh);
                        } else {
                            next = i + 1;
                            if (bad <= i - m) {
                                // the run of (block, prefix), sorted by packed code:
                                // stop at the first code not below the window's
                                const uint2 run = s_run[(blk << (2 * Bp)) | uint32_t(code >> pshift)];
                                for (uint32_t k0 = run.x; k0 < run.y; k0 += 4) {
                                    CT cc[4];
#pragma unroll
                                    for (int u = 0; u < 4; ++u) cc[u] = k0 + u < run.y ? CT(__ldg(a.ccode + k0 + u)) : CT(0);
                                    bool stop = false;
                                    int hu = -1;
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        const bool ok = k0 + u < run.y;
                                        stop |= ok && cc[u] >= code;
                                        if (ok && cc[u] == code) hu = u;
                                    }
                                    if (hu >= 0) hit(i - (m - 1), __ldg(a.cr + k0 + hu));
                                    if (stop) break;
                                }
                            }
                        }
                    }
                }
            }
        }
    }
}

// MAXT: launch bound, 512 threads, or 768 for exact-code plans of more than
// 16 warps (up to 85 registers)
template <bool SHIFT_SMEM, bool DNA, int NV, bool WIDE, bool VAR, int MAXT = 512>
__global__ void __launch_bounds__(MAXT, 1) wm_scan_kernel(const WmArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *p = smem;
    uint8_t *s_shift = p;
    p += (SHIFT_SMEM && !DNA) ? r16w(1LL << a.hbits) : 0;
    uint8_t *s_shift2 = p;
    p += DNA ? r16w(1LL << (2 * a.B)) : 0;
    uint2 *s_run = reinterpret_cast<uint2 *>(p);   // (first, end) of each run
    p += DNA ? r16w((long long)a.nkey * 8) : 0;
    uint32_t *s_hist = a.hist_smem ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += a.hist_smem ? r16w((long long)a.d * 4) : 0;
    p += warp * wm_warp_bytes(a.mbuf, a.pool_cap, DNA);
    uint64_t *bar = reinterpret_cast<uint64_t *>(p);
    uint8_t *buf = p + 16;
    uint32_t *pool = reinterpret_cast<uint32_t *>(buf + r16w(a.buf));

    if (DNA) {
        for (int i = threadIdx.x; i < (1 << (2 * a.B)); i += blockDim.x) s_shift2[i] = a.shift2_g[i];
        for (int i = threadIdx.x; i < a.nkey; i += blockDim.x) s_run[i] = make_uint2(a.dir_g[i], a.dir_g[i + 1]);
    } else if (SHIFT_SMEM) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.shift_g);
        uint4 *dst = reinterpret_cast<uint4 *>(s_shift);
        const int nvec = int(((1LL << a.hbits) + 15) / 16);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = src[i];
    }
    if (s_hist)
        for (int i = threadIdx.x; i < a.d; i += blockDim.x) s_hist[i] = 0u;
    if (lane == 0) dev::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dev::fence_proxy_async_smem();
    __syncthreads();

    uint32_t *pl = pool + lane;
    const uint32_t cap = uint32_t(a.pool_cap);
    const int m = a.m;
    const long long G = (long long)gridDim.x * (blockDim.x >> 5);
    const long long gwarp = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    uint32_t phase = 0;
    bool inflight = false;
    unsigned long long my_total = 0;
    if (gwarp < a.ntiles) {
        if (lane == 0) wm_stage_issue(a, gwarp, buf, bar);
        inflight = true;
    }

    // a match code counts every id it stands for; returns how many
    auto count_code = [&](uint32_t code) -> uint32_t {
        if (!(code & kWmGroup)) {
            dev::count_pattern(code, s_hist, a.counts);
            return 1u;
        }
        const uint32_t g = code & ~kWmGroup;
        const uint32_t j1 = __ldg(a.grp_off + g + 1);
        uint32_t c = 0;
        for (uint32_t j = __ldg(a.grp_off + g); j < j1; ++j, ++c) dev::count_pattern(__ldg(a.grp_ids + j), s_hist, a.counts);
        return c;
    };

    for (long long t = gwarp; t < a.ntiles; t += G) {
        const bool got = __all_sync(kFull, dev::mbar_wait_bounded(bar, phase));
        if (!got) {
            if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutTma);
            break;  // the copy stays in flight: waited for below
        }
        inflight = false;
        phase ^= 1u;
        const long long tile0 = t * kWarpTile;
        const int got_bytes = wm_stage_bytes(a, t);
        if (got_bytes < a.buf) {
            for (int b = got_bytes + lane; b < a.buf; b += 32) {
                const long long g = tile0 + b;
                buf[b] = g < a.n ? a.text[g] : uint8_t(0);
            }
        }
        __syncwarp();

        const int cs = lane * kChunk;
        int lim = kChunk + m - 1;  // window ends at offsets < lim
        {
            const long long left = a.n - (tile0 + cs);
            if (left < lim) lim = left <= 0 ? 0 : int(left);
        }
        uint32_t nh = 0;
        auto rec = [&](int off, uint32_t code) {
            if (nh < cap) pl[nh * 32] = (uint32_t(off) << 24) | code;
            ++nh;
        };
        uint4 tv[DNA ? NV : 1];
        if (DNA && !VAR) {
            const uint4 *bv = reinterpret_cast<const uint4 *>(buf + cs);
#pragma unroll
            for (int v = 0; v < (DNA ? NV : 1); ++v) tv[v] = bv[v];
            // the buffer is free: stage the next tile while this one is walked
            dev::fence_proxy_async_smem();
            __syncwarp();
            if (t + G < a.ntiles) {
                if (lane == 0) wm_stage_issue(a, t + G, buf, bar);
                inflight = true;
            }
            wm_walk_dna<(DNA ? NV : 1), WIDE>(a, s_shift2, s_run, tv, rec);
        } else if (VAR && DNA) {
            wmv_walk_dna(a, s_shift2, s_run, buf + cs, lim, a.n - (tile0 + cs), rec);
        } else if (VAR) {
            wmv_walk<SHIFT_SMEM>(a, s_shift, buf + cs, lim, a.n - (tile0 + cs), rec);
        } else {
            wm_walk<SHIFT_SMEM>(a, s_shift, buf + cs, lim, rec);
        }
        const bool ovf = nh > cap;

        // slot of this tile (list mode): the lane's entries follow the
        // entries of the lanes before it
        long long first = 0;
        uint32_t e_incl = 0;
        if (a.list) {
            e_incl = dev::warp_incl_scan(nh, lane);
            first = t * a.slot_stride + (e_incl - nh);
        }
        // slot entry: (start offset in the tile << 16) | code with group flag
        // 2^15 (4-byte entries), or << 32 with group flag 2^31
        auto put = [&](uint32_t k, int off, uint32_t code) {
            if (VAR) {  // (start << 20) | r or (start << 32) | r: no groups
                if (a.se4)
                    static_cast<uint32_t *>(a.slots)[first + k] = (uint32_t(cs + off) << 20) | code;
                else
                    static_cast<unsigned long long *>(a.slots)[first + k] =
                        ((unsigned long long)(cs + off) << 32) | code;
                return;
            }
            const bool grp = (code & kWmGroup) != 0;
            const uint32_t c = code & ~kWmGroup;
            if (a.se4)
                static_cast<uint32_t *>(a.slots)[first + k] = (uint32_t(cs + off) << 16) | (grp ? 0x8000u : 0u) | c;
            else
                static_cast<unsigned long long *>(a.slots)[first + k] =
                    ((unsigned long long)(cs + off) << 32) | (grp ? 0x80000000u : 0u) | c;
        };
        uint32_t cnt = 0;  // keys of this lane (groups expanded)
        if (!ovf) {
            for (uint32_t k = 0; k < nh; ++k) {
                const uint32_t v = pl[k * 32];
                cnt += count_code(v & 0xFFFFFFu);
                if (a.list) put(k, int(v >> 24), v & 0xFFFFFFu);
            }
        } else {
            // the pool overflowed: walk again and take the matches as they come
            uint32_t k = 0;
            auto again = [&](int off, uint32_t code) {
                cnt += count_code(code);
                if (a.list && k < nh) put(k, off, code);
                ++k;
            };
            if (DNA && !VAR) {
                // the staged copy may already hold the next tile: text from global memory
                uint4 tw[DNA ? NV : 1];
                uint8_t *tb = reinterpret_cast<uint8_t *>(tw);
                const long long g0 = tile0 + cs;
                for (int b = 0; b < 16 * (DNA ? NV : 1); ++b) tb[b] = g0 + b < a.n ? a.text[g0 + b] : uint8_t(0);
                wm_walk_dna<(DNA ? NV : 1), WIDE>(a, s_shift2, s_run, tw, again);
            } else if (VAR && DNA) {
                wmv_walk_dna(a, s_shift2, s_run, buf + cs, lim, a.n - (tile0 + cs), again);
            } else if (VAR) {
                wmv_walk<SHIFT_SMEM>(a, s_shift, buf + cs, lim, a.n - (tile0 + cs), again);
            } else {
                wm_walk<SHIFT_SMEM>(a, s_shift, buf + cs, lim, again);
            }
        }
        if (!a.list) {
            my_total += cnt;
        } else {
            uint32_t o_tot = cnt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) o_tot += __shfl_xor_sync(kFull, o_tot, o);
            if (lane == 31) {
                a.tile_ent[t] = e_incl;
                a.tile_out[t] = o_tot;
                if (o_tot) atomicAdd(&a.seg_sum[t / a.seg_tiles], (unsigned long long)o_tot);
            }
        }

        if (!DNA || VAR) {
            // the buffer is free: stage the next tile
            dev::fence_proxy_async_smem();
            __syncwarp();
            if (t + G < a.ntiles) {
                if (lane == 0) wm_stage_issue(a, t + G, buf, bar);
                inflight = true;
            }
        }
    }

    // a copy still in flight after an error exit: wait for it (bounded) so
    // it is not still writing this CTA's shared memory when the CTA exits
    if (inflight) (void)dev::mbar_wait_bounded(bar, phase);

    if (!a.list) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_total += __shfl_down_sync(kFull, my_total, o);
        if (lane == 0 && my_total)
            atomicAdd(reinterpret_cast<unsigned long long *>(a.n_occ), my_total);
    }
    __syncthreads();
    if (s_hist) {
        for (int r = threadIdx.x; r < a.d; r += blockDim.x) {
            const uint32_t c = s_hist[r];
            if (c) atomicAdd(reinterpret_cast<unsigned long long *>(a.counts) + r, (unsigned long long)c);
        }
    }
}

long long wm_smem_bytes(int hbits, bool shift_smem, int hist, int d, int warps, int m,
                        int pool_cap, bool dna, int B, int nkey)
{
    const long long tables = dna ? r16w(1LL << (2 * B)) + r16w((long long)nkey * 8)
                                 : (shift_smem ? r16w(1LL << hbits) : 0);
    return tables + (hist ? r16w((long long)d * 4) : 0) + (long long)warps * wm_warp_bytes(m, pool_cap, dna);
}

}  // namespace

int wm_plan(const WmTables &t, const pm_params &opt, const DeviceProps &dp, DevWm &dev)
{
    const long long budget = (long long)dp.smem_optin - 1024;
    const int hbits = 5 * t.B;
    dev.pool_cap = 40;
    dev.ctas_per_sm = opt.ctas_per_sm > 0 ? opt.ctas_per_sm : 1;
    // more than 16 warps only in the 768-thread exact-code kernels (ACGT sets)
    const int forced = opt.warps_per_cta > 0 ? std::min(opt.warps_per_cta, t.dna ? 24 : 16) : 0;
    const bool shift_smem = hbits <= 15;
    const int choices[3] = {16, 12, 8};
    for (int pass = 0; pass < 2; ++pass) {
        for (int wi = 0; wi < 3; ++wi) {
            const int w = forced ? forced : choices[wi];
            const int hist = pass == 0 ? 1 : 0;
            const long long need = wm_smem_bytes(hbits, shift_smem, hist, int(t.d), w, t.var ? t.m_max : t.m,
                                                 dev.pool_cap, t.dna, t.B, 1 << (2 * (t.B + t.Bp)));
            if (need <= budget) {
                dev.warps = w;
                dev.hist_smem = hist;
                dev.shift_smem = shift_smem;
                dev.dna = t.dna ? 1 : 0;
                dev.smem_bytes = need;
                return PM_OK;
            }
            if (forced) break;
        }
    }
    return PM_ETOOBIG;
}

// slot entry bytes: 4 when every code (pattern id, or group | 2^15) fits 16 bits
int wm_slot_bytes(const WmTables &t)
{
    const int64_t groups = t.grp_off.empty() ? 0 : int64_t(t.grp_off.size()) - 1;
    return t.d < 32768 && groups < 32768 ? 4 : 8;
}

// mixed lengths: 4-byte (start << 20) | r entries for d <= 2^20, K per position
static int wmv_slot_bytes(const WmTables &t) { return t.d <= (1 << 20) ? 4 : 8; }

int64_t wm_workspace_bytes(const WmTables &t, int64_t n, bool list)
{
    if (t.var) return list_workspace_bytes(warp_tiles(n), list, 0, wmv_slot_bytes(t) * t.K);
    return list_workspace_bytes(warp_tiles(n), list, 0, wm_slot_bytes(t));
}

int wm_launch(const WmTables &t, const DevWm &dv, const uint8_t *d_text, int64_t n, bool list,
              int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
              void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const long long ntiles = warp_tiles(n);
    const int se = t.var ? wmv_slot_bytes(t) : wm_slot_bytes(t);
    const int per_pos = t.var ? t.K : 1;
    ListParts L;
    list_workspace_parts(d_ws, ntiles, 0, se * per_pos, L);
    const int64_t zeroed = list ? L.zeroed_bytes : kWsHeader;
    e = cudaMemsetAsync(d_counts, 0, size_t(t.d) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_n_occ, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ws, 0, size_t(zeroed), st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (n < t.m || ntiles == 0) return PM_OK;

    typedef void (*K)(const WmArgs);
    const int nv = wm_nv(t.m);
    const bool wide = t.m > 16;
    K fn;
    const bool big = dv.warps > 16;   // exact-code kernels with a 768-thread bound
    if (t.var && dv.dna) {
        fn = big ? wm_scan_kernel<false, true, 1, false, true, 768> : wm_scan_kernel<false, true, 1, false, true>;
    } else if (t.var) {
        fn = dv.shift_smem ? wm_scan_kernel<true, false, 1, false, true> : wm_scan_kernel<false, false, 1, false, true>;
    } else if (dv.dna && big) {
        fn = nv == 6 ? (wide ? wm_scan_kernel<false, true, 6, true, false, 768> : wm_scan_kernel<false, true, 6, false, false, 768>)
                     : wm_scan_kernel<false, true, 7, true, false, 768>;
    } else if (dv.dna) {
        fn = nv == 6 ? (wide ? wm_scan_kernel<false, true, 6, true, false> : wm_scan_kernel<false, true, 6, false, false>)
                     : wm_scan_kernel<false, true, 7, true, false>;
    } else {
        fn = dv.shift_smem ? wm_scan_kernel<true, false, 1, false, false> : wm_scan_kernel<false, false, 1, false, false>;
    }
    int rc = kernel_smem_attr(reinterpret_cast<const void *>(fn), dv.smem_bytes);
    if (rc) return rc;
    DeviceProps dp;
    rc = device_props(dp);
    if (rc) return rc;

    WmArgs a;
    a.text = d_text;
    a.n = n;
    a.aligned = (reinterpret_cast<uintptr_t>(d_text) & 15) == 0;
    a.shift_g = dv.shift;
    a.hbits = 5 * t.B;
    a.hoff = dv.hoff;
    a.hids = dv.hids;
    a.hcode = dv.hcode;
    a.hpfx = dv.hpfx;
    a.pats = dv.pats;
    a.poff = reinterpret_cast<const long long *>(dv.poff);
    a.m = t.m;
    a.mbuf = t.var ? t.m_max : t.m;
    a.B = t.B;
    a.Bp = t.Bp;
    a.ntiles = ntiles;
    a.pool_cap = dv.pool_cap;
    a.buf = wm_tile_buf(a.mbuf, dv.dna != 0);
    a.list = list ? 1 : 0;
    a.hist_smem = dv.hist_smem;
    a.d = int(t.d);
    a.counts = reinterpret_cast<long long *>(d_counts);
    a.n_occ = reinterpret_cast<long long *>(d_n_occ);
    a.ws = reinterpret_cast<dev::WsHeader *>(d_ws);
    a.grp_off = dv.grp_off;
    a.grp_ids = dv.grp_ids;
    a.tile_ent = L.tile_ent;
    a.tile_out = L.tile_out;
    a.seg_sum = L.seg_sum;
    a.seg_tiles = L.seg_tiles;
    a.slots = L.slots;
    a.slot_stride = (long long)kWarpTile * per_pos;
    a.se4 = se == 4 ? 1 : 0;
    a.lut = t.lut;
    a.shift2_g = dv.shift2;
    a.dir_g = dv.dir;
    a.ccode = reinterpret_cast<const unsigned long long *>(dv.ccode);
    a.cr = dv.cr;
    a.fcode = reinterpret_cast<const unsigned long long *>(dv.fcode);
    a.flen = dv.flen;
    a.nkey = t.dna ? (1 << (2 * (t.B + t.Bp))) : 0;

    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, dv.warps * 32, size_t(dv.smem_bytes));
    if (e != cudaSuccess || per_sm < 1) { set_cuda_error(int(e)); return PM_ECUDA; }
    long long grid = (long long)dp.sm_count * std::min(per_sm, dv.ctas_per_sm);
    const long long want = (ntiles + dv.warps - 1) / dv.warps;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    fn<<<dim3(unsigned(grid)), dim3(unsigned(dv.warps * 32)), size_t(dv.smem_bytes), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (!list) return PM_OK;
    if (t.var) return sorted_expand_launch(d_ws, ntiles, se, per_pos, d_occ, occ_cap, d_n_occ, stream);
    return expand_launch(d_ws, ntiles, 0, se, dv.grp_off, dv.grp_ids, (int64_t)t.grp_off.size(),
                         (int64_t)t.grp_ids.size(), d_occ, occ_cap, d_n_occ, nullptr, 0, stream);
}

}  // namespace pm
