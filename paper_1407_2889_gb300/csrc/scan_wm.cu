// scan_wm.cu -- Wu-Manber block scan on sm_103a (Section 3.2, Algorithm 5,
// parallelised as in Section 4.2.1 / Algorithms 7 and 9).
//
// Same warp-tile decomposition as the Aho-Corasick kernel: lane l owns the
// windows that start in [tile + 80 l, tile + 80 l + 80), i.e. window ends
// from its chunk start + m - 1 on, and runs Algorithm 5 over them: hash the
// B-byte block ending at the window end, jump by SHIFT when it is non-zero,
// else hash the B'-byte window prefix, take the run of HASH[h] whose PREFIX
// equals it (buckets are sorted by PREFIX, so a binary search finds it) and
// verify each candidate byte by byte. SHIFT lives in shared memory when it
// has at most 2^15 entries (B <= 3); HASH, PREFIX and the patterns are read
// through L1/L2. Matches go through the same pool / warp scan / look-back /
// staged-store path as the Aho-Corasick kernel.
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
    const uint16_t *hpfx;
    const uint8_t *pats;
    int m, B, Bp;
    long long ntiles;
    int pool_cap, stage_cap, buf;
    int list, hist_smem, d;
    long long *counts;
    unsigned long long *occ;
    long long occ_cap;
    long long *n_occ;
    dev::WsHeader *ws;
    dev::LookbackRefs lb;
    // exact-code tables (ACGT-like sets, m <= 32)
    uint32_t lut;
    const uint8_t *shift2_g;
    const uint32_t *dir_g;
    const unsigned long long *ccode;
    const uint32_t *cr;
    int nkey;                     // 4^(B + B')
};

__host__ __device__ constexpr int r16w(long long x) { return int((x + 15) & ~15LL); }

__host__ __device__ inline int wm_buf_bytes(int m) { return kWarpTile + r16w(m - 1 > 0 ? m - 1 : 0); }

__host__ __device__ inline int wm_warp_bytes(int m, int pool_cap, int stage_cap)
{
    return 16 + r16w(wm_buf_bytes(m)) + r16w((long long)pool_cap * 32 * 4) + stage_cap * 8;
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

// Algorithm 5 over one lane's windows; hit(start_offset, r) per match, in
// ascending (start, r).
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
            const uint32_t r = __ldg(a.hids + k);
            const uint8_t *pp = a.pats + (size_t)r * m;
            int j = 0;
            while (j < m && __ldg(pp + j) == win[j]) ++j;
            if (j == m) hit(i - (m - 1), r);
        }
        ++i;
    }
}

// Algorithm 5 over one lane's windows on an ACGT-like set, with h1 and h2
// the exact 2-bit codes of the block and the prefix. The lane keeps the
// packed code of its last m characters (first character in the high bits)
// and the offset of its last byte outside the alphabet; the window ends
// Algorithm 5 visits are the same as with the byte hash (a block holding a
// byte outside the alphabet occurs in no pattern: SHIFT m-B+1), and each
// candidate of the (block, prefix) run is verified by one comparison of
// packed codes (equal patterns are adjacent in the run, in ascending r).
template <class F>
__device__ __forceinline__ void wm_walk_dna(const WmArgs &a, const uint8_t *s_shift2,
                                            const uint32_t *s_dir, const uint8_t *w, int lim, F &&hit)
{
    const int m = a.m, B = a.B, Bp = a.Bp;
    const unsigned long long mask = m >= 32 ? ~0ull : ((1ull << (2 * m)) - 1ull);
    const uint32_t bmask = (1u << (2 * B)) - 1u;
    const int pshift = 2 * (m - Bp);
    unsigned long long code = 0;
    int bad = -1;   // last offset holding a byte outside the alphabet
    int skip = 0;   // window ends still to pass over after a SHIFT > 1
    for (int i = 0; i < lim; ++i) {
        const uint32_t b = w[i];
        const uint32_t c = ((b >> 1) ^ (b >> 2)) & 3u;
        if (((a.lut >> (8 * c)) & 0xFFu) != b) bad = i;
        code = ((code << 2) | c) & mask;
        if (i < m - 1) continue;
        if (skip > 0) { --skip; continue; }
        const uint32_t sh = bad > i - B ? uint32_t(m - B + 1) : uint32_t(s_shift2[uint32_t(code) & bmask]);
        if (sh > 0) { skip = int(sh) - 1; continue; }
        if (bad > i - m) continue;  // the window holds a byte no pattern has
        const uint32_t key = ((uint32_t(code) & bmask) << (2 * Bp)) | uint32_t(code >> pshift);
        const uint32_t lo = s_dir[key], hi = s_dir[key + 1];
        for (uint32_t k0 = lo; k0 < hi; k0 += 4) {
            unsigned long long cc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) cc[u] = k0 + u < hi ? __ldg(a.ccode + k0 + u) : ~code;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (cc[u] == code) hit(i - (m - 1), __ldg(a.cr + k0 + u));
        }
    }
}

template <bool SHIFT_SMEM, bool DNA>
__global__ void __launch_bounds__(512, 1) wm_scan_kernel(const WmArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *p = smem;
    uint8_t *s_shift = p;
    p += (SHIFT_SMEM && !DNA) ? r16w(1LL << a.hbits) : 0;
    uint8_t *s_shift2 = p;
    p += DNA ? r16w(1LL << (2 * a.B)) : 0;
    uint32_t *s_dir = reinterpret_cast<uint32_t *>(p);
    p += DNA ? r16w((long long)(a.nkey + 1) * 4) : 0;
    uint32_t *s_hist = a.hist_smem ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += a.hist_smem ? r16w((long long)a.d * 4) : 0;
    p += warp * wm_warp_bytes(a.m, a.pool_cap, a.stage_cap);
    uint64_t *bar = reinterpret_cast<uint64_t *>(p);
    uint8_t *buf = p + 16;
    uint32_t *pool = reinterpret_cast<uint32_t *>(buf + r16w(a.buf));
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(
        reinterpret_cast<unsigned char *>(pool) + r16w((long long)a.pool_cap * 32 * 4));

    if (DNA) {
        for (int i = threadIdx.x; i < (1 << (2 * a.B)); i += blockDim.x) s_shift2[i] = a.shift2_g[i];
        for (int i = threadIdx.x; i <= a.nkey; i += blockDim.x) s_dir[i] = a.dir_g[i];
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
    dev::TileSchedule sch;
    sch.init(a.ntiles);
    uint32_t phase = 0;
    unsigned long long my_total = 0;
    if (sch.cur >= 0 && lane == 0) wm_stage_issue(a, sch.cur, buf, bar);

    for (long long t = sch.cur; t >= 0; t = sch.next_of(t)) {
        const bool got = __all_sync(kFull, dev::mbar_wait_bounded(bar, phase));
        if (!got) {
            if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutTma);
            break;
        }
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
        const long long g0 = tile0 + cs;
        int lim = kChunk + m - 1;          // window ends at offsets < lim
        {
            const long long left = a.n - g0;
            if (left < lim) lim = left <= 0 ? 0 : int(left);
        }
        const uint8_t *w = buf + cs;
        uint32_t nh = 0;
        auto rec = [&](int off, uint32_t r) {
            if (nh < cap) pl[nh * 32] = (uint32_t(off) << 24) | r;
            ++nh;
        };
        if (DNA) wm_walk_dna(a, s_shift2, s_dir, w, lim, rec);
        else wm_walk<SHIFT_SMEM>(a, s_shift, w, lim, rec);
        const bool ovf = nh > cap;
        const uint32_t cnt = nh;

        if (!a.list) {
            if (!ovf) {
                for (uint32_t k = 0; k < nh; ++k)
                    dev::count_pattern(pl[k * 32] & 0xFFFFFFu, s_hist, a.counts);
            } else {
                auto cnt_hit = [&](int, uint32_t r) { dev::count_pattern(r, s_hist, a.counts); };
                if (DNA) wm_walk_dna(a, s_shift2, s_dir, w, lim, cnt_hit);
                else wm_walk<SHIFT_SMEM>(a, s_shift, w, lim, cnt_hit);
            }
            my_total += cnt;
        } else {
            const uint32_t incl = dev::warp_incl_scan(cnt, lane);
            const uint32_t excl = incl - cnt;
            const uint32_t wtot = __shfl_sync(kFull, incl, 31);
            bool ok;
            const unsigned long long base = dev::lookback(a.lb, t, wtot, lane, ok);
            if (!ok) {
                if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutLookback);
                break;
            }
            if (lane == 0 && t == a.ntiles - 1) *a.n_occ = (long long)(base + wtot);
            if (!__any_sync(kFull, ovf)) {
                uint32_t k = 0, my = excl;
                const uint32_t S = uint32_t(a.stage_cap);
                for (uint32_t w0 = 0; w0 < wtot; w0 += S) {
                    const uint32_t wend = min(w0 + S, wtot);
                    const uint32_t lim = min(wend, incl);  // this lane's entries in the window
                    while (my < lim) {
                        const uint32_t v = pl[k * 32];
                        ++k;
                        const uint32_t r = v & 0xFFFFFFu;
                        stage[my - w0] = ((unsigned long long)(g0 + (v >> 24)) << 32) | r;
                        dev::count_pattern(r, s_hist, a.counts);
                        ++my;
                    }
                    __syncwarp();
                    for (uint32_t q = w0 + lane; q < wend; q += 32) {
                        const unsigned long long gi = base + q;
                        if (gi < (unsigned long long)a.occ_cap) a.occ[gi] = stage[q - w0];
                    }
                    __syncwarp();
                }
            } else {
                unsigned long long gi = base + excl;
                auto put = [&](long long pos, uint32_t r) {
                    if (gi < (unsigned long long)a.occ_cap)
                        a.occ[gi] = ((unsigned long long)pos << 32) | r;
                    ++gi;
                    dev::count_pattern(r, s_hist, a.counts);
                };
                if (!ovf) {
                    for (uint32_t k = 0; k < nh; ++k) {
                        const uint32_t v = pl[k * 32];
                        put(g0 + (v >> 24), v & 0xFFFFFFu);
                    }
                } else {
                    auto put_hit = [&](int off, uint32_t r) { put(g0 + off, r); };
                    if (DNA) wm_walk_dna(a, s_shift2, s_dir, w, lim, put_hit);
                    else wm_walk<SHIFT_SMEM>(a, s_shift, w, lim, put_hit);
                }
            }
        }

        // the buffer is free: stage the next tile
        dev::fence_proxy_async_smem();
        __syncwarp();
        if (sch.next_of(t) >= 0 && lane == 0) wm_stage_issue(a, sch.next_of(t), buf, bar);
    }

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
                        int pool_cap, int stage_cap, bool dna, int B, int nkey)
{
    const long long tables = dna ? r16w(1LL << (2 * B)) + r16w((long long)(nkey + 1) * 4)
                                 : (shift_smem ? r16w(1LL << hbits) : 0);
    return tables + (hist ? r16w((long long)d * 4) : 0) + (long long)warps * wm_warp_bytes(m, pool_cap, stage_cap);
}

}  // namespace

int wm_plan(const WmTables &t, const pm_params &opt, const DeviceProps &dp, DevWm &dev)
{
    const long long budget = (long long)dp.smem_optin - 1024;
    const int hbits = 5 * t.B;
    dev.pool_cap = 40;
    dev.stage_cap = 128;
    dev.ctas_per_sm = opt.ctas_per_sm > 0 ? opt.ctas_per_sm : 1;
    const int forced = opt.warps_per_cta > 0 ? std::min(opt.warps_per_cta, 16) : 0;
    const bool shift_smem = hbits <= 15;
    const int choices[3] = {16, 12, 8};
    for (int pass = 0; pass < 2; ++pass) {
        for (int wi = 0; wi < 3; ++wi) {
            const int w = forced ? forced : choices[wi];
            const int hist = pass == 0 ? 1 : 0;
            const long long need = wm_smem_bytes(hbits, shift_smem, hist, int(t.d), w, t.m, dev.pool_cap,
                                                 dev.stage_cap, t.dna, t.B, 1 << (2 * (t.B + t.Bp)));
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

int wm_launch(const WmTables &t, const DevWm &dv, const uint8_t *d_text, int64_t n, bool list,
              int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
              void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const long long ntiles = warp_tiles(n);
    e = cudaMemsetAsync(d_counts, 0, size_t(t.d) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_n_occ, 0, sizeof(int64_t), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_ws, 0, size_t(zeroed_workspace_bytes(ntiles, list, 0)), st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (n < t.m || ntiles == 0) return PM_OK;

    typedef void (*K)(const WmArgs);
    K fn = dv.dna ? wm_scan_kernel<false, true>
                  : (dv.shift_smem ? wm_scan_kernel<true, false> : wm_scan_kernel<false, false>);
    static int attr_bytes[3] = {0, 0, 0};
    const int slot = dv.dna ? 2 : (dv.shift_smem ? 1 : 0);
    if (attr_bytes[slot] < dv.smem_bytes) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dv.smem_bytes));
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        attr_bytes[slot] = int(dv.smem_bytes);
    }
    DeviceProps dp;
    int rc = device_props(dp);
    if (rc) return rc;

    WmArgs a;
    a.text = d_text;
    a.n = n;
    a.aligned = (reinterpret_cast<uintptr_t>(d_text) & 15) == 0;
    a.shift_g = dv.shift;
    a.hbits = 5 * t.B;
    a.hoff = dv.hoff;
    a.hids = dv.hids;
    a.hpfx = dv.hpfx;
    a.pats = dv.pats;
    a.m = t.m;
    a.B = t.B;
    a.Bp = t.Bp;
    a.ntiles = ntiles;
    a.pool_cap = dv.pool_cap;
    a.stage_cap = dv.stage_cap;
    a.buf = wm_buf_bytes(t.m);
    a.list = list ? 1 : 0;
    a.hist_smem = dv.hist_smem;
    a.d = int(t.d);
    a.counts = reinterpret_cast<long long *>(d_counts);
    a.occ = reinterpret_cast<unsigned long long *>(d_occ);
    a.occ_cap = list ? occ_cap : 0;
    a.n_occ = reinterpret_cast<long long *>(d_n_occ);
    char *w = static_cast<char *>(d_ws);
    a.ws = reinterpret_cast<dev::WsHeader *>(w);
    a.lb.tile_st = reinterpret_cast<unsigned long long *>(w + kWsHeader);
    a.lb.super_acc = reinterpret_cast<unsigned long long *>(w + kWsHeader + ntiles * 8);
    a.lb.super_pre = reinterpret_cast<unsigned long long *>(w + kWsHeader + ntiles * 16);
    a.lb.ntiles = ntiles;
    a.lut = t.lut;
    a.shift2_g = dv.shift2;
    a.dir_g = dv.dir;
    a.ccode = reinterpret_cast<const unsigned long long *>(dv.ccode);
    a.cr = dv.cr;
    a.nkey = t.dna ? (1 << (2 * (t.B + t.Bp))) : 0;

    // the static tile schedule needs every CTA of the grid resident at once
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, dv.warps * 32, size_t(dv.smem_bytes));
    if (e != cudaSuccess || per_sm < 1) { set_cuda_error(int(e)); return PM_ECUDA; }
    long long grid = (long long)dp.sm_count * std::min(per_sm, dv.ctas_per_sm);
    const long long want = (ntiles + dv.warps - 1) / dv.warps;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    a.lb.super_tiles = dev::super_size_for(grid * dv.warps);
    fn<<<dim3(unsigned(grid)), dim3(unsigned(dv.warps * 32)), size_t(dv.smem_bytes), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    return PM_OK;
}

}  // namespace pm
