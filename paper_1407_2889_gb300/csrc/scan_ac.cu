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
// Output: each lane records the table index of every match transition
// (pool, in shared memory) and a bit per step. After the walk the warp
// resolves multiplicities of duplicate patterns, computes per-lane offsets
// with a warp scan and the tile's global offset with a decoupled look-back
// over tiles, then writes the sorted (i, r) keys through a shared-memory
// staging window so global stores are coalesced (the paper's coalesced
// writes, GPU-CW). Per-pattern counts go to shared-memory counters when
// they fit, else to global atomics.
#include <cstdio>

#include "scan_common.cuh"

namespace pm {
namespace {

using dev::kFull;

struct AcArgs {
    const uint8_t *text;
    long long n;
    int aligned;
    const void *table_g;
    int smem_entries;
    const uint32_t *mid;
    uint32_t mid_base;
    const uint32_t *grp_off;
    const uint32_t *grp_ids;
    const uint8_t *cls_g;
    int m, lw;
    uint32_t lut;
    uint32_t pad;
    long long ntiles;
    int pool_cap, stage_cap;
    int list, has_dups, hist_smem, d;
    long long *counts;
    unsigned long long *occ;
    long long occ_cap;
    long long *n_occ;
    dev::WsHeader *ws;
    unsigned long long *tile_status;
};

__host__ __device__ constexpr int r16(long long x) { return int((x + 15) & ~15LL); }

template <int HV>
__host__ __device__ constexpr int ac_buf_bytes() { return kWarpTile + 16 * HV; }

__host__ __device__ inline int ac_warp_bytes(int hv, int pool_cap, int eb, int stage_cap)
{
    return 16 + r16(kWarpTile + 16 * hv) + r16((long long)pool_cap * 32 * eb) + stage_cap * 8;
}

template <typename E, bool HYB>
struct TableRef {
    const E *s;
    const E *g;
    uint32_t lim;
    __device__ __forceinline__ uint32_t operator()(uint32_t idx) const
    {
        if (!HYB) return s[idx];
        return idx < lim ? uint32_t(s[idx]) : uint32_t(__ldg(g + idx));
    }
};

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int q)
{
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// DFA walk over one lane's register text, ACGT-like alphabet. Calls
// hit(step, idx) for every transition that enters a terminal state; step is
// the index of the byte that completes the match.
template <int NV, class Tab, class F>
__device__ __forceinline__ void walk_dna(const uint4 (&tv)[NV], int steps, uint32_t lut,
                                         const Tab &tab, F &&hit)
{
    uint32_t e = 2u;  // root (row 1)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t w = word_of(tv[v], q);
            const uint32_t a4 = ((w >> 1) ^ (w >> 2)) & 0x03030303u;
            const uint32_t sel = __byte_perm(a4 | (a4 >> 4), 0u, 0x4420);
            const uint32_t x = w ^ __byte_perm(lut, 0u, sel);  // zero byte = in alphabet
            const uint32_t y = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
            const uint32_t vb = (y >> 7) * 0xFFu;   // 0xFF per valid byte
            const uint32_t v2 = vb & 0xFCFCFCFCu;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int step = v * 16 + q * 4 + k;
                if (step < kChunk || step < steps) {
                    const uint32_t c = __byte_perm(a4, 0u, 0x4440 | k);
                    const uint32_t vm = __byte_perm(
                        v2, vb, (k) | ((4 + k) << 4) | ((4 + k) << 8) | ((4 + k) << 12));
                    const uint32_t idx = ((e << 1) & vm) | c;  // invalid byte -> row 0
                    e = tab(idx);
                    if (e & 1u) hit(step, idx);
                }
            }
        }
    }
}

// General alphabet: class map in shared memory; steps already clipped to n.
template <int NV, class Tab, class F>
__device__ __forceinline__ void walk_gen(const uint4 (&tv)[NV], int steps, int lw,
                                         const uint8_t *s_cls, const Tab &tab, F &&hit)
{
    uint32_t e = 2u;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t w = word_of(tv[v], q);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int step = v * 16 + q * 4 + k;
                if (step < steps) {
                    const uint32_t c = s_cls[(w >> (8 * k)) & 0xFFu];
                    const uint32_t idx = c == 0xFFu ? 0u : (((e >> 1) << lw) | c);
                    e = tab(idx);
                    if (e & 1u) hit(step, idx);
                }
            }
        }
    }
}

// Rolled re-walk of one lane's chunk straight from global memory, for the
// rare lanes whose hit pool overflowed; same transitions as the fast walks.
template <class Tab, class F>
__device__ __forceinline__ void walk_slow(const uint8_t *text, long long n, long long g0,
                                          int steps, bool dna, uint32_t lut, int lw,
                                          const uint8_t *s_cls, const Tab &tab, F &&hit)
{
    uint32_t e = 2u;
#pragma unroll 1
    for (int step = 0; step < steps; ++step) {
        const long long g = g0 + step;
        if (g >= n) break;
        const uint32_t b = text[g];
        uint32_t idx;
        if (dna) {
            const uint32_t c = ((b >> 1) ^ (b >> 2)) & 3u;
            idx = ((lut >> (8 * c)) & 0xFFu) == b ? (((e >> 1) << 2) | c) : c;
        } else {
            const uint32_t c = s_cls[b];
            idx = c == 0xFFu ? 0u : (((e >> 1) << lw) | c);
        }
        e = tab(idx);
        if (e & 1u) hit(step, idx);
    }
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

// Iterates one lane's hits in step order: positions from the step bitmask,
// table indices from the pool.
template <int HMW>
struct HitBits {
    unsigned long long c0, c1, c2;
    int wbase;
    // -1 if no bit is left (cannot happen when called once per recorded hit)
    __device__ __forceinline__ int next()
    {
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (c0 != 0ull) break;
            c0 = c1;
            c1 = c2;
            c2 = 0ull;
            wbase += 64;
        }
        if (c0 == 0ull) return -1;
        const int b = __ffsll((long long)c0) - 1;
        c0 &= c0 - 1ull;
        return wbase + b;
    }
};

template <typename E, int NV, int HV, bool DNA, bool HYB>
__global__ void __launch_bounds__(512, 1) ac_scan_kernel(const AcArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int BUF = ac_buf_bytes<HV>();
    constexpr int HMW = (16 * NV + 63) / 64;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    // ---- shared memory carve-up (mirrors ac_smem_bytes on the host) -------
    unsigned char *p = smem;
    E *s_tab = reinterpret_cast<E *>(p);
    p += r16((long long)a.smem_entries * sizeof(E));
    uint32_t *s_hist = a.hist_smem ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += a.hist_smem ? r16((long long)a.d * 4) : 0;
    uint8_t *s_cls = p;
    p += DNA ? 0 : 256;
    p += warp * ac_warp_bytes(HV, a.pool_cap, sizeof(E), a.stage_cap);
    uint64_t *bar = reinterpret_cast<uint64_t *>(p);
    uint8_t *buf = p + 16;
    E *pool = reinterpret_cast<E *>(buf + r16(BUF));
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(
        reinterpret_cast<unsigned char *>(pool) + r16((long long)a.pool_cap * 32 * sizeof(E)));

    {   // table prefix -> shared memory (16-byte vectors; the global copy is padded)
        const uint4 *src = reinterpret_cast<const uint4 *>(a.table_g);
        uint4 *dst = reinterpret_cast<uint4 *>(s_tab);
        const int nvec = int(((long long)a.smem_entries * sizeof(E) + 15) / 16);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = src[i];
    }
    if (s_hist)
        for (int i = threadIdx.x; i < a.d; i += blockDim.x) s_hist[i] = 0u;
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

    dev::TileCursor cur;
    long long t = cur.claim(a.ws, lane, a.ntiles);
    uint32_t phase = 0;
    bool inflight = false;
    unsigned long long my_total = 0;
    if (t >= 0) {
        if (lane == 0) stage_issue(a, t, buf, bar, BUF);
        inflight = true;
    }

    while (t >= 0) {
        const bool got = __all_sync(kFull, dev::mbar_wait_bounded(bar, phase));
        if (!got) {
            if (lane == 0) dev::set_status(a.ws, dev::kErrTimeoutTma);
            inflight = false;  // the copy never completed; nothing to wait for
            break;
        }
        inflight = false;
        phase ^= 1u;
        const long long tile0 = t * kWarpTile;
        const int got_bytes = stage_bytes(a, t, BUF);
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
        const long long tn = cur.next(a.ws, lane, a.ntiles);
        dev::fence_proxy_async_smem();
        __syncwarp();
        if (tn >= 0) {
            if (lane == 0) stage_issue(a, tn, buf, bar, BUF);
            inflight = true;
        }

        // ---- walk ----------------------------------------------------------
        const long long g0 = tile0 + (long long)lane * kChunk;
        int steps = kChunk + m - 1;
        if (!DNA) {
            const long long left = a.n - g0;
            steps = left <= 0 ? 0 : (left < steps ? int(left) : steps);
        }
        uint32_t nh = 0;
        unsigned long long hm[3] = {0ull, 0ull, 0ull};
        auto rec = [&](int step, uint32_t idx) {
            hm[step >> 6] |= 1ull << (step & 63);
            if (nh < cap) pl[nh * 32] = E(idx - a.mid_base);
            ++nh;
        };
        if (DNA) walk_dna<NV>(tv, steps, a.lut, tab, rec);
        else walk_gen<NV>(tv, steps, a.lw, s_cls, tab, rec);
        const bool ovf = nh > cap;

        // ---- multiplicity of duplicate patterns ----------------------------
        uint32_t cnt = nh;
        if (a.has_dups) {
            if (!ovf) {
                for (uint32_t k = 0; k < nh; ++k) {
                    const uint32_t v = __ldg(a.mid + pl[k * 32]);
                    if (v & 0x80000000u) {
                        const uint32_t g = v & 0x7FFFFFFFu;
                        cnt += __ldg(a.grp_off + g + 1) - __ldg(a.grp_off + g) - 1u;
                    }
                }
            } else {
                cnt = 0;
                auto cm = [&](int, uint32_t idx) {
                    const uint32_t v = __ldg(a.mid + (idx - a.mid_base));
                    if (v & 0x80000000u) {
                        const uint32_t g = v & 0x7FFFFFFFu;
                        cnt += __ldg(a.grp_off + g + 1) - __ldg(a.grp_off + g);
                    } else {
                        cnt += 1u;
                    }
                };
                walk_slow(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab, cm);
            }
        }

        // direct emission of one match (overflow path); gi < 0: count only
        auto emit_direct = [&](long long pos, uint32_t v, unsigned long long &gi, bool write) {
            if (v & 0x80000000u) {
                const uint32_t g = v & 0x7FFFFFFFu;
                const uint32_t hi = __ldg(a.grp_off + g + 1);
                for (uint32_t k = __ldg(a.grp_off + g); k < hi; ++k) {
                    const uint32_t r = __ldg(a.grp_ids + k);
                    if (write && gi < (unsigned long long)a.occ_cap)
                        a.occ[gi] = ((unsigned long long)pos << 32) | r;
                    ++gi;
                    dev::count_pattern(r, s_hist, a.counts);
                }
            } else {
                if (write && gi < (unsigned long long)a.occ_cap)
                    a.occ[gi] = ((unsigned long long)pos << 32) | v;
                ++gi;
                dev::count_pattern(v, s_hist, a.counts);
            }
        };

        if (!a.list) {
            // ---- counts only ---------------------------------------------
            unsigned long long gi = 0;
            if (!ovf) {
                for (uint32_t k = 0; k < nh; ++k)
                    emit_direct(0, __ldg(a.mid + pl[k * 32]), gi, false);
            } else {
                auto cd = [&](int, uint32_t idx) {
                    emit_direct(0, __ldg(a.mid + (idx - a.mid_base)), gi, false);
                };
                walk_slow(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab, cd);
            }
            my_total += cnt;
            t = tn;
            continue;
        }

        // ---- offsets: warp scan + decoupled look-back over tiles ----------
        const uint32_t incl = dev::warp_incl_scan(cnt, lane);
        const uint32_t excl = incl - cnt;
        const uint32_t wtot = __shfl_sync(kFull, incl, 31);
        unsigned long long base = 0;
        int okl = 1;
        if (lane == 0) {
            bool ok;
            base = dev::lookback(a.tile_status, t, wtot, ok);
            okl = ok;
            if (!ok) dev::set_status(a.ws, dev::kErrTimeoutLookback);
            if (t == a.ntiles - 1) *a.n_occ = (long long)(base + wtot);
        }
        base = __shfl_sync(kFull, base, 0);
        if (!__shfl_sync(kFull, okl, 0)) break;

        if (!__any_sync(kFull, ovf)) {
            // ---- staged, coalesced emission -------------------------------
            HitBits<HMW> it{hm[0], hm[1], hm[2], 0};
            uint32_t k = 0, my = excl;
            bool have = false, single = true;
            uint32_t rs = 0, glo = 0, ghi = 0;
            long long pos = 0;
            const uint32_t S = uint32_t(a.stage_cap);
            for (uint32_t w0 = 0; w0 < wtot; w0 += S) {
                const uint32_t wend = min(w0 + S, wtot);
                const uint32_t lim = min(wend, incl);  // this lane's entries in the window
                while (my < lim) {
                    if (!have) {
                        const int st = it.next();
                        if (st < 0) dev::set_status(a.ws, dev::kErrInternal);
                        pos = g0 + st - (m - 1);
                        const uint32_t v = __ldg(a.mid + pl[k * 32]);
                        ++k;
                        single = !(v & 0x80000000u);
                        if (single) {
                            rs = v;
                        } else {
                            const uint32_t g = v & 0x7FFFFFFFu;
                            glo = __ldg(a.grp_off + g);
                            ghi = __ldg(a.grp_off + g + 1);
                        }
                        have = true;
                    }
                    const uint32_t r = single ? rs : __ldg(a.grp_ids + glo);
                    stage[my - w0] = ((unsigned long long)pos << 32) | r;
                    dev::count_pattern(r, s_hist, a.counts);
                    ++my;
                    if (single || ++glo >= ghi) have = false;
                }
                __syncwarp();
                for (uint32_t q = w0 + lane; q < wend; q += 32) {
                    const unsigned long long gi = base + q;
                    if (gi < (unsigned long long)a.occ_cap) a.occ[gi] = stage[q - w0];
                }
                __syncwarp();
            }
        } else {
            // ---- a lane overflowed its pool: every lane writes directly --
            unsigned long long gi = base + excl;
            if (!ovf) {
                HitBits<HMW> it{hm[0], hm[1], hm[2], 0};
                for (uint32_t k = 0; k < nh; ++k) {
                    const int st = it.next();
                    if (st < 0) dev::set_status(a.ws, dev::kErrInternal);
                    const long long pos = g0 + st - (m - 1);
                    emit_direct(pos, __ldg(a.mid + pl[k * 32]), gi, true);
                }
            } else {
                auto ed = [&](int step, uint32_t idx) {
                    emit_direct(g0 + step - (m - 1), __ldg(a.mid + (idx - a.mid_base)), gi, true);
                };
                walk_slow(a.text, a.n, g0, kChunk + m - 1, DNA, a.lut, a.lw, s_cls, tab, ed);
            }
        }
        t = tn;
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
    __syncthreads();
    if (s_hist) {
        for (int r = threadIdx.x; r < a.d; r += blockDim.x) {
            const uint32_t c = s_hist[r];
            if (c) atomicAdd(reinterpret_cast<unsigned long long *>(a.counts) + r, (unsigned long long)c);
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

long long ac_smem_bytes(long long smem_entries, int eb, int hist_smem, int d, bool dna, int warps,
                        int hv, int pool_cap, int stage_cap)
{
    return r16(smem_entries * eb) + (hist_smem ? r16((long long)d * 4) : 0) + (dna ? 0 : 256) +
           (long long)warps * ac_warp_bytes(hv, pool_cap, eb, stage_cap);
}

}  // namespace

int ac_plan(const AcTables &t, const pm_params &opt, const DeviceProps &dp, DevAc &dev)
{
    const int hv = hv_for_m(t.m);
    if (hv < 0) return PM_ETOOBIG;
    const int eb = t.dna ? t.entry_bytes : 4;
    const long long entries = (long long)t.n_rows << t.lw;
    const long long budget = (long long)dp.smem_optin - 1024;
    const int pool_cap = 40, stage_cap = 128;
    int place = opt.placement;
    const int warp_choices[3] = {16, 12, 8};
    int forced_warps = opt.warps_per_cta > 0 ? std::min(opt.warps_per_cta, 16) : 0;

    dev.pool_cap = pool_cap;
    dev.stage_cap = stage_cap;
    dev.hv = hv;
    dev.nv = 5 + hv;
    dev.ctas_per_sm = opt.ctas_per_sm > 0 ? opt.ctas_per_sm : 1;

    bool chosen = false;
    if (place == PM_PLACE_AUTO || place == PM_PLACE_SMEM) {
        // whole table in shared memory: prefer per-pattern counters in
        // shared memory with >= 12 warps, then 16 warps without them
        for (int pass = 0; pass < 2 && !chosen; ++pass) {
            for (int wi = 0; wi < 3 && !chosen; ++wi) {
                const int w = forced_warps ? forced_warps : warp_choices[wi];
                const int hist = pass == 0 ? 1 : 0;
                if (pass == 0 && w < 12 && !forced_warps) continue;
                const long long need = ac_smem_bytes(entries, eb, hist, int(t.d), t.dna, w, hv,
                                                     pool_cap, stage_cap);
                const bool per_sm_ok =
                    need * dev.ctas_per_sm + 1024LL * dev.ctas_per_sm <= (long long)dp.smem_per_sm;
                if (need <= budget && per_sm_ok &&
                    (opt.smem_table_bytes <= 0 || entries * eb <= opt.smem_table_bytes)) {
                    dev.warps = w;
                    dev.hist_smem = hist;
                    dev.smem_entries = entries;
                    dev.placement = PM_PLACE_SMEM;
                    chosen = true;
                }
                if (forced_warps) break;
            }
        }
        if (!chosen && place == PM_PLACE_SMEM) return PM_ETOOBIG;
    }
    if (!chosen) {
        // hybrid / global: breadth-first prefix of rows in shared memory
        const int w = forced_warps ? forced_warps : 16;
        const long long fixed = ac_smem_bytes(0, eb, 0, int(t.d), t.dna, w, hv, pool_cap, stage_cap);
        long long room = budget - fixed;
        if (opt.smem_table_bytes > 0) room = std::min<long long>(room, opt.smem_table_bytes);
        if (place == PM_PLACE_GLOBAL) room = 0;
        long long se = room > 0 ? room / eb : 0;
        se &= ~((long long)(16 / eb) - 1);   // whole 16-byte vectors
        if (se > entries) se = entries;
        dev.warps = w;
        dev.hist_smem = 0;
        dev.smem_entries = se;
        dev.placement = place == PM_PLACE_GLOBAL ? PM_PLACE_GLOBAL : PM_PLACE_HYBRID;
    }
    const bool hyb = dev.smem_entries < entries || !t.dna || eb == 4;
    int group;
    if (!t.dna) group = 3;
    else if (eb == 4) group = 2;
    else group = hyb ? 1 : 0;
    dev.variant = group * 3 + hv_slot(hv);
    dev.smem_bytes = ac_smem_bytes(dev.smem_entries, eb, dev.hist_smem, int(t.d), t.dna, dev.warps,
                                   hv, pool_cap, stage_cap);
    return PM_OK;
}

int ac_launch(const AcTables &t, const DevAc &dv, const uint8_t *d_text, int64_t n, bool list,
              int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
              void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const long long ntiles = warp_tiles(n);
    e = cudaMemsetAsync(d_counts, 0, size_t(t.d) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_n_occ, 0, sizeof(int64_t), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_ws, 0, size_t(workspace_bytes_for(n, list)), st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (n < t.m || ntiles == 0) return PM_OK;

    const Variant &v = kVariants[dv.variant];
    static bool attr_set[sizeof(kVariants) / sizeof(kVariants[0])] = {};
    static int attr_bytes[sizeof(kVariants) / sizeof(kVariants[0])] = {};
    if (!attr_set[dv.variant] || attr_bytes[dv.variant] < dv.smem_bytes) {
        e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dv.smem_bytes));
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        attr_set[dv.variant] = true;
        attr_bytes[dv.variant] = int(dv.smem_bytes);
    }
    DeviceProps dp;
    int rc = device_props(dp);
    if (rc) return rc;

    AcArgs a;
    a.text = d_text;
    a.n = n;
    a.aligned = (reinterpret_cast<uintptr_t>(d_text) & 15) == 0;
    a.table_g = dv.table ? dv.table : nullptr;
    a.smem_entries = int(dv.smem_entries);
    a.mid = dv.mid;
    a.mid_base = uint32_t(t.d0_row << t.lw);
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
    a.pool_cap = dv.pool_cap;
    a.stage_cap = dv.stage_cap;
    a.list = list ? 1 : 0;
    a.has_dups = t.has_dups ? 1 : 0;
    a.hist_smem = dv.hist_smem;
    a.d = int(t.d);
    a.counts = reinterpret_cast<long long *>(d_counts);
    a.occ = reinterpret_cast<unsigned long long *>(d_occ);
    a.occ_cap = list ? occ_cap : 0;
    a.n_occ = reinterpret_cast<long long *>(d_n_occ);
    a.ws = reinterpret_cast<dev::WsHeader *>(d_ws);
    a.tile_status = reinterpret_cast<unsigned long long *>(static_cast<char *>(d_ws) + kWsHeader);

    const int threads = dv.warps * 32;
    long long want = (ntiles + (long long)dv.warps * dev::kClaimBatch - 1) /
                     ((long long)dv.warps * dev::kClaimBatch);
    long long grid = (long long)dp.sm_count * dv.ctas_per_sm;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    v.fn<<<dim3(unsigned(grid)), dim3(unsigned(threads)), size_t(dv.smem_bytes), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    return PM_OK;
}

}  // namespace pm
