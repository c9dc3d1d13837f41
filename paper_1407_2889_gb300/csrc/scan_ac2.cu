// scan_ac2.cu -- Aho-Corasick DFA scan taking two characters per table
// lookup (a multi-character table of the DFA form of Section 3.1, Algorithm
// 3) on sm_103a, for ACGT-like sets of at most 4096 rows and m <= 33.
//
// A row has 16 entries, one per pair of character classes, holding the
// state after both characters and a match flag for each, (r2 << 4) |
// (m1 << 1) | m2: the one-character table applied twice (the same rows, terminal rows elided). A lane walks
// its chunk + halo a pair at a time. A byte outside the alphabet resets the
// walk inside the lookup chain: as the pair's first byte it selects row 0
// (the one-character reset row applied first, so its entry for (c1, c2) is
// the root's transition on c2), as the second it sends the state to the
// root after the pair and drops the pair's second flag. The walk keeps a
// step bitmask of matches in registers and stores each 16-byte vector's
// eight pair indices with one shared-memory store; the matches are resolved
// afterwards from those records (a second-character match through one more
// lookup of the one-character table). The workspace, slots and expand
// kernel are those of the one-character scan.
#include "ac_device.cuh"

namespace pm {
namespace {

using dev::kFull;

struct Ac2Args {
    const uint8_t *text;
    long long n;
    int aligned;
    const uint16_t *tab1_g;       // one-character table, index entries (row << 2) | flag
    const uint16_t *tab2_g;       // two-character table
    int n_rows;
    uint32_t mid_base;            // first table index of the match rows
    const uint32_t *mask_g;       // match-entry bitmap words
    const uint16_t *rank_g;       // set bits before each word
    const uint16_t *canon_g;      // pattern id, or 0x8000 | group, per terminal
    int nwords, nterms;
    const uint32_t *grp_off;
    const uint32_t *grp_ids;
    int m;
    uint32_t lut;
    uint32_t pad;
    long long nsub;
    int pool_cap;
    int list, hist_smem, d;
    long long *counts;
    long long *n_occ;
    dev::WsHeader *ws;
    unsigned long long *ccount;   // per-terminal totals
    uint32_t *tile_ent, *tile_out;
    unsigned long long *seg_sum;
    long long seg_tiles;
    uint32_t *slots;              // (start offset in the tile << 16) | code
    // Multipliers of the walk's shifts and adds, passed as arguments so the
    // compiler issues them as integer multiply-adds (the fused multiply-add
    // pipe, idle in this walk) instead of folding them into shifts on the
    // integer logic pipe, which the byte decoding keeps busy.
    uint32_t k_sh1, k_sh2, k_sh4, k_sh8, k_sh16, k_x2, k_x4, k_x65536, k_one;
};

__host__ __device__ constexpr long long r16a(long long x) { return (x + 15) & ~15LL; }

constexpr int kAc2MaxWarps = 24;  // one CTA per SM (a 768-thread launch bound, up to 85 registers)

// prmt.b32 in its generic mode: a selector nibble with bit 3 set fills its
// result byte with the sign (bit 7) of the selected byte (the __byte_perm
// intrinsic ignores that bit)
__device__ __forceinline__ uint32_t prmt_sign(uint32_t a, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(0u), "r"(sel));
    return d;
}

__host__ __device__ inline long long ac2_warp_bytes(int hv, int)
{
    // barrier | text buffer | pair records (16 bytes per lane per text vector)
    return 16 + r16a(kWarpTile + 16 * hv) + (long long)(5 + hv) * 32 * 16;
}

__device__ __forceinline__ int ac2_stage_bytes(const Ac2Args &a, long long t, int buf)
{
    if (!a.aligned) return 0;
    const long long avail = (a.n & ~15LL) - t * kWarpTile;
    if (avail <= 0) return 0;
    return avail >= buf ? buf : int(avail);
}

__device__ __forceinline__ void ac2_stage_issue(const Ac2Args &a, long long t, uint8_t *buf, uint64_t *bar,
                                                int bufsz)
{
    const int bytes = ac2_stage_bytes(a, t, bufsz);
    dev::mbar_arrive_expect_tx(bar, uint32_t(bytes));
    if (bytes > 0) dev::tma_load_1d(buf, a.text + t * kWarpTile, uint32_t(bytes), bar);
}

template <int NV, int HV>
__global__ void __launch_bounds__(kAc2MaxWarps * 32, 1) ac2_scan_kernel(const Ac2Args a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr uint32_t kGrp = 0x8000u;
    constexpr int HW = (NV * 16 + 31) / 32;  // words of the per-step masks
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int BUF = kWarpTile + 16 * HV;

    // ---- shared memory carve-up (mirrors ac2_smem_bytes on the host) ------
    unsigned char *p = smem;
    uint16_t *s_t1 = reinterpret_cast<uint16_t *>(p);
    p += r16a((long long)a.n_rows * 4 * 2);
    uint16_t *s_t2 = reinterpret_cast<uint16_t *>(p);
    p += r16a((long long)a.n_rows * 16 * 2);
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(p);
    p += r16a((long long)a.nwords * 4);
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(p);
    p += r16a((long long)(a.nwords + 1) * 2);
    uint16_t *s_canon = reinterpret_cast<uint16_t *>(p);
    p += r16a((long long)a.nterms * 2);
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(p);
    const long long hist_words = a.hist_smem == 2 ? (a.nterms + 1) / 2 : a.nterms;
    p += r16a(hist_words * 4);
    p += warp * ac2_warp_bytes(HV, a.pool_cap);
    uint64_t *bar = reinterpret_cast<uint64_t *>(p);
    uint8_t *buf = p + 16;
    unsigned char *rec = buf + r16a(BUF);  // lane l, vector v: 16 bytes at (v * 32 + l) * 16

    {
        const int n1 = int(((long long)a.n_rows * 8 + 15) / 16), n2 = int(((long long)a.n_rows * 32 + 15) / 16);
        const uint4 *g1 = reinterpret_cast<const uint4 *>(a.tab1_g);
        const uint4 *g2 = reinterpret_cast<const uint4 *>(a.tab2_g);
        for (int i = threadIdx.x; i < n1; i += blockDim.x) reinterpret_cast<uint4 *>(s_t1)[i] = g1[i];
        for (int i = threadIdx.x; i < n2; i += blockDim.x) reinterpret_cast<uint4 *>(s_t2)[i] = g2[i];
    }
    for (int i = threadIdx.x; i < a.nwords; i += blockDim.x) s_mask[i] = a.mask_g[i];
    for (int i = threadIdx.x; i <= a.nwords; i += blockDim.x) s_rank[i] = a.rank_g[i];
    for (int i = threadIdx.x; i < a.nterms; i += blockDim.x) s_canon[i] = a.canon_g[i];
    for (int i = threadIdx.x; i < hist_words; i += blockDim.x) s_hist[i] = 0u;
    if (lane == 0) dev::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dev::fence_proxy_async_smem();
    __syncthreads();

    const int m = a.m;
    const long long G = (long long)gridDim.x * (blockDim.x >> 5);
    const long long gwarp = (long long)blockIdx.x * (blockDim.x >> 5) + warp;

    // terminal of a match entry of the one-character table, its pattern code,
    // and a bump of its counter
    auto terminal = [&](uint32_t idx1) {
        const uint32_t off = uint32_t(uint16_t(idx1 - a.mid_base));
        const uint32_t w = off >> 5;
        return uint32_t(s_rank[w]) + __popc(s_mask[w] & ((1u << (off & 31u)) - 1u));
    };
    auto count_terminal = [&](uint32_t c) {
        if (a.hist_smem == 1) {
            atomicAdd(&s_hist[c], 1u);
        } else {
            // 16-bit halves: the add that takes a half to 0x8000 moves 0x8000
            // to the device counter
            const uint32_t sh = (c & 1u) << 4;
            const uint32_t old = atomicAdd(&s_hist[c >> 1], 1u << sh);
            if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
                atomicSub(&s_hist[c >> 1], 0x8000u << sh);
                atomicAdd(&a.ccount[c], 0x8000ull);
            }
        }
    };
    auto mult_of = [&](uint32_t code) -> uint32_t {
        if (!(code & kGrp)) return 1u;
        const uint32_t g = code & ~kGrp;
        return __ldg(a.grp_off + g + 1) - __ldg(a.grp_off + g);
    };

    uint32_t phase = 0;
    bool inflight = false;
    unsigned long long my_total = 0;
    if (gwarp < a.nsub) {
        if (lane == 0) ac2_stage_issue(a, gwarp, buf, bar, BUF);
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
        const int got_bytes = ac2_stage_bytes(a, st, BUF);
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
            if (lane == 0) ac2_stage_issue(a, st + G, buf, bar, BUF);
            inflight = true;
        }

        // ---- walk, a pair of characters per lookup ------------------------
        const int steps = kChunk + m - 1;
        uint32_t hw[HW];
#pragma unroll
        for (int j = 0; j < HW; ++j) hw[j] = 0u;
        uint32_t e2 = 16u;  // root: row 1
        const uint32_t rec0 = dev::smem_addr(rec) + uint32_t(lane) * 16u;
        const uint32_t t2_base = dev::smem_addr(s_t2);
        // x >> k as the high word of x * 2^(32-k), x << k and x + c as x * 2^k
        // + c: integer multiply-adds with multipliers the compiler cannot see
        const uint32_t K1 = a.k_sh1, K2 = a.k_sh2, K4 = a.k_sh4, K8 = a.k_sh8, K16 = a.k_sh16;
        const uint32_t X2 = a.k_x2, X4 = a.k_x4, X64K = a.k_x65536, ONE = a.k_one;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            uint32_t pk[4] = {0u, 0u, 0u, 0u};
            uint32_t hv = 0u;  // this vector's match bits, two per pair, first pair highest
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t w = acdev::word_of(tv[v], q);
                const int s0 = v * 16 + q * 4;
                if (!(s0 < kChunk || s0 < steps)) {
                    hv <<= 4;  // two pairs past the lane's walk
                    continue;
                }
                // class of each byte: ((b >> 1) ^ (b >> 2)) & 3
                const uint32_t a4 = (__umulhi(w, K1) ^ __umulhi(w, K2)) & 0x03030303u;
                // selector of the alphabet's byte for each class (nibbles)
                const uint32_t sel = __byte_perm(__umulhi(a4, K4) + a4, 0u, 0x4420);
                const uint32_t lutb = __byte_perm(a.lut, 0u, sel);
                // bit 7 of each byte of y: the byte is outside the alphabet
                const uint32_t t7 = (w ^ lutb) & 0x7F7F7F7Fu;
                const uint32_t y = (t7 * ONE + 0x7F7F7F7Fu) | (w ^ lutb);
                // pair codes (c1 << 2) | c2 in bytes 0 and 2
                const uint32_t u = __umulhi(a4, K8) + a4 * X4;
                // per pair (16-bit halves): t2 = 0xFFF0 | code, or the code
                // alone (row 0) when the first byte is outside; mx = 0xFFFF,
                // or 0x0002 (keep the first character's flag) when the second
                // byte is outside
                const uint32_t t2w = (~prmt_sign(y, 0xAA88u) & 0xFFF0FFF0u) | (u & 0x000F000Fu);
                const uint32_t mxw = ~prmt_sign(y, 0xBB99u) | 0x00020002u;
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int j0 = s0 + 2 * pp;  // first character's step
                    if (j0 < kChunk || j0 < steps) {
                        const uint32_t t2 = pp ? __umulhi(t2w, K16) : t2w;
                        const uint32_t mx = pp ? __umulhi(mxw, K16) : mxw;
                        const uint32_t idx2 = (e2 & t2 & ~15u) | (t2 & 15u);
                        uint16_t ev;
                        asm("ld.shared.u16 %0, [%1];" : "=h"(ev) : "r"(idx2 * X2 + t2_base));
                        e2 = (uint32_t(ev) & mx) | (16u & ~mx);
                        hv = hv * X4 + (e2 & 3u);
                        pk[q] = pp ? idx2 * X64K + pk[q] : idx2;
                    } else {
                        hv = hv * X4;
                    }
                }
            }
            if (v * 16 < steps)
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(rec0 + uint32_t(v) * 512u),
                             "r"(pk[0]), "r"(pk[1]), "r"(pk[2]), "r"(pk[3])
                             : "memory");
            // an entry's flags are (first character << 1) | second, so pair k
            // of the vector sits at bits 15 - 2k (first) and 14 - 2k: the
            // reversed word, shifted down, has step 16 v + i at bit i
            hw[v >> 1] |= (__brev(hv) >> 16) << (16 * (v & 1));
        }
        // a match at a step past the lane's last (the second byte of a last
        // pair that straddles it) is not this lane's
#pragma unroll
        for (int j = 0; j < HW; ++j) {
            const int lo = j * 32;
            if (lo + 32 > steps) hw[j] &= lo >= steps ? 0u : ((1u << (steps - lo)) - 1u);
        }
        uint32_t nh = 0;
#pragma unroll
        for (int j = 0; j < HW; ++j) nh += __popc(hw[j]);
        __syncwarp();

        // ---- matches -> counters, and the tile's slot in text order -------
        const uint32_t e_incl = a.list ? dev::warp_incl_scan(nh, lane) : 0u;
        uint32_t *dst = a.slots + st * kWarpTile + (e_incl - nh);
        const uint32_t off0 = uint32_t(lane * kChunk - (m - 1));
        uint32_t cnt = 0, kout = 0;
        const uint16_t *rec16 = reinterpret_cast<const uint16_t *>(rec);
#pragma unroll
        for (int j = 0; j < HW; ++j) {
            uint32_t wj = hw[j];
            while (wj) {
                const int b = __ffs(int(wj)) - 1;
                wj &= wj - 1u;
                const int step = j * 32 + b;
                const int p = step >> 1;
                const uint32_t idx2 = rec16[((p >> 3) * 32 + lane) * 8 + (p & 7)];
                uint32_t idx1 = idx2 >> 2;
                if (step & 1) idx1 = (uint32_t(s_t1[idx1]) & ~3u) | (idx2 & 3u);
                const uint32_t c = terminal(idx1);
                const uint32_t code = s_canon[c];
                count_terminal(c);
                cnt += mult_of(code);
                if (a.list) dst[kout] = ((off0 + uint32_t(step)) << 16) | code;
                ++kout;
            }
        }

        if (!a.list) {
            my_total += cnt;
            continue;
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

    // a copy still in flight after an error exit: wait for it (bounded)
    if (inflight) (void)dev::mbar_wait_bounded(bar, phase);

    if (!a.list) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_total += __shfl_down_sync(kFull, my_total, o);
        if (lane == 0 && my_total) atomicAdd(reinterpret_cast<unsigned long long *>(a.n_occ), my_total);
    }

    // ---- per-terminal counters -> global; the last CTA writes counts[r] ----
    __syncthreads();
    for (int c = threadIdx.x; c < a.nterms; c += blockDim.x) {
        const uint32_t v = a.hist_smem == 2 ? (s_hist[c >> 1] >> ((c & 1) << 4)) & 0xFFFFu : s_hist[c];
        if (v) atomicAdd(&a.ccount[c], (unsigned long long)v);
    }
    __threadfence();
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) s_last = atomicAdd(&a.ws->done_ctas, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int c = threadIdx.x; c < a.nterms; c += blockDim.x) {
            const unsigned long long v = dev::ld_acquire(&a.ccount[c]);
            const uint32_t code = a.canon_g[c];
            if (code & kGrp) {
                const uint32_t g = code & ~kGrp;
                for (uint32_t j = a.grp_off[g]; j < a.grp_off[g + 1]; ++j) a.counts[a.grp_ids[j]] = (long long)v;
            } else {
                a.counts[code] = (long long)v;
            }
        }
    }
}

long long ac2_smem_bytes(const AcTables &t, int hist, int warps, int hv, int pool_cap)
{
    const long long nwords = (long long)t.flag_mask.size(), nterms = (long long)t.canon.size();
    const long long hw = hist == 2 ? (nterms + 1) / 2 : nterms;
    return r16a(t.n_rows * 8) + r16a(t.n_rows * 32) + r16a(nwords * 4) + r16a((nwords + 1) * 2) + r16a(nterms * 2) +
           r16a(hw * 4) + (long long)warps * ac2_warp_bytes(hv, pool_cap);
}

}  // namespace

int ac2_plan(const AcTables &t, const pm_params &opt, const DeviceProps &dp, DevAc2 &dev)
{
    if (!ac2_eligible(t) || t.table2.empty()) return PM_ETOOBIG;
    const int hv = t.m - 1 <= 16 ? 1 : 2;
    const long long budget = (long long)dp.smem_optin - 1024;
    const int forced = opt.warps_per_cta > 0 ? std::min(opt.warps_per_cta, kAc2MaxWarps) : 0;
    // the most warps that fit, 32-bit counters before 16-bit ones
    for (int w = forced ? forced : kAc2MaxWarps; w >= (forced ? forced : 4); --w)
        for (int hist : {1, 2}) {
            const long long need = ac2_smem_bytes(t, hist, w, hv, 0);
            if (need > budget) continue;
            dev.warps = w;
            dev.pool_cap = 0;
            dev.hist_smem = hist;
            dev.hv = hv;
            dev.nv = 5 + hv;
            dev.smem_bytes = need;
            return PM_OK;
        }
    return PM_ETOOBIG;
}

int ac2_launch(const AcTables &t, const DevAc &dv, const DevAc2 &d2, const uint8_t *d_text, int64_t n, bool list,
               int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long nsub = warp_tiles(n);
    const long long nterms = (long long)t.canon.size();
    ListParts L;
    list_workspace_parts(d_ws, nsub, nterms, 4, L);
    const int64_t zeroed = list ? L.zeroed_bytes : kWsHeader + r16a(nterms * 8);
    cudaError_t e = cudaMemsetAsync(d_counts, 0, size_t(t.d) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_n_occ, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ws, 0, size_t(zeroed), st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (n < t.m || nsub == 0) return PM_OK;

    typedef void (*K)(const Ac2Args);
    const K fn = d2.hv == 1 ? ac2_scan_kernel<6, 1> : ac2_scan_kernel<7, 2>;
    int rc = kernel_smem_attr(reinterpret_cast<const void *>(fn), d2.smem_bytes);
    if (rc) return rc;
    DeviceProps dp;
    rc = device_props(dp);
    if (rc) return rc;
    Ac2Args a;
    a.text = d_text;
    a.n = n;
    a.aligned = (reinterpret_cast<uintptr_t>(d_text) & 15) == 0;
    a.tab1_g = static_cast<const uint16_t *>(dv.table);
    a.tab2_g = static_cast<const uint16_t *>(d2.table2);
    a.n_rows = int(t.n_rows);
    a.mid_base = uint32_t(t.d0_row << t.lw);
    a.mask_g = dv.flag_mask;
    a.rank_g = static_cast<const uint16_t *>(dv.flag_rank);
    a.canon_g = static_cast<const uint16_t *>(dv.canon);
    a.nwords = int(t.flag_mask.size());
    a.nterms = int(nterms);
    a.grp_off = dv.grp_off;
    a.grp_ids = dv.grp_ids;
    a.m = t.m;
    a.lut = t.lut;
    a.pad = 0;
    for (int b = 0; b < 256; ++b)
        if (t.cls[b] == 0xFF) { a.pad = uint32_t(b); break; }
    a.nsub = nsub;
    a.pool_cap = d2.pool_cap;
    a.list = list ? 1 : 0;
    a.hist_smem = d2.hist_smem;
    a.d = int(t.d);
    a.counts = reinterpret_cast<long long *>(d_counts);
    a.n_occ = reinterpret_cast<long long *>(d_n_occ);
    a.ws = reinterpret_cast<dev::WsHeader *>(d_ws);
    a.ccount = reinterpret_cast<unsigned long long *>(static_cast<char *>(d_ws) + kWsHeader);
    a.tile_ent = L.tile_ent;
    a.tile_out = L.tile_out;
    a.seg_sum = L.seg_sum;
    a.seg_tiles = L.seg_tiles;
    a.slots = static_cast<uint32_t *>(L.slots);
    a.k_sh1 = 1u << 31;
    a.k_sh2 = 1u << 30;
    a.k_sh4 = 1u << 28;
    a.k_sh8 = 1u << 24;
    a.k_sh16 = 1u << 16;
    a.k_x2 = 2u;
    a.k_x4 = 4u;
    a.k_x65536 = 65536u;
    a.k_one = 1u;

    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, d2.warps * 32, size_t(d2.smem_bytes));
    if (e != cudaSuccess || per_sm < 1) { set_cuda_error(int(e)); return PM_ECUDA; }
    long long grid = dp.sm_count;
    const long long want = (nsub + d2.warps - 1) / d2.warps;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    fn<<<dim3(unsigned(grid)), dim3(unsigned(d2.warps * 32)), size_t(d2.smem_bytes), st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (!list) return PM_OK;
    return expand_launch(d_ws, nsub, nterms, 4, dv.grp_off, dv.grp_ids, (int64_t)t.grp_off.size(),
                         (int64_t)t.grp_ids.size(), d_occ, occ_cap, d_n_occ, nullptr, 0, stream);
}

}  // namespace pm
