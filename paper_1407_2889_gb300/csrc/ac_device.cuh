// ac_device.cuh -- device building blocks of the Aho-Corasick scans (plain
// and batched): table access with shared-memory / L2 placement, the
// canonical-terminal lookup, the DFA walks over register-held text (ACGT
// alphabet decoded arithmetically, or a shared-memory class map), a rolled
// re-walk from global memory, and the iterator over recorded match steps.
#pragma once

#include "scan_common.cuh"

namespace pm {
namespace acdev {

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

// Canonical terminal id and pattern code of a match entry.
template <typename E>
struct Ids {
    const uint32_t *mask;
    const E *rank;
    const E *canon;
    __device__ __forceinline__ uint32_t terminal(uint32_t off) const
    {
        const uint32_t w = off >> 5, b = off & 31u;
        return uint32_t(rank[w]) + __popc(mask[w] & ((1u << b) - 1u));
    }
    __device__ __forceinline__ uint32_t code(uint32_t c) const { return canon[c]; }
};

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int q)
{
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// Entries (PRE false): (next_row << 1) | match; (PRE true, device copies of
// ACGT tables): (next_row << 2) | match, i.e. the table index of the next
// row's first entry, which saves a shift on every step.
template <bool PRE>
__device__ __forceinline__ uint32_t row_base(uint32_t e)
{
    return PRE ? (e & ~3u) : ((e >> 1) << 2);
}

// DFA walk over one lane's register text, ACGT-like alphabet. For every step
// calls on_step(step, idx, e): idx the table index used, e the entry read
// (bit 0 set when the transition entered a terminal state). Per byte, t is
// 0xFFFFFFFC | class for a byte of the alphabet and just the class (row 0,
// whose entries all lead to the root) for any other byte; the next index is
// then (row base & t & ~3) | (t & 3).
template <int NV, bool PRE, class Tab, class F>
__device__ __forceinline__ void walk_dna(const uint4 (&tv)[NV], int steps, uint32_t lut,
                                         const Tab &tab, F &&on_step)
{
    uint32_t e = PRE ? 4u : 2u;  // root (row 1)
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
            const uint32_t a4v = a4 | (vb & 0xFCFCFCFCu);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int step = v * 16 + q * 4 + k;
                if (step < kChunk || step < steps) {
                    const uint32_t t = __byte_perm(
                        a4v, vb, (k) | ((4 + k) << 4) | ((4 + k) << 8) | ((4 + k) << 12));
                    const uint32_t base = PRE ? e : (e << 1);
                    const uint32_t idx = (base & t & ~3u) | (t & 3u);
                    e = tab(idx);
                    on_step(step, idx, e);
                }
            }
        }
    }
}

// General alphabet: class map in shared memory; steps already clipped to n.
template <int NV, class Tab, class F>
__device__ __forceinline__ void walk_gen(const uint4 (&tv)[NV], int steps, int lw,
                                         const uint8_t *s_cls, const Tab &tab, F &&on_step)
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
                    on_step(step, idx, e);
                }
            }
        }
    }
}

// Rolled re-walk of one lane's chunk straight from global memory, for the
// rare lanes whose hit pool overflowed; same transitions as the fast walks.
// Calls hit(step, idx) for every match.
template <bool PRE = false, class Tab, class F>
__device__ __forceinline__ void walk_slow(const uint8_t *text, long long n, long long g0,
                                          int steps, bool dna, uint32_t lut, int lw,
                                          const uint8_t *s_cls, const Tab &tab, F &&hit)
{
    uint32_t e = PRE ? 4u : 2u;
#pragma unroll 1
    for (int step = 0; step < steps; ++step) {
        const long long g = g0 + step;
        if (g >= n) break;
        const uint32_t b = text[g];
        uint32_t idx;
        if (dna) {
            const uint32_t c = ((b >> 1) ^ (b >> 2)) & 3u;
            idx = ((lut >> (8 * c)) & 0xFFu) == b ? (row_base<PRE>(e) | c) : c;
        } else {
            const uint32_t c = s_cls[b];
            idx = c == 0xFFu ? 0u : (((e >> 1) << lw) | c);
        }
        e = tab(idx);
        if (e & 1u) hit(step, idx);
    }
}

// Iterates one lane's match steps in order from its 32-bit step bitmask.
template <int HW>
struct StepBits {
    uint32_t w[HW];
    int base;
    // -1 if no bit is left (cannot happen when called once per recorded hit)
    __device__ __forceinline__ int next()
    {
#pragma unroll
        for (int s = 0; s < HW; ++s) {
            if (w[0] != 0u) break;
#pragma unroll
            for (int j = 0; j + 1 < HW; ++j) w[j] = w[j + 1];
            w[HW - 1] = 0u;
            base += 32;
        }
        if (w[0] == 0u) return -1;
        const int b = __ffs(int(w[0])) - 1;
        w[0] &= w[0] - 1u;
        return base + b;
    }
};


}  // namespace acdev
}  // namespace pm
