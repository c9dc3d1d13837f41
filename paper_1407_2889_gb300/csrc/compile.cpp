// compile.cpp -- host-side pattern-set compiler for libpmscan.
//
// Aho-Corasick (Section 3.1): the trie is grown pattern by pattern in input
// order as in Algorithm 1 (goto function); supply (failure) links are
// computed in breadth-first order as in Algorithm 2, and at the same time
// every missing goto is filled with the transition of the supply state, so
// the result is the full DFA ("an array of size |Sigma|" per state, Section
// 3.1) and the scan never follows a supply link. States are then renumbered
// breadth-first (shallow states first, which also makes the shallow prefix
// of rows the hot part of the table), and the rows of depth-m states are
// elided: all patterns have length m, so a depth-m state t has no children,
// its transitions equal those of Supply(t), and a transition into t is
// stored as "go to Supply(t) and report t".
//
// Wu-Manber (Section 3.2, Algorithm 4): SHIFT, HASH and PREFIX over blocks
// of B characters ending at pattern position q-1, for q = m down to B.
#include <algorithm>
#include <cstring>
#include <new>

#include "pm_internal.h"

namespace pm {

static inline uint32_t dna_code(uint32_t b) { return ((b >> 1) ^ (b >> 2)) & 3u; }

// Character classes of a pattern alphabet: an ACGT-like alphabet (at most
// four bytes with distinct codes ((b >> 1) ^ (b >> 2)) & 3) is decoded
// arithmetically (dna, 4 columns, lut holds the byte of each code); any other
// alphabet gets dense class numbers and 2^lw columns.
static void set_classes(const bool present[256], AcTables &t)
{
    int nbytes = 0;
    for (int b = 0; b < 256; ++b) nbytes += present[b];
    bool dna = nbytes <= 4;
    int byte_of_code[4] = {-1, -1, -1, -1};
    for (int b = 0; b < 256 && dna; ++b) {
        if (!present[b]) continue;
        int c = int(dna_code(uint32_t(b)));
        if (byte_of_code[c] >= 0) dna = false;
        byte_of_code[c] = b;
    }
    std::memset(t.cls, 0xFF, sizeof(t.cls));
    if (dna) {
        t.dna = true;
        t.lw = 2;
        t.n_classes = 4;
        uint32_t lut = 0;
        for (int c = 0; c < 4; ++c) {
            int b = byte_of_code[c];
            if (b < 0) {
                // a byte whose own code differs from c can never pass the
                // check T == lut[code(T)] for code c
                for (b = 0; b < 256; ++b)
                    if (int(dna_code(uint32_t(b))) != c) break;
            }
            lut |= uint32_t(b) << (8 * c);
        }
        t.lut = lut;
        for (int b = 0; b < 256; ++b)
            if (present[b]) t.cls[b] = uint8_t(dna_code(uint32_t(b)));
    } else {
        int k = 0;
        for (int b = 0; b < 256; ++b)
            if (present[b]) t.cls[b] = uint8_t(k++);
        t.n_classes = k;
        int lw = 0;
        while ((1 << lw) < k) ++lw;
        t.lw = lw;
    }
}

int build_ac(const uint8_t *P, int64_t d, int32_t m, AcTables &t)
{
    if (!P || d < 1 || m < 1) return PM_EINVAL;
    if (d >= (int64_t(1) << 24) || m > 255) return PM_ETOOBIG;
    const int64_t max_states = d * int64_t(m) + 1;
    if (max_states >= (int64_t(1) << 30)) return PM_ETOOBIG;
    try {
        t = AcTables();
        t.m = m;
        t.d = d;

        // ---- character classes -------------------------------------------
        bool present[256] = {};
        for (int64_t k = 0; k < d * int64_t(m); ++k) present[P[k]] = true;
        set_classes(present, t);
        const int W = 1 << t.lw;

        // ---- goto function: the trie, states in creation order -----------
        std::vector<int32_t> go;      // state * W + class -> state, -1 = none
        std::vector<int32_t> depth;
        std::vector<int32_t> first_pat, next_pat(size_t(d), -1), last_pat;
        go.reserve(size_t(std::min<int64_t>(max_states, int64_t(1) << 26)) * W);
        auto new_state = [&](int32_t dep) {
            int32_t s = int32_t(depth.size());
            go.insert(go.end(), size_t(W), -1);
            depth.push_back(dep);
            first_pat.push_back(-1);
            last_pat.push_back(-1);
            return s;
        };
        new_state(0);
        for (int64_t r = 0; r < d; ++r) {
            const uint8_t *p = P + r * int64_t(m);
            int32_t s = 0;
            for (int32_t j = 0; j < m; ++j) {
                int c = t.cls[p[j]];
                int32_t nx = go[size_t(s) * W + c];
                if (nx < 0) {
                    nx = new_state(depth[s] + 1);
                    go[size_t(s) * W + c] = nx;
                }
                s = nx;
            }
            // Output(s) gains pattern r (kept in ascending r)
            if (last_pat[s] < 0) first_pat[s] = int32_t(r);
            else next_pat[last_pat[s]] = int32_t(r);
            last_pat[s] = int32_t(r);
        }
        const int64_t S = int64_t(depth.size());
        t.n_states = S;

        // ---- breadth-first order, supply links, full transition function -
        std::vector<int32_t> order;
        order.reserve(size_t(S));
        order.push_back(0);
        for (size_t h = 0; h < order.size(); ++h) {
            int32_t s = order[h];
            for (int c = 0; c < W; ++c) {
                int32_t nx = go[size_t(s) * W + c];
                if (nx >= 0) order.push_back(nx);
            }
        }
        std::vector<int32_t> supply(size_t(S), 0);  // depth-1 states: root
        for (int c = 0; c < W; ++c)
            if (go[size_t(c)] < 0) go[size_t(c)] = 0;  // root loops on absent characters
        for (size_t h = 1; h < order.size(); ++h) {
            int32_t s = order[h];
            int32_t f = supply[s];
            for (int c = 0; c < W; ++c) {
                // entries of s are still pure goto entries here; f is
                // shallower than s, so its row is already complete
                int32_t nx = go[size_t(s) * W + c];
                int32_t via = go[size_t(f) * W + c];
                if (nx >= 0) supply[nx] = via;   // real child
                else go[size_t(s) * W + c] = via; // missing goto -> supply's move
            }
        }

        // ---- rows: reset row 0, then non-terminal states breadth-first ----
        std::vector<int32_t> row_of(size_t(S), -1);
        int64_t rows = 1, shallow = 0;
        for (size_t h = 0; h < order.size(); ++h) {
            int32_t s = order[h];
            if (depth[s] < m) {
                row_of[s] = int32_t(rows++);
                if (depth[s] < m - 1) ++shallow;
            }
        }
        t.n_rows = rows;
        t.d0_row = 1 + shallow;
        t.n_distinct = S - (rows - 1);
        if (rows >= (int64_t(1) << 30)) return PM_ETOOBIG;

        // groups of equal patterns (terminal states reached by >= 2 ids)
        std::vector<int32_t> group_of(size_t(S), -1);
        t.grp_off.push_back(0);
        for (size_t h = 0; h < order.size(); ++h) {
            int32_t s = order[h];
            if (depth[s] != m || first_pat[s] < 0 || next_pat[first_pat[s]] < 0) continue;
            group_of[s] = int32_t(t.grp_off.size() - 1);
            for (int32_t r = first_pat[s]; r >= 0; r = next_pat[r]) t.grp_ids.push_back(uint32_t(r));
            t.grp_off.push_back(uint32_t(t.grp_ids.size()));
        }
        t.has_dups = t.grp_ids.size() > 0;

        t.table.assign(size_t(rows) << t.lw, 0u);
        t.mid.assign(size_t(rows - t.d0_row) << t.lw, 0xFFFFFFFFu);
        t.row_depth.assign(size_t(rows), 0);
        const uint32_t root_entry = uint32_t(row_of[0]) << 1;
        for (int c = 0; c < W; ++c) t.table[size_t(c)] = root_entry;
        for (size_t h = 0; h < order.size(); ++h) {
            int32_t s = order[h];
            if (depth[s] >= m) continue;
            const int64_t row = row_of[s];
            t.row_depth[size_t(row)] = depth[s];
            for (int c = 0; c < W; ++c) {
                int32_t nx = go[size_t(s) * W + c];
                uint32_t e;
                if (depth[nx] == m) {
                    e = (uint32_t(row_of[supply[nx]]) << 1) | 1u;
                    const size_t mi = size_t((row - t.d0_row) << t.lw) + size_t(c);
                    t.mid[mi] = group_of[nx] >= 0 ? (0x80000000u | uint32_t(group_of[nx]))
                                                  : uint32_t(first_pat[nx]);
                } else {
                    e = uint32_t(row_of[nx]) << 1;
                }
                t.table[size_t(row << t.lw) + size_t(c)] = e;
            }
        }
        // canonical terminal ids = rank of the match entry
        const size_t nflag = size_t(rows - t.d0_row) << t.lw;
        const size_t nwords = (nflag + 31) / 32;
        t.flag_mask.assign(nwords, 0u);
        t.flag_rank.assign(nwords + 1, 0u);
        t.canon.clear();
        for (size_t k = 0; k < nflag; ++k) {
            if (t.mid[k] != 0xFFFFFFFFu) {
                t.flag_mask[k >> 5] |= 1u << (k & 31);
                t.canon.push_back(t.mid[k]);
            }
        }
        for (size_t w = 0; w < nwords; ++w)
            t.flag_rank[w + 1] = t.flag_rank[w] + uint32_t(__builtin_popcount(t.flag_mask[w]));
        // 16-bit entries: rows and pool codes (pattern id or group | 0x8000)
        // must fit in 15 bits, table indices of match rows and terminal
        // ranks in 16
        const bool fits16 = rows <= 32768 && nflag <= 65536 && d < 32768 &&
                            t.grp_off.size() <= 32768 && t.canon.size() < 65536;
        t.entry_bytes = fits16 ? 2 : 4;
        return PM_OK;
    } catch (const std::bad_alloc &) {
        t = AcTables();
        return PM_ENOMEM;
    }
}

static inline uint32_t wm_hash(const uint8_t *s, int len)
{
    uint32_t h = 0;
    for (int k = 0; k < len; ++k) h = (h << 5) | (s[k] & 31u);
    return h;
}

// The exact-code tables of an ACGT-like set (see WmTables): the same SHIFT
// rule (the minimum over every block occurrence of m - q, initialised to
// m - B + 1) and the same HASH / PREFIX partition as Algorithm 4, with the
// 2-bit codes of the B-character block and of the B'-character prefix as h1
// and h2. A run holds the patterns of one (block, prefix) pair sorted by
// (packed pattern, r), so equal patterns are adjacent in ascending r.
static void build_wm_packed(const uint8_t *P, int64_t d, int32_t m, int32_t B, int32_t Bp,
                            const std::vector<uint32_t> &code_of, WmTables &t)
{
    t.dna = false;
    if (m > 32 || B + Bp > 6) return;
    bool present[256] = {};
    for (int64_t k = 0; k < d * int64_t(m); ++k) present[P[k]] = true;
    int byte_of_code[4] = {-1, -1, -1, -1};
    for (int b = 0; b < 256; ++b) {
        if (!present[b]) continue;
        const int c = int(dna_code(uint32_t(b)));
        if (byte_of_code[c] >= 0) return;  // two bytes share a code: not ACGT-like
        byte_of_code[c] = b;
    }
    uint32_t lut = 0;
    for (int c = 0; c < 4; ++c) {
        int b = byte_of_code[c];
        if (b < 0)  // a byte whose own code is not c never passes the check
            for (b = 0; b < 256; ++b)
                if (int(dna_code(uint32_t(b))) != c) break;
        lut |= uint32_t(b) << (8 * c);
    }
    const size_t NB = size_t(1) << (2 * B), NK = size_t(1) << (2 * (B + Bp));
    std::vector<uint8_t> shift2(NB, uint8_t(m - B + 1));
    std::vector<uint64_t> code(static_cast<size_t>(d));
    std::vector<uint32_t> key(static_cast<size_t>(d));
    std::vector<uint32_t> fill(NK + 1, 0);
    for (int64_t r = 0; r < d; ++r) {
        const uint8_t *p = P + r * int64_t(m);
        uint64_t c = 0;
        for (int32_t j = 0; j < m; ++j) c = (c << 2) | dna_code(p[j]);
        code[size_t(r)] = c;
        for (int32_t q = m; q >= B; --q) {
            uint32_t h = 0;
            for (int32_t j = q - B; j < q; ++j) h = (h << 2) | dna_code(p[j]);
            if (uint8_t(m - q) < shift2[h]) shift2[h] = uint8_t(m - q);
        }
        const uint32_t blk = uint32_t(c & (NB - 1));
        const uint32_t pre = uint32_t(c >> (2 * (m - Bp)));
        key[size_t(r)] = (blk << (2 * Bp)) | pre;
        if (code_of[size_t(r)] != 0xFFFFFFFFu) fill[key[size_t(r)] + 1]++;
    }
    for (size_t k = 0; k < NK; ++k) fill[k + 1] += fill[k];
    std::vector<uint32_t> order;
    for (int64_t r = 0; r < d; ++r)
        if (code_of[size_t(r)] != 0xFFFFFFFFu) order.push_back(uint32_t(r));
    std::sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (key[x] != key[y]) return key[x] < key[y];
        return code[x] < code[y];  // distinct patterns: distinct codes
    });
    t.shift2 = std::move(shift2);
    t.dir = std::move(fill);
    t.ccode.resize(order.size());
    t.cr.resize(order.size());
    for (size_t k = 0; k < order.size(); ++k) {
        t.ccode[k] = code[order[k]];
        t.cr[k] = code_of[order[k]];
    }
    t.lut = lut;
    t.dna = true;
}

// PFAC (failure-less Aho-Corasick): keep only the goto edges of the merged
// table -- an edge whose target is one level deeper, or a match entry (the
// edge into a depth-m terminal) -- and make every other entry 0, a dead end.
int build_pfac(const uint8_t *P, int64_t d, int32_t m, AcTables &t)
{
    const int rc = build_ac(P, d, m, t);
    if (rc) return rc;
    t.goto_only = true;
    const int64_t W = int64_t(1) << t.lw;
    for (int64_t row = 0; row < t.n_rows; ++row) {
        for (int64_t c = 0; c < W; ++c) {
            uint32_t &e = t.table[size_t(row * W + c)];
            if (row == 0) { e = 0; continue; }
            if (e & 1u) continue;
            const int64_t next = int64_t(e >> 1);
            if (t.row_depth[size_t(next)] != t.row_depth[size_t(row)] + 1) e = 0;
        }
    }
    return PM_OK;
}

int build_wm(const uint8_t *P, int64_t d, int32_t m, int32_t B, int32_t Bp, WmTables &t)
{
    if (!P || d < 1 || m < 1 || B < 1 || B > m || Bp < 1) return PM_EINVAL;
    if (B > 4 || Bp > 3) return PM_EINVAL;
    if (Bp > m) Bp = m;
    if (d >= int64_t(kWmGroup) || m > 255) return PM_ETOOBIG;
    try {
        t = WmTables();
        t.m = m; t.B = B; t.Bp = Bp; t.d = d;
        // equal patterns: sort the ids by pattern bytes (ties by id); each
        // run of equal patterns is one distinct pattern, entered once under
        // its smallest id with the code r, or kWmGroup | g for a group
        std::vector<uint32_t> code_of(static_cast<size_t>(d), 0xFFFFFFFFu);
        {
            std::vector<uint32_t> ids(static_cast<size_t>(d));
            for (int64_t r = 0; r < d; ++r) ids[size_t(r)] = uint32_t(r);
            std::stable_sort(ids.begin(), ids.end(), [&](uint32_t x, uint32_t y) {
                return std::memcmp(P + size_t(x) * m, P + size_t(y) * m, size_t(m)) < 0;
            });
            t.grp_off.assign(1, 0u);
            for (size_t a = 0; a < ids.size();) {
                size_t b = a + 1;
                while (b < ids.size() && std::memcmp(P + size_t(ids[a]) * m, P + size_t(ids[b]) * m, size_t(m)) == 0) ++b;
                if (b - a == 1) {
                    code_of[ids[a]] = ids[a];
                } else {
                    code_of[ids[a]] = kWmGroup | uint32_t(t.grp_off.size() - 1);
                    for (size_t k = a; k < b; ++k) t.grp_ids.push_back(ids[k]);
                    t.grp_off.push_back(uint32_t(t.grp_ids.size()));
                }
                ++t.n_distinct;
                a = b;
            }
            if (t.grp_ids.empty()) t.grp_off.clear();
        }
        const size_t H = size_t(1) << (5 * B);
        t.shift.assign(H, uint8_t(m - B + 1));
        std::vector<uint32_t> bucket_of(static_cast<size_t>(d));
        std::vector<uint16_t> prefix(static_cast<size_t>(d));
        std::vector<uint32_t> fill(H + 1, 0);
        for (int64_t r = 0; r < d; ++r) {
            const uint8_t *p = P + r * int64_t(m);
            for (int32_t q = m; q >= B; --q) {
                uint32_t h = wm_hash(p + (q - B), B);
                uint8_t sh = uint8_t(m - q);
                if (sh < t.shift[h]) t.shift[h] = sh;
                if (q == m) {
                    bucket_of[size_t(r)] = h;
                    prefix[size_t(r)] = uint16_t(wm_hash(p, Bp));
                    if (code_of[size_t(r)] != 0xFFFFFFFFu) fill[h + 1]++;
                }
            }
        }
        for (size_t h = 0; h < H; ++h) fill[h + 1] += fill[h];
        t.hoff = fill;
        t.hids.assign(size_t(t.n_distinct), 0);
        for (int64_t r = 0; r < d; ++r)
            if (code_of[size_t(r)] != 0xFFFFFFFFu) t.hids[fill[bucket_of[size_t(r)]]++] = uint32_t(r);
        for (size_t h = 0; h < H; ++h) {
            auto b = t.hids.begin() + t.hoff[h], e = t.hids.begin() + t.hoff[h + 1];
            std::stable_sort(b, e, [&](uint32_t x, uint32_t y) { return prefix[x] < prefix[y]; });
        }
        t.hpfx.resize(t.hids.size());
        t.hcode.resize(t.hids.size());
        for (size_t k = 0; k < t.hids.size(); ++k) {
            t.hpfx[k] = prefix[t.hids[k]];
            t.hcode[k] = code_of[t.hids[k]];
        }
        t.pats.assign(P, P + d * int64_t(m));
        t.n_zero_shift = 0;
        for (size_t h = 0; h < H; ++h) t.n_zero_shift += t.shift[h] == 0;
        build_wm_packed(P, d, m, B, Bp, code_of, t);
        return PM_OK;
    } catch (const std::bad_alloc &) {
        t = WmTables();
        return PM_ENOMEM;
    }
}

static inline void emit_entry(std::vector<uint64_t> &occ, std::vector<int64_t> &counts,
                              int64_t i, uint32_t r)
{
    occ.push_back((uint64_t(i) << 32) | r);
    counts[r]++;
}

// a Wu-Manber match code: one pattern id, or every id of a group in ascending order
static inline void emit_wm(const WmTables &t, std::vector<uint64_t> &occ, std::vector<int64_t> &counts,
                           int64_t i, uint32_t code)
{
    if (code & kWmGroup) {
        const uint32_t g = code & ~kWmGroup;
        for (uint32_t k = t.grp_off[g]; k < t.grp_off[g + 1]; ++k) emit_entry(occ, counts, i, t.grp_ids[k]);
    } else {
        emit_entry(occ, counts, i, code);
    }
}

void host_walk_ac(const AcTables &t, const uint8_t *T, int64_t n,
                  std::vector<uint64_t> &occ, std::vector<int64_t> &counts)
{
    counts.assign(size_t(t.d), 0);
    occ.clear();
    uint32_t e = 2u;  // root is row 1
    const uint32_t mid_base = uint32_t(t.d0_row << t.lw);
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t b = T[i];
        uint32_t idx;
        if (t.dna) {
            const uint32_t c = dna_code(b);
            const bool ok = ((t.lut >> (8 * c)) & 0xFFu) == b;
            idx = ok ? (((e >> 1) << 2) | c) : c;   // row 0 = reset row
        } else {
            const uint32_t c = t.cls[b];
            idx = c == 0xFFu ? 0u : (((e >> 1) << t.lw) | c);
        }
        e = t.table[idx];
        if (e & 1u) {
            const uint32_t v = t.mid[idx - mid_base];
            const int64_t pos = i - t.m + 1;
            if (v & 0x80000000u) {
                const uint32_t g = v & 0x7FFFFFFFu;
                for (uint32_t k = t.grp_off[g]; k < t.grp_off[g + 1]; ++k)
                    emit_entry(occ, counts, pos, t.grp_ids[k]);
            } else {
                emit_entry(occ, counts, pos, v);
            }
        }
    }
}

// Algorithm 5 over the exact-code tables, as the device runs it (one text,
// one walk): the same window ends, SHIFT values and verification result.
static void host_walk_wm_packed(const WmTables &t, const uint8_t *T, int64_t n,
                                std::vector<uint64_t> &occ, std::vector<int64_t> &counts)
{
    const int32_t m = t.m, B = t.B, Bp = t.Bp;
    const uint64_t mask = m >= 32 ? ~uint64_t(0) : ((uint64_t(1) << (2 * m)) - 1);
    const uint32_t bmask = (1u << (2 * B)) - 1u;
    uint64_t code = 0;
    int64_t bad = -1, skip = 0;
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t b = T[i], c = dna_code(b);
        if (((t.lut >> (8 * c)) & 0xFFu) != b) bad = i;
        code = ((code << 2) | c) & mask;
        if (i < m - 1) continue;
        if (skip > 0) { --skip; continue; }
        const uint32_t sh = bad > i - B ? uint32_t(m - B + 1) : t.shift2[uint32_t(code) & bmask];
        if (sh > 0) { skip = int64_t(sh) - 1; continue; }
        if (bad > i - m) continue;
        const uint32_t key = ((uint32_t(code) & bmask) << (2 * Bp)) | uint32_t(code >> (2 * (m - Bp)));
        for (uint32_t k = t.dir[key]; k < t.dir[key + 1]; ++k)
            if (t.ccode[k] == code) {
                emit_wm(t, occ, counts, i - m + 1, t.cr[k]);
                break;
            }
    }
}

void host_walk_pfac(const AcTables &t, const uint8_t *T, int64_t n,
                    std::vector<uint64_t> &occ, std::vector<int64_t> &counts)
{
    counts.assign(size_t(t.d), 0);
    occ.clear();
    const uint32_t mid_base = uint32_t(t.d0_row << t.lw);
    for (int64_t i = 0; i + t.m <= n; ++i) {
        uint32_t e = 2u;  // root is row 1
        for (int32_t j = 0; j < t.m; ++j) {
            const uint32_t b = T[i + j];
            uint32_t c;
            if (t.dna) {
                c = dna_code(b);
                if (((t.lut >> (8 * c)) & 0xFFu) != b) break;
            } else {
                c = t.cls[b];
                if (c == 0xFFu) break;
            }
            const uint32_t idx = ((e >> 1) << t.lw) | c;
            e = t.table[idx];
            if (e & 1u) {
                const uint32_t v = t.mid[idx - mid_base];
                if (v & 0x80000000u) {
                    const uint32_t g = v & 0x7FFFFFFFu;
                    for (uint32_t k = t.grp_off[g]; k < t.grp_off[g + 1]; ++k)
                        emit_entry(occ, counts, i, t.grp_ids[k]);
                } else {
                    emit_entry(occ, counts, i, v);
                }
                break;
            }
            if (e == 0u) break;
        }
    }
}

void host_walk_wm(const WmTables &t, const uint8_t *T, int64_t n,
                  std::vector<uint64_t> &occ, std::vector<int64_t> &counts)
{
    if (t.dna) {
        counts.assign(size_t(t.d), 0);
        occ.clear();
        host_walk_wm_packed(t, T, n, occ, counts);
        return;
    }
    counts.assign(size_t(t.d), 0);
    occ.clear();
    const int32_t m = t.m, B = t.B, Bp = t.Bp;
    int64_t i = m - 1;
    while (i < n) {
        const uint32_t h = wm_hash(T + (i - B + 1), B);
        const uint32_t sh = t.shift[h];
        if (sh > 0) {
            i += sh;
            continue;
        }
        const uint16_t hp = uint16_t(wm_hash(T + (i - m + 1), Bp));
        for (uint32_t k = t.hoff[h]; k < t.hoff[h + 1]; ++k) {
            if (t.hpfx[k] != hp) continue;
            const uint32_t r = t.hids[k];
            if (std::memcmp(t.pats.data() + size_t(r) * m, T + (i - m + 1), size_t(m)) == 0) {
                emit_wm(t, occ, counts, i - m + 1, t.hcode[k]);
                break;
            }
        }
        i += 1;
    }
}

// ---------------------------------------------------------------------------
// Mixed-length sets: Algorithms 1-2 over patterns of their own lengths. The
// trie and the supply links are built as for one length; Output(s) takes
// the patterns ending at s (ascending r) followed by Output(Supply(s))
// (breadth-first, so the supply's set is complete first). No row is elided.
// ---------------------------------------------------------------------------
int build_acv(const uint8_t *P, const int64_t *off, int64_t d, AcvTables &out)
{
    if (!P || !off || d < 1 || off[0] != 0) return PM_EINVAL;
    for (int64_t r = 0; r < d; ++r) {
        const int64_t len = off[r + 1] - off[r];
        if (len < 1) return PM_EINVAL;
        if (len > kAcvMaxLen) return PM_ETOOBIG;
    }
    if (d >= (int64_t(1) << 25)) return PM_ETOOBIG;
    const int64_t total = off[d];
    if (total + 1 >= (int64_t(1) << 30)) return PM_ETOOBIG;
    try {
        out = AcvTables();
        AcTables &t = out.ac;
        t.d = d;
        bool present[256] = {};
        for (int64_t k = 0; k < total; ++k) present[P[k]] = true;
        set_classes(present, t);
        const int W = 1 << t.lw;
        out.lens.resize(size_t(d));
        int32_t mmin = kAcvMaxLen, mmax = 0;
        for (int64_t r = 0; r < d; ++r) {
            const int32_t len = int32_t(off[r + 1] - off[r]);
            out.lens[size_t(r)] = len;
            mmin = std::min(mmin, len);
            mmax = std::max(mmax, len);
        }
        t.m = mmax;
        out.m_min = mmin;

        // ---- goto trie (Algorithm 1), patterns in input order ------------
        std::vector<int32_t> go, depth, parent, own_first, own_last;
        std::vector<int32_t> own_next(size_t(d), -1);
        auto new_state = [&](int32_t dep, int32_t par) {
            const int32_t st = int32_t(depth.size());
            go.insert(go.end(), size_t(W), -1);
            depth.push_back(dep);
            parent.push_back(par);
            own_first.push_back(-1);
            own_last.push_back(-1);
            return st;
        };
        new_state(0, 0);
        for (int64_t r = 0; r < d; ++r) {
            int32_t st = 0;
            for (int64_t j = off[r]; j < off[r + 1]; ++j) {
                const int c = t.cls[P[j]];
                int32_t nx = go[size_t(st) * W + c];
                if (nx < 0) {
                    nx = new_state(depth[st] + 1, st);
                    go[size_t(st) * W + c] = nx;
                }
                st = nx;
            }
            if (own_last[st] < 0) own_first[st] = int32_t(r);
            else own_next[own_last[st]] = int32_t(r);
            own_last[st] = int32_t(r);
        }
        const int64_t S = int64_t(depth.size());
        t.n_states = S;

        // ---- breadth-first order, supply links, full transitions (Alg. 2)
        std::vector<int32_t> order;
        order.reserve(size_t(S));
        order.push_back(0);
        for (size_t h = 0; h < order.size(); ++h)
            for (int c = 0; c < W; ++c) {
                const int32_t nx = go[size_t(order[h]) * W + c];
                if (nx >= 0) order.push_back(nx);
            }
        std::vector<int32_t> supply(size_t(S), 0);
        for (int c = 0; c < W; ++c)
            if (go[size_t(c)] < 0) go[size_t(c)] = 0;
        for (size_t h = 1; h < order.size(); ++h) {
            const int32_t st = order[h], f = supply[st];
            for (int c = 0; c < W; ++c) {
                const int32_t nx = go[size_t(st) * W + c];
                const int32_t via = go[size_t(f) * W + c];
                if (nx >= 0) supply[nx] = via;
                else go[size_t(st) * W + c] = via;
            }
        }
        // the patterns on a state's root path (prefixes of its string): the
        // most patterns that can start at one text position is their maximum
        std::vector<int32_t> chain(size_t(S), 0);
        int32_t K = 1;
        for (size_t h = 1; h < order.size(); ++h) {
            const int32_t st = order[h];
            int32_t own = 0;
            for (int32_t r = own_first[st]; r >= 0; r = own_next[r]) ++own;
            chain[size_t(st)] = chain[size_t(parent[st])] + own;
            K = std::max(K, chain[size_t(st)]);
        }
        out.K = K;

        // ---- Output(s) = own(s) + Output(Supply(s)), breadth-first -------
        std::vector<std::vector<uint32_t>> outs(static_cast<size_t>(S));
        for (size_t h = 0; h < order.size(); ++h) {
            const int32_t st = order[h];
            std::vector<uint32_t> &o = outs[size_t(st)];
            for (int32_t r = own_first[st]; r >= 0; r = own_next[r])
                o.push_back((uint32_t(r) << 7) | uint32_t(out.lens[size_t(r)]));
            if (h > 0) {
                const std::vector<uint32_t> &f = outs[size_t(supply[st])];
                o.insert(o.end(), f.begin(), f.end());
            }
            std::sort(o.begin(), o.end(), [](uint32_t x, uint32_t y) {
                const uint32_t lx = x & 127u, ly = y & 127u;
                if (lx != ly) return lx > ly;  // longer first (earlier start)
                return (x >> 7) < (y >> 7);
            });
            out.max_out = std::max(out.max_out, int32_t(o.size()));
        }

        // ---- rows: reset row 0, every state breadth-first -------------------
        std::vector<int32_t> row_of(size_t(S), -1);
        for (size_t h = 0; h < order.size(); ++h) row_of[order[h]] = int32_t(h + 1);
        const int64_t rows = S + 1;
        t.n_rows = rows;
        t.d0_row = 1;
        t.table.assign(size_t(rows) << t.lw, 0u);
        t.row_depth.assign(size_t(rows), 0);
        for (int c = 0; c < W; ++c) t.table[size_t(c)] = uint32_t(row_of[0]) << 1;  // reset row -> root
        for (size_t h = 0; h < order.size(); ++h) {
            const int32_t st = order[h];
            const int64_t row = row_of[st];
            t.row_depth[size_t(row)] = depth[st];
            for (int c = 0; c < W; ++c) {
                const int32_t nx = go[size_t(st) * W + c];
                t.table[size_t(row << t.lw) + size_t(c)] =
                    (uint32_t(row_of[nx]) << 1) | (outs[size_t(nx)].empty() ? 0u : 1u);
            }
        }
        const size_t nwords = size_t((rows + 31) / 32);
        out.omask.assign(nwords, 0u);
        out.orank.assign(nwords + 1, 0u);
        out.out_off.assign(1, 0u);
        for (int64_t row = 1; row < rows; ++row) {
            const std::vector<uint32_t> &o = outs[size_t(order[size_t(row - 1)])];
            if (o.empty()) continue;
            out.omask[size_t(row) >> 5] |= 1u << (row & 31);
            out.out_ent.insert(out.out_ent.end(), o.begin(), o.end());
            out.out_off.push_back(uint32_t(out.out_ent.size()));
        }
        for (size_t w = 0; w < nwords; ++w)
            out.orank[w + 1] = out.orank[w] + uint32_t(__builtin_popcount(out.omask[w]));
        int64_t distinct = 0;
        for (int64_t st = 0; st < S; ++st) distinct += own_first[st] >= 0;
        t.n_distinct = distinct;
        t.entry_bytes = rows <= 32768 ? 2 : 4;
        return PM_OK;
    } catch (const std::bad_alloc &) {
        out = AcvTables();
        return PM_ENOMEM;
    }
}

// One sequential pass over the DFA; every position reports its output set
// (each pattern at its own start), then the pairs are put in (i, r) order.
void host_walk_acv(const AcvTables &v, const uint8_t *T, int64_t n,
                   std::vector<uint64_t> &occ, std::vector<int64_t> &counts)
{
    const AcTables &t = v.ac;
    counts.assign(size_t(t.d), 0);
    occ.clear();
    uint32_t e = 2u;  // root is row 1
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t b = T[i];
        uint32_t idx;
        if (t.dna) {
            const uint32_t c = dna_code(b);
            idx = ((t.lut >> (8 * c)) & 0xFFu) == b ? (((e >> 1) << 2) | c) : c;
        } else {
            const uint32_t c = t.cls[b];
            idx = c == 0xFFu ? 0u : (((e >> 1) << t.lw) | c);
        }
        e = t.table[idx];
        if (!(e & 1u)) continue;
        const uint32_t row = e >> 1;
        const uint32_t w = row >> 5;
        const uint32_t rank = v.orank[w] + uint32_t(__builtin_popcount(v.omask[w] & ((1u << (row & 31)) - 1u)));
        for (uint32_t k = v.out_off[rank]; k < v.out_off[rank + 1]; ++k) {
            const uint32_t r = v.out_ent[k] >> 7, len = v.out_ent[k] & 127u;
            emit_entry(occ, counts, i - int64_t(len) + 1, r);
        }
    }
    std::sort(occ.begin(), occ.end());
}

// Exact-code tables of a mixed-length ACGT-like set (longest length <= 32,
// B + B' <= 6): those of build_wm_packed over every pattern's first m
// characters, every id kept (runs sorted by (code of the m characters, r)),
// plus each candidate's whole packed pattern and its length.
static void build_wmv_packed(const uint8_t *P, const int64_t *off, int64_t d, int32_t m, int32_t mmax,
                             int32_t B, int32_t Bp, WmTables &t)
{
    t.dna = false;
    if (mmax > 32 || B + Bp > 6) return;
    bool present[256] = {};
    for (int64_t k = 0; k < off[d]; ++k) present[P[k]] = true;
    int byte_of_code[4] = {-1, -1, -1, -1};
    for (int b = 0; b < 256; ++b) {
        if (!present[b]) continue;
        const int c = int(dna_code(uint32_t(b)));
        if (byte_of_code[c] >= 0) return;  // not ACGT-like
        byte_of_code[c] = b;
    }
    uint32_t lut = 0;
    for (int c = 0; c < 4; ++c) {
        int b = byte_of_code[c];
        if (b < 0)
            for (b = 0; b < 256; ++b)
                if (int(dna_code(uint32_t(b))) != c) break;
        lut |= uint32_t(b) << (8 * c);
    }
    const size_t NB = size_t(1) << (2 * B), NK = size_t(1) << (2 * (B + Bp));
    std::vector<uint8_t> shift2(NB, uint8_t(m - B + 1));
    std::vector<uint64_t> pre(static_cast<size_t>(d)), full(static_cast<size_t>(d));
    std::vector<uint32_t> key(static_cast<size_t>(d));
    std::vector<uint32_t> fill(NK + 1, 0);
    for (int64_t r = 0; r < d; ++r) {
        const uint8_t *p = P + off[r];
        const int32_t len = int32_t(off[r + 1] - off[r]);
        uint64_t c = 0;
        for (int32_t j = 0; j < len; ++j) {
            c = (c << 2) | dna_code(p[j]);
            if (j == m - 1) pre[size_t(r)] = c;
        }
        full[size_t(r)] = c;
        for (int32_t q = m; q >= B; --q) {
            uint32_t h = 0;
            for (int32_t j = q - B; j < q; ++j) h = (h << 2) | dna_code(p[j]);
            if (uint8_t(m - q) < shift2[h]) shift2[h] = uint8_t(m - q);
        }
        const uint64_t pc = pre[size_t(r)];
        key[size_t(r)] = (uint32_t(pc & (NB - 1)) << (2 * Bp)) | uint32_t(pc >> (2 * (m - Bp)));
        fill[key[size_t(r)] + 1]++;
    }
    for (size_t k = 0; k < NK; ++k) fill[k + 1] += fill[k];
    std::vector<uint32_t> order(static_cast<size_t>(d));
    for (int64_t r = 0; r < d; ++r) order[size_t(r)] = uint32_t(r);
    std::sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (key[x] != key[y]) return key[x] < key[y];
        if (pre[x] != pre[y]) return pre[x] < pre[y];
        return x < y;
    });
    t.shift2 = std::move(shift2);
    t.dir = std::move(fill);
    t.ccode.resize(size_t(d));
    t.cr.resize(size_t(d));
    t.fcode.resize(size_t(d));
    t.flen.resize(size_t(d));
    for (int64_t k = 0; k < d; ++k) {
        const uint32_t r = order[size_t(k)];
        t.ccode[size_t(k)] = pre[r];
        t.cr[size_t(k)] = r;
        t.fcode[size_t(k)] = full[r];
        t.flen[size_t(k)] = uint8_t(off[r + 1] - off[r]);
    }
    t.lut = lut;
    t.dna = true;
}

// ---------------------------------------------------------------------------
// Wu-Manber over mixed lengths (m = the shortest length): Algorithm 4 over
// every pattern's first m characters, HASH sorted by (PREFIX, r) with every
// id, the patterns kept whole for verification over their own lengths.
// ---------------------------------------------------------------------------
int build_wmv(const uint8_t *P, const int64_t *off, int64_t d, int32_t B, int32_t Bp, WmTables &t)
{
    if (!P || !off || d < 1 || off[0] != 0 || B < 1 || Bp < 1) return PM_EINVAL;
    int32_t mmin = kAcvMaxLen + 1, mmax = 0;
    for (int64_t r = 0; r < d; ++r) {
        const int64_t len = off[r + 1] - off[r];
        if (len < 1) return PM_EINVAL;
        if (len > kAcvMaxLen) return PM_ETOOBIG;
        mmin = std::min<int32_t>(mmin, int32_t(len));
        mmax = std::max<int32_t>(mmax, int32_t(len));
    }
    if (B > mmin || B > 4 || Bp > 3) return PM_EINVAL;
    if (Bp > mmin) Bp = mmin;
    if (d >= int64_t(kWmGroup)) return PM_ETOOBIG;
    try {
        t = WmTables();
        t.var = true;
        t.m = mmin;
        t.m_max = mmax;
        t.B = B;
        t.Bp = Bp;
        t.d = d;
        const int32_t m = mmin;
        const size_t H = size_t(1) << (5 * B);
        t.shift.assign(H, uint8_t(m - B + 1));
        std::vector<uint32_t> bucket_of(static_cast<size_t>(d));
        std::vector<uint16_t> prefix(static_cast<size_t>(d));
        std::vector<uint32_t> fill(H + 1, 0);
        for (int64_t r = 0; r < d; ++r) {
            const uint8_t *p = P + off[r];
            for (int32_t q = m; q >= B; --q) {
                const uint32_t h = wm_hash(p + (q - B), B);
                const uint8_t sh = uint8_t(m - q);
                if (sh < t.shift[h]) t.shift[h] = sh;
                if (q == m) {
                    bucket_of[size_t(r)] = h;
                    prefix[size_t(r)] = uint16_t(wm_hash(p, Bp));
                    fill[h + 1]++;
                }
            }
        }
        for (size_t h = 0; h < H; ++h) fill[h + 1] += fill[h];
        t.hoff = fill;
        t.hids.assign(size_t(d), 0);
        for (int64_t r = 0; r < d; ++r) t.hids[fill[bucket_of[size_t(r)]]++] = uint32_t(r);
        for (size_t h = 0; h < H; ++h) {
            auto b = t.hids.begin() + t.hoff[h], e = t.hids.begin() + t.hoff[h + 1];
            std::stable_sort(b, e, [&](uint32_t x, uint32_t y) { return prefix[x] < prefix[y]; });
        }
        t.hpfx.resize(size_t(d));
        t.hcode.resize(size_t(d));
        for (int64_t k = 0; k < d; ++k) {
            t.hpfx[size_t(k)] = prefix[t.hids[size_t(k)]];
            t.hcode[size_t(k)] = t.hids[size_t(k)];
        }
        t.pats.assign(P, P + off[d]);
        t.poff.assign(off, off + d + 1);
        t.n_distinct = d;
        t.n_zero_shift = 0;
        for (size_t h = 0; h < H; ++h) t.n_zero_shift += t.shift[h] == 0;
        // most patterns that are prefixes of one of them (with multiplicity)
        std::vector<int64_t> ids(static_cast<size_t>(d));
        for (int64_t r = 0; r < d; ++r) ids[size_t(r)] = r;
        std::sort(ids.begin(), ids.end(), [&](int64_t x, int64_t y) {
            const int64_t lx = off[x + 1] - off[x], ly = off[y + 1] - off[y];
            const int c = std::memcmp(P + off[x], P + off[y], size_t(std::min(lx, ly)));
            if (c) return c < 0;
            return lx < ly;
        });
        int32_t K = 1;
        std::vector<int64_t> stack;  // the chain of patterns that are prefixes of the current one
        for (int64_t r : ids) {
            const int64_t len = off[r + 1] - off[r];
            while (!stack.empty()) {
                const int64_t q = stack.back(), lq = off[q + 1] - off[q];
                if (lq <= len && std::memcmp(P + off[q], P + off[r], size_t(lq)) == 0) break;
                stack.pop_back();
            }
            stack.push_back(r);
            K = std::max<int32_t>(K, int32_t(stack.size()));
        }
        t.K = K;
        build_wmv_packed(P, off, d, mmin, mmax, B, Bp, t);
        return PM_OK;
    } catch (const std::bad_alloc &) {
        t = WmTables();
        return PM_ENOMEM;
    }
}

// Algorithm 5 over the shortest length's windows with the exact-code
// tables: the run of the window's (block, prefix) entries whose code of the
// first m characters equals the window's, in ascending r; a longer
// candidate also needs the text's next len - m bytes to extend the window's
// code to its whole packed pattern.
static void host_walk_wmv_packed(const WmTables &t, const uint8_t *T, int64_t n,
                                 std::vector<uint64_t> &occ, std::vector<int64_t> &counts)
{
    const int32_t m = t.m, B = t.B, Bp = t.Bp;
    const uint64_t mask = m >= 32 ? ~uint64_t(0) : ((uint64_t(1) << (2 * m)) - 1);
    const uint32_t bmask = (1u << (2 * B)) - 1u;
    auto ok = [&](uint32_t b) { return ((t.lut >> (8 * dna_code(b))) & 0xFFu) == b; };
    uint64_t code = 0;
    int64_t bad = -1, skip = 0;
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t b = T[i];
        if (!ok(b)) bad = i;
        code = ((code << 2) | dna_code(b)) & mask;
        if (i < m - 1) continue;
        if (skip > 0) { --skip; continue; }
        const uint32_t sh = bad > i - B ? uint32_t(m - B + 1) : t.shift2[uint32_t(code) & bmask];
        if (sh > 0) { skip = int64_t(sh) - 1; continue; }
        if (bad > i - m) continue;
        const uint32_t key = ((uint32_t(code) & bmask) << (2 * Bp)) | uint32_t(code >> (2 * (m - Bp)));
        for (uint32_t k = t.dir[key]; k < t.dir[key + 1]; ++k) {
            if (t.ccode[k] < code) continue;
            if (t.ccode[k] > code) break;
            const int64_t len = t.flen[k], start = i - m + 1;
            if (start + len > n) continue;
            uint64_t ext = code;
            bool good = true;
            for (int64_t j = i + 1; j < start + len && good; ++j) {
                good = ok(T[j]);
                ext = (ext << 2) | dna_code(T[j]);
            }
            if (good && ext == t.fcode[k]) emit_entry(occ, counts, start, t.cr[k]);
        }
    }
}

// Algorithm 5 over the shortest length's windows; every candidate whose
// whole pattern fits and equals the text is reported at the window start.
void host_walk_wmv(const WmTables &t, const uint8_t *T, int64_t n,
                   std::vector<uint64_t> &occ, std::vector<int64_t> &counts)
{
    counts.assign(size_t(t.d), 0);
    occ.clear();
    if (t.dna) {
        host_walk_wmv_packed(t, T, n, occ, counts);
        return;
    }
    const int32_t m = t.m, B = t.B, Bp = t.Bp;
    int64_t i = m - 1;
    while (i < n) {
        const uint32_t h = wm_hash(T + (i - B + 1), B);
        const uint32_t sh = t.shift[h];
        if (sh > 0) {
            i += sh;
            continue;
        }
        const int64_t start = i - m + 1;
        const uint16_t hp = uint16_t(wm_hash(T + start, Bp));
        for (uint32_t k = t.hoff[h]; k < t.hoff[h + 1]; ++k) {
            if (t.hpfx[k] != hp) continue;
            const uint32_t r = t.hids[k];
            const int64_t len = t.poff[r + 1] - t.poff[r];
            if (start + len > n) continue;
            if (std::memcmp(t.pats.data() + t.poff[r], T + start, size_t(len)) == 0)
                emit_entry(occ, counts, start, r);
        }
        i += 1;
    }
}

// ---------------------------------------------------------------------------
// Two characters per lookup (the multi-character table of the DFA form of
// Section 3.1): the one-character table composed with itself.
// ---------------------------------------------------------------------------
bool ac2_eligible(const AcTables &t)
{
    return t.dna && t.entry_bytes == 2 && t.n_rows <= 4096 && t.m >= 1 && t.m - 1 <= 32 && !t.table.empty();
}

void build_ac2(AcTables &t)
{
    t.table2.clear();
    if (!ac2_eligible(t)) return;
    t.table2.assign(size_t(t.n_rows) * 16, 0);
    for (int64_t r = 0; r < t.n_rows; ++r)
        for (uint32_t c1 = 0; c1 < 4; ++c1) {
            const uint32_t e1 = t.table[size_t(r) * 4 + c1];
            const uint32_t r1 = e1 >> 1, m1 = e1 & 1u;
            for (uint32_t c2 = 0; c2 < 4; ++c2) {
                const uint32_t e2 = t.table[size_t(r1) * 4 + c2];
                t.table2[size_t(r) * 16 + c1 * 4 + c2] = uint16_t(((e2 >> 1) << 4) | (m1 << 1) | (e2 & 1u));
            }
        }
}

// The two-character walk as the device runs it: a pair (b1, b2) moves the
// state to table2[row * 16 + c1 * 4 + c2] (flags: bit 1 after c1, bit 0
// after c2). A byte outside the alphabet
// resets the walk: as b1 it selects row 0 (after a reset byte: the entry of
// (c1, c2) is the root's transition on c2, whatever c1), as b2 it sends the
// state to the root after the pair and drops the pair's second flag.
void host_walk_ac2(const AcTables &t, const uint8_t *T, int64_t n,
                   std::vector<uint64_t> &occ, std::vector<int64_t> &counts)
{
    counts.assign(size_t(t.d), 0);
    occ.clear();
    const int64_t m = t.m;
    const uint32_t mid_base = uint32_t(t.d0_row << t.lw);
    auto bad = [&](uint32_t b) { return ((t.lut >> (8 * dna_code(b))) & 0xFFu) != b; };
    auto report = [&](int64_t j, uint32_t idx1) {
        const uint32_t v = t.mid[idx1 - mid_base];
        const int64_t pos = j - m + 1;
        if (v & 0x80000000u) {
            const uint32_t g = v & 0x7FFFFFFFu;
            for (uint32_t k = t.grp_off[g]; k < t.grp_off[g + 1]; ++k) emit_entry(occ, counts, pos, t.grp_ids[k]);
        } else {
            emit_entry(occ, counts, pos, v);
        }
    };
    uint32_t E = 16u;  // the root: row 1, as an index of its first entry
    for (int64_t i = 0; i < n; i += 2) {
        const uint32_t b1 = T[i];
        const bool last = i + 1 >= n;          // the text ends inside this pair
        const uint32_t b2 = last ? 0u : T[i + 1];
        const uint32_t c1 = dna_code(b1), c2 = dna_code(b2);
        const uint32_t row = bad(b1) ? 0u : (E & ~15u);
        const uint32_t idx2 = row | (c1 << 2) | c2;
        E = t.table2[idx2];
        if (last || bad(b2)) E = (E & 2u) | 16u;   // keep the first character's flag
        if (E & 2u) report(i, idx2 >> 2);
        if (E & 1u) {
            const uint32_t e1 = t.table[idx2 >> 2];
            report(i + 1, ((e1 >> 1) << 2) | c2);
        }
    }
}

}  // namespace pm
