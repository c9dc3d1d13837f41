// pm_internal.h -- shared declarations of libpmscan (host compiler, C ABI,
// kernel launchers). Not installed; the public interface is include/pmscan.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "pmscan.h"

namespace pm {

// ---------------------------------------------------------------------------
// Aho-Corasick DFA (Section 3.1, Algorithms 1-2 merged into one table).
//
// Layout of the transition table: row 0 is a "reset" row whose entries all
// lead to the root (used for bytes outside the pattern alphabet); rows
// 1..n_rows-1 are the non-terminal trie states in breadth-first order (root
// is row 1). An entry is (next_row << 1) | match, where match says the
// transition entered a depth-m (terminal) state t; next_row is then the row
// of Supply(t), whose outgoing transitions equal t's (t has no children), so
// t's own row is never stored. Only rows of depth m-1 can hold match
// entries; they are the last rows, from d0_row on. For a match entry at
// index idx = row * W + code, mid[idx - d0_row * W] names what matched:
// bit 31 clear -> the pattern id r; set -> a group g of equal patterns whose
// ids are grp_ids[grp_off[g] .. grp_off[g+1]).
// ---------------------------------------------------------------------------
struct AcTables {
    int32_t m = 0;
    int64_t d = 0;
    bool dna = false;        // ACGT-like alphabet decoded arithmetically
    uint32_t lut = 0;        // dna: byte for code c in byte c of lut
    uint8_t cls[256];        // general: class of each byte, 0xFF = absent
    int32_t n_classes = 0;
    int32_t lw = 0;          // log2 of the row width W
    int64_t n_states = 0;    // trie states including terminals
    int64_t n_rows = 0;      // table rows (reset row + non-terminal states)
    int64_t d0_row = 0;      // first row holding match entries
    int64_t n_distinct = 0;  // distinct patterns (= terminal states)
    bool has_dups = false;
    bool goto_only = false;  // PFAC: every non-goto entry dead
    int32_t entry_bytes = 2;
    std::vector<uint32_t> table;   // n_rows << lw encoded entries
    std::vector<uint32_t> mid;     // (n_rows - d0_row) << lw
    std::vector<uint32_t> grp_off; // groups of >= 2 equal patterns
    std::vector<uint32_t> grp_ids;
    std::vector<int32_t> row_depth; // depth of each row's state (row 0: 0)
    // Canonical terminal ids: each terminal state is entered by exactly one
    // table entry (the trie edge into it), so numbering terminals in the
    // order of those entries makes a terminal's id the rank of its entry
    // among the match entries. flag_mask has one bit per entry of the match
    // rows (from d0_row on), flag_rank the number of set bits before each
    // 32-entry word, canon[c] the pattern id of terminal c, or
    // 0x80000000 | group when several patterns are equal.
    std::vector<uint32_t> flag_mask;
    std::vector<uint32_t> flag_rank;
    std::vector<uint32_t> canon;
    // Two characters per lookup (ACGT sets of at most 4096 rows, m <= 33):
    // row r, classes (c1, c2) -> (r2 << 4) | (m1 << 1) | m2, where r1 and m1
    // are the state and flag after c1 and r2, m2 those after c2 (the
    // one-character table applied twice). Empty when not eligible.
    std::vector<uint16_t> table2;
};

// ---------------------------------------------------------------------------
// Wu-Manber tables (Section 3.2, Algorithm 4). h1 over B bytes and h2 over
// B' bytes: h = (h << 5) | (byte & 31). HASH is stored as CSR buckets over
// h1 values; inside a bucket the pattern ids are sorted by (PREFIX, r), so
// the candidates with PREFIX[r] = h' form one contiguous run in ascending r.
// ---------------------------------------------------------------------------
struct WmTables {
    int32_t m = 0, B = 0, Bp = 0;
    int64_t d = 0;
    std::vector<uint8_t> shift;    // 2^(5B) entries, values <= m-B+1 <= 255
    std::vector<uint32_t> hoff;    // 2^(5B)+1 bucket offsets
    std::vector<uint32_t> hids;    // d pattern ids, bucket-major
    std::vector<uint16_t> hpfx;    // PREFIX of hids[k]
    std::vector<uint8_t> pats;     // d*m pattern bytes
    int64_t n_zero_shift = 0;
    // Equal patterns: only the smallest id of each distinct pattern enters
    // HASH (and the exact-code runs); what a match there reports is a code,
    // the pattern id r, or kWmGroup | g for a group g of equal patterns whose
    // ids are grp_ids[grp_off[g] .. grp_off[g+1]) in ascending order. A
    // window then matches at most one distinct pattern.
    std::vector<uint32_t> hcode;   // code of hids[k]
    std::vector<uint32_t> grp_off;
    std::vector<uint32_t> grp_ids;
    int64_t n_distinct = 0;
    // ACGT-like sets with m <= 32 (and B + B' <= 6) also get tables over the
    // exact 2-bit codes of the blocks (an injective h1 / h2): SHIFT over the
    // 4^B blocks, a directory of the candidate runs of each (block, prefix)
    // pair, and each candidate's whole pattern packed 2 bits per character
    // (first character in the high bits), so that verification is one
    // comparison with the window's packed code.
    bool dna = false;
    uint32_t lut = 0;              // byte of code c in byte c
    std::vector<uint8_t> shift2;   // 4^B
    std::vector<uint32_t> dir;     // 4^(B+B') + 1 run offsets, key = block << 2B' | prefix
    std::vector<uint64_t> ccode;   // distinct packed patterns, run order (ascending code)
    std::vector<uint32_t> cr;      // their codes (pattern id or kWmGroup | g)
    // Mixed lengths (pm_wmv_compile): m is the shortest length; SHIFT, HASH
    // and PREFIX are those of every pattern's first m characters, HASH holds
    // every id (no group codes: the matches at one start are reported in
    // ascending r), and a candidate is verified over its own length.
    bool var = false;
    int32_t m_max = 0;
    std::vector<int64_t> poff;     // pattern r is pats[poff[r] .. poff[r+1])
    int32_t K = 1;                 // most patterns that can start at one position
    // mixed lengths on an ACGT-like set (longest length <= 32): the exact-code
    // tables keyed by the first m characters (dir, shift2, ccode = the code
    // of those m characters, cr = r, runs sorted by (code, r)), plus each
    // candidate's whole packed pattern and its length
    std::vector<uint64_t> fcode;
    std::vector<uint8_t> flen;
};
constexpr uint32_t kWmGroup = 0x800000u;  // codes fit 24 bits: d < 2^23

// ---------------------------------------------------------------------------
// Aho-Corasick over a set whose patterns have their own lengths (the
// Section 1 definition with each pattern's length for m). The DFA keeps a
// row for every trie state (no terminal elision: a terminal may have
// children); an entry is (next_row << 1) | flag, the flag set when the
// next state's output set is not empty. Output(s) = the patterns ending at
// s plus Output(Supply(s)) (Algorithm 2's output propagation), so a
// position reports every pattern that ends there. Rows with an output set
// are numbered by a bitmap with per-word prefix counts; their outputs are a
// CSR list of (r << 7) | len, longer patterns first, then ascending r.
// ---------------------------------------------------------------------------
struct AcvTables {
    AcTables ac;                   // classes, table, n_rows, entry_bytes (m = longest length)
    int32_t m_min = 0;
    std::vector<int32_t> lens;     // per pattern
    std::vector<uint32_t> omask;   // one bit per row: Output not empty
    std::vector<uint32_t> orank;   // set bits before each word
    std::vector<uint32_t> out_off; // CSR over the output rows, in rank order
    std::vector<uint32_t> out_ent; // (r << 7) | len
    int32_t K = 1;                 // most patterns that can start at one position
    int32_t max_out = 1;           // largest output set
};
constexpr int32_t kAcvMaxLen = 65; // the halo of the scan kernels (64 bytes)

int build_ac(const uint8_t *P, int64_t d, int32_t m, AcTables &out);
// pattern r is P[off[r] .. off[r+1]); lengths 1..kAcvMaxLen
int build_acv(const uint8_t *P, const int64_t *off, int64_t d, AcvTables &out);
void host_walk_acv(const AcvTables &t, const uint8_t *T, int64_t n,
                   std::vector<uint64_t> &occ, std::vector<int64_t> &counts);
int build_wm(const uint8_t *P, int64_t d, int32_t m, int32_t B, int32_t Bp, WmTables &out);
// pattern r is P[off[r] .. off[r+1]); 1 <= B <= shortest length, lengths <= kAcvMaxLen
int build_wmv(const uint8_t *P, const int64_t *off, int64_t d, int32_t B, int32_t Bp, WmTables &out);
// PFAC: build_ac, then every entry that is not a goto edge becomes 0 (dead)
int build_pfac(const uint8_t *P, int64_t d, int32_t m, AcTables &out);

// host walks used by pm_selfcheck_host_walk
// the two-character table of an eligible set (fills t.table2)
bool ac2_eligible(const AcTables &t);
void build_ac2(AcTables &t);
// the two-character walk as the device runs it (bytes outside the alphabet
// walked under their class, matches whose window holds one dropped)
void host_walk_ac2(const AcTables &t, const uint8_t *T, int64_t n,
                   std::vector<uint64_t> &occ, std::vector<int64_t> &counts);
void host_walk_ac(const AcTables &t, const uint8_t *T, int64_t n,
                  std::vector<uint64_t> &occ, std::vector<int64_t> &counts);
void host_walk_wm(const WmTables &t, const uint8_t *T, int64_t n,
                  std::vector<uint64_t> &occ, std::vector<int64_t> &counts);
void host_walk_wmv(const WmTables &t, const uint8_t *T, int64_t n,
                   std::vector<uint64_t> &occ, std::vector<int64_t> &counts);
void host_walk_pfac(const AcTables &t, const uint8_t *T, int64_t n,
                    std::vector<uint64_t> &occ, std::vector<int64_t> &counts);

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------
constexpr int kLane = 32;
constexpr int kChunk = 80;          // start positions owned by one lane (L)
constexpr int kWarpTile = kLane * kChunk;

struct AcLaunch;                    // defined in scan_ac.cu
struct WmLaunch;

// Everything a launcher needs about the device copy of a set.
struct DevAc {
    void *table = nullptr;          // entry_bytes * (n_rows << lw)
    uint32_t *grp_off = nullptr;
    uint32_t *grp_ids = nullptr;
    uint8_t *cls = nullptr;         // 256 bytes
    uint32_t *flag_mask = nullptr;
    void *flag_rank = nullptr;      // u16 or u32 per mask word (entry_bytes)
    void *canon = nullptr;          // u16 or u32 per terminal (entry_bytes)
    uint32_t *tmul = nullptr;       // 2 bits per terminal: min(multiplicity - 1, 3)
    uint32_t *emul = nullptr;       // 2 bits per match entry: the same for the terminal it enters
    int64_t smem_entries = 0;       // table entries copied to shared memory
    int32_t warps = 0, ctas_per_sm = 0, pool_cap = 0;
    int32_t hist_smem = 0;          // per-terminal counters in shared memory
    // 1: rank structure and canon in shared memory; 2 (late ids): in counts
    // mode rank structure and 2-bit multiplicities per terminal there, canon
    // in device memory; in list mode only 2-bit multiplicities per match
    // entry there, and the slots carry match-entry offsets that the expand
    // kernel maps to terminal ids and pattern codes and counts (hist_smem
    // then applies to counts mode only)
    int32_t ids_smem = 0;
    int32_t nv = 0, hv = 0;         // register text vectors (chunk + halo)
    int32_t variant = 0;            // kernel instance id
    int32_t pre = 0;                // ACGT table stored on the device as (next_row << 2) | match
    int64_t smem_bytes = 0;
    // list mode; with late ids its layout has no counters, so it may run more
    // warps than counts mode (warps, variant and smem_bytes above)
    int32_t warps_list = 0, variant_list = 0;
    int64_t smem_bytes_list = 0;
    int32_t placement = 0;
    int64_t max_warps = 0;          // warps in the largest grid a launch uses
};

// Plan and table of the two-character AC scan (scan_ac2.cu).
struct DevAc2 {
    void *table2 = nullptr;         // u16, n_rows * 16
    bool use = false;               // pm_params.stride == 2
    int32_t warps = 0, pool_cap = 0, hist_smem = 0, hv = 0, nv = 0;
    int64_t smem_bytes = 0;
};

struct DevAcv {
    void *table = nullptr;          // entry_bytes * (n_rows << lw), index entries for ACGT sets
    uint8_t *cls = nullptr;
    uint32_t *omask = nullptr, *orank = nullptr, *out_off = nullptr, *out_ent = nullptr;
    int64_t smem_entries = 0;
    int32_t warps = 0, pool_cap = 0, hist_smem = 0, hv = 0, entry_bytes = 0, pre = 0, variant = 0;
    int32_t placement = 0, omask_smem = 0;
    int64_t smem_bytes = 0;
};

struct DevWm {
    uint8_t *shift = nullptr;
    uint32_t *hoff = nullptr;
    uint32_t *hids = nullptr;
    uint16_t *hpfx = nullptr;
    uint8_t *pats = nullptr;
    uint8_t *shift2 = nullptr;      // exact-code tables (WmTables::dna)
    uint32_t *dir = nullptr;
    uint64_t *ccode = nullptr;
    uint32_t *cr = nullptr;
    uint32_t *hcode = nullptr;      // code of each HASH entry
    int64_t *poff = nullptr;        // mixed lengths: pattern offsets
    uint64_t *fcode = nullptr;      // mixed lengths, exact codes: whole packed patterns
    uint8_t *flen = nullptr;
    uint32_t *grp_off = nullptr;    // groups of equal patterns
    uint32_t *grp_ids = nullptr;
    int32_t warps = 0, ctas_per_sm = 0, pool_cap = 0;
    int32_t shift_smem = 0, hist_smem = 0, dna = 0;
    int64_t smem_bytes = 0;
};

// Workspace (device scratch) of a plain scan: a 256-byte header (status
// word, finished-CTA count) first; the list-mode layout is ListParts below.
constexpr int64_t kWsHeader = 256;
int64_t warp_tiles(int64_t n);

struct DeviceProps {
    int sm_count = 0;
    int smem_optin = 0;   // max dynamic shared memory per block
    int smem_per_sm = 0;
    int l2_bytes = 0;
};
int device_props(DeviceProps &p);
// raise a kernel's dynamic shared memory limit on the current device (once
// per device, kernel and size; thread-safe)
int kernel_smem_attr(const void *fn, int64_t bytes);

// Plan and launch. Return PM_* codes; PM_ECUDA records the CUDA error.
int ac_plan(const AcTables &t, const pm_params &opt, const DeviceProps &dp, DevAc &dev);
int ac_launch(const AcTables &t, const DevAc &dev, const uint8_t *d_text, int64_t n,
              bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap,
              int64_t *d_n_occ, void *d_ws, void *stream);
// allocation-free variant: scratch from a fixed device array in the library
int ac_launch_noalloc(const AcTables &t, const DevAc &dev, const uint8_t *d_text, int64_t n,
                      bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap,
                      int64_t *d_n_occ, void *stream);
int64_t ac_noalloc_limit_bytes();
// status word of the last allocation-free scan on the current device
int ac_noalloc_status(void *stream);
// One piece of a longer Aho-Corasick / PFAC scan (the text split with an
// m-1 halo, as Section 4.3 splits it over nodes): the first piece zeroes the
// results, later ones add to them; keys go after *occ_base keys with
// positions shifted by pos_base; *d_n_occ receives the running total.
int ac_launch_piece(const AcTables &t, const DevAc &dev, bool pfac, const uint8_t *d_text, int64_t n,
                    bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ,
                    void *d_ws, void *stream, bool first, const unsigned long long *occ_base,
                    unsigned long long pos_base);
// PFAC scan (scan_ac.cu): same tables layout, workspace and outputs as AC
int pfac_launch(const AcTables &t, const DevAc &dev, const uint8_t *d_text, int64_t n,
                bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap,
                int64_t *d_n_occ, void *d_ws, void *stream);
// device workspace of an Aho-Corasick scan of n bytes
int64_t ac_workspace_bytes(const AcTables &t, int64_t n, bool list);

// List mode shared by the Aho-Corasick and Wu-Manber scans (scan_ac.cu):
// the scan kernel writes each warp tile's entries ((start offset in the
// tile << shift) | code, in text order) into the tile's slot, the tile's
// entry and key counts, and adds the key count to its segment's sum; the
// expand kernel turns the slots into sorted keys. Workspace:
//   [header][per-terminal counters u64 x nterms][segment sums] -- zeroed
//   [tile entries u32][tile keys u32][slots: kWarpTile entries per tile]
struct ListParts {
    int64_t zeroed_bytes = 0;
    unsigned long long *seg_sum = nullptr;
    uint32_t *tile_ent = nullptr, *tile_out = nullptr;
    void *slots = nullptr;
    int64_t seg_tiles = 0;
};
int64_t list_workspace_bytes(int64_t nsub, bool list, int64_t nterms, int slot_entry_bytes);
void list_workspace_parts(void *d_ws, int64_t nsub, int64_t nterms, int slot_entry_bytes, ListParts &out);
// slots of 4-byte entries hold (offset << 16) | 16-bit code (group flag
// 0x8000), 8-byte entries (offset << 32) | 32-bit code (group flag 2^31).
// With `late` (late ids) the low half is a match-entry offset instead: the
// expand kernel takes its rank in the match bitmap (the terminal id), maps
// that through canon (entry-sized: u16 for 4-byte slots), counts it into the
// workspace's per-terminal counters, and its last CTA writes counts[r] (d
// entries) from them.
struct ExpandLate {
    const void *canon = nullptr;
    const uint32_t *mask = nullptr;  // match-entry bitmap and its ranks (type of canon)
    const void *rank = nullptr;
    int64_t nterms = 0, nwords = 0;
    int64_t *counts = nullptr;
};
int expand_launch(void *d_ws, int64_t nsub, int64_t nterms, int slot_entry_bytes, const uint32_t *grp_off,
                  const uint32_t *grp_ids, int64_t n_grp_off, int64_t n_grp_ids, uint64_t *d_occ,
                  int64_t occ_cap, int64_t *d_n_occ, const unsigned long long *occ_base,
                  unsigned long long pos_base, void *stream, const ExpandLate *late = nullptr);
// two characters per lookup (scan_ac2.cu): plan (PM_ETOOBIG if the set is
// not eligible or the tables do not fit) and scan on the AC workspace
int ac2_plan(const AcTables &t, const pm_params &opt, const DeviceProps &dp, DevAc2 &dev);
int ac2_launch(const AcTables &t, const DevAc &dv, const DevAc2 &d2, const uint8_t *d_text, int64_t n,
               bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
               void *stream);
// mixed-length Aho-Corasick (scan_acv.cu)
int acv_plan(const AcvTables &v, const pm_params &opt, const DeviceProps &dp, DevAcv &dev);
int64_t acv_workspace_bytes(const AcvTables &v, int64_t n, bool list);
int acv_launch(const AcvTables &v, const DevAcv &dv, const uint8_t *d_text, int64_t n, bool list,
               int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap, int64_t *d_n_occ, void *d_ws,
               void *stream);
// list mode of the mixed-length scans: slots of kWarpTile * per_pos entries
// per tile, (start << 20) | r (4 bytes) or (start << 32) | r (8 bytes), each
// lane's run sorted by (start, r) while the keys are written
int sorted_expand_launch(void *d_ws, int64_t nsub, int slot_bytes, int per_pos, uint64_t *d_occ,
                         int64_t occ_cap, int64_t *d_n_occ, void *stream);
// device workspace of a Wu-Manber scan of n bytes (scan_wm.cu)
int64_t wm_workspace_bytes(const WmTables &t, int64_t n, bool list);
int wm_plan(const WmTables &t, const pm_params &opt, const DeviceProps &dp, DevWm &dev);
int wm_launch(const WmTables &t, const DevWm &dev, const uint8_t *d_text, int64_t n,
              bool list, int64_t *d_counts, uint64_t *d_occ, int64_t occ_cap,
              int64_t *d_n_occ, void *d_ws, void *stream);

void set_cuda_error(int err);
// a library-owned result (plain host arrays), released by pm_result_free
pm_result *make_result(int64_t d, int64_t n_occ, bool list);
// a result whose arrays came from another allocator: pm_result_free hands
// them to release(ctx, counts, occ)
typedef void (*ResultRelease)(void *ctx, void *counts, void *occ);
pm_result *make_result_owned(int64_t d, int64_t n_occ, int64_t *counts, uint64_t *occ,
                             ResultRelease release, void *ctx);

}  // namespace pm

struct pm_set;

namespace pm {

// ---------------------------------------------------------------------------
// Batched Aho-Corasick scan (scan_batch.cu): many (text, set) instances in
// one persistent launch. Offsets are relative to the base pointers given to
// batch_launch_raw: bytes for the text, elements for counts and occ.
// ---------------------------------------------------------------------------
struct BatchDesc {                 // one instance, in processing order
    long long text_off, n;         // text bytes [text_off, text_off + n)
    long long count_off;           // counts of the instance start here (d entries)
    long long occ_off, occ_cap;    // occurrence keys go here (capacity occ_cap)
    long long ccount_off;          // into the workspace, when counters are global
    long long out_slot;            // n_occ[out_slot] receives the total
    const void *table;
    const uint32_t *mask;
    const void *rank;
    const void *canon;
    const uint32_t *grp_off;
    const uint32_t *grp_ids;
    int smem_entries, eb, m, nwords, nterms, d;
    int ids_off, hist_off;         // byte offsets in the CTA's table region; -1 = global
    uint32_t mid_base, lut, pad, pre;  // pre: DevAc::pre of the set
    int resident;                  // the whole table is in the CTA's shared memory
    // A large instance is split into parts, one queue item each: the part
    // scans warp tiles [t_lo, t_hi) of the instance. Parts add their counts
    // into the instance's device counters (ccount_off), publish their output
    // totals at workspace word pstat_off + part, and the last part to finish
    // (word done_off counts them) writes the instance's counts and total.
    // In list mode a part writes its keys, while it walks, to staging words
    // [spill_off, spill_off + spill_cap) after the counters, and copies them
    // into place once the parts before it have published their totals; a
    // part whose keys do not fit walks its tiles again to write them.
    long long t_lo, t_hi;
    long long pstat_off, done_off;
    long long spill_off, spill_cap;
    int part, nparts;
};

struct BatchShape {                // launch shape and shared-memory split
    int warps = 12;
    // where an instance whose tables do not all fit puts its ids and
    // counters: 0 shared memory while each takes at most a quarter of the
    // region, 1 device memory (the table prefix gets the whole region)
    int policy = 0;
    int region_bytes = 0;          // per-CTA table / ids / counters region
    long long smem_bytes = 0;
    int sm_count = 0;
};

struct BatchInst {
    const pm_set *set;
    int64_t text_off, text_len, count_off, occ_off, occ_cap, out_slot;
};

int batch_shape(int warps, BatchShape &out);
bool batch_supports(const pm_set *s);   // AC, ACGT-like alphabet, m <= 65, device tables
// Descriptors of k instances in the order given, one per instance (out may
// be NULL); returns the number of global counter words the workspace needs.
int64_t batch_fill(const BatchInst *inst, int k, const BatchShape &sh, BatchDesc *out);
// Queue items of k instances: the instances ordered by estimated cost (text
// bytes, weighted up for tables read through L2), costliest first, and each
// instance costing more than about a quarter of a CTA's share of the batch
// split into parts of whole warp tiles (at least two rounds of the CTA's
// warps each). Returns the global counter words the workspace needs; in list
// mode *spill_words receives the key staging words of the parts, which
// follow the counters and need no clearing.
int64_t batch_items(const BatchInst *inst, int k, const BatchShape &sh, bool list, std::vector<BatchDesc> &out,
                    int64_t *spill_words);
inline int64_t batch_ws_bytes(int64_t ccount_words) { return kWsHeader + 8 * ccount_words; }
// An upper bound on the workspace words (counters, part words and key
// staging) one instance adds to any batch_items plan of the shape,
// whatever the rest of the batch (list: the instance's keys are listed).
int64_t batch_words_bound(const BatchInst &I, const BatchShape &sh, bool list);
// Queue items of a batch of k instances fit at most this many descriptors.
inline int64_t batch_items_bound(int64_t k, const BatchShape &sh) { return 2 * k + 4 * int64_t(sh.sm_count) + 16; }
int batch_prepare_launch(const BatchShape &sh);  // host-side set-up, before any capture
int batch_launch_raw(const BatchDesc *d_desc, int k, const uint8_t *text, int64_t *counts,
                     uint64_t *occ, int64_t *n_occ, void *ws, int64_t ccount_total,
                     const BatchShape &sh, bool list, void *stream);

}  // namespace pm

// The opaque handle of the C ABI.
struct pm_set {
    int32_t algo = 0;
    pm_params params{};
    bool host_only = false;
    pm::AcTables ac;
    pm::WmTables wm;
    pm::AcvTables acv;               // PM_ALGO_ACV
    pm::DevAc dac;
    pm::DevWm dwm;
    pm::DevAcv dacv;
    pm::DevAc2 dac2;
    int64_t device_bytes = 0;
    // caches for pm_scan (host-pointer convenience path)
    void *c_text = nullptr;  int64_t c_text_cap = 0;
    void *c_ws = nullptr;    int64_t c_ws_cap = 0;
    void *c_out = nullptr;   int64_t c_out_cap = 0;   // uint64 entries
    void *c_counts = nullptr;                         // int64[d] + n_occ + running total
    void *c_pin = nullptr;                            // page-locked per-piece totals
};
