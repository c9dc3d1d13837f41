/*
 * pmscan.h -- C ABI of libpmscan: multiple pattern matching on one GB300.
 *
 * The operation (Kouzinopoulos et al., "A Hybrid Parallel Implementation of
 * the Aho-Corasick and Wu-Manber Algorithms Using NVIDIA CUDA and MPI",
 * Section 1, Definition): given a text T = t_0..t_{n-1} and a set of d
 * patterns p^0..p^{d-1}, all of length m, find every pair (i, r) with
 * 0 <= i <= n-m and t_{i+j} = p^r_j for every 0 <= j < m.
 *
 * Two methods compute that set, both from Section 3 of the paper:
 *   - Aho-Corasick (Section 3.1, Algorithms 1-3), compiled here to a full
 *     DFA: goto and supply functions merged into one transition table with a
 *     next state for every state and every character class (the "array of
 *     size |Sigma|" representation the paper names in Section 3.1);
 *   - Wu-Manber (Section 3.2, Algorithms 4-5): SHIFT / HASH / PREFIX tables
 *     over blocks of B characters, candidates verified against the text.
 * The data-parallel split of the text into chunks that overlap by m-1
 * characters follows Section 4.2.1 (Algorithms 6-9). pm_pfac_compile adds
 * the failure-less Aho-Corasick variant; pm_acv_compile and pm_wmv_compile
 * take sets whose patterns have their own lengths (the definition with each
 * pattern's length in place of m).
 *
 * Conventions shared by every call:
 *   - P is d*m contiguous bytes, row r = p^r. Any byte values are allowed.
 *     P is copied during compilation; the caller keeps ownership.
 *   - Pattern ids r are 0-based in input order; positions i are 0-based
 *     start positions. Duplicate patterns are each reported under their own
 *     id (ascending r at the same i).
 *   - Occurrences are uint64 keys ((uint64_t)i << 32) | r, sorted ascending,
 *     i.e. by position, then by pattern id.
 *   - counts[r] is the number of occurrences of pattern r (int64).
 *   - n must be < 2^32 and d < 2^24 (2^23 for Wu-Manber sets); otherwise
 *     PM_ETOOBIG.
 *   - n < m is not an error: the result is empty.
 *   - Every call returns PM_OK (0) or one of the error codes below; no C++
 *     exception crosses this boundary. On error, output pointers are left
 *     untouched and nothing is leaked.
 *   - Calls that take a stream (cudaStream_t passed as void*, NULL = the
 *     legacy default stream) are asynchronous unless documented otherwise.
 */
#ifndef PMSCAN_H
#define PMSCAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes -------------------------------------------------------- */
#define PM_OK 0
#define PM_EINVAL 1    /* bad argument (NULL pointer, d < 1, m < 1, bad B ...) */
#define PM_ENOMEM 2    /* host or device allocation failed */
#define PM_ECUDA 3     /* a CUDA runtime call failed (see pm_last_cuda_error) */
#define PM_ETOOBIG 4   /* n >= 2^32, d >= 2^24, m > 255, or a table too large */
#define PM_ETIMEOUT 5  /* a bounded device wait gave up (status word set) */
#define PM_ECAPACITY 6 /* occurrence buffer too small; *d_n_occ holds the need */
#define PM_ENODEV 7    /* no usable CUDA device (the library never computes on the CPU) */

/* ---- scan flags ---------------------------------------------------------- */
#define PM_HOST_TEXT 0u     /* T is a host pointer (copied to the device) */
#define PM_DEVICE_TEXT 1u   /* T is a device pointer */
#define PM_COUNTS_ONLY 2u   /* per-pattern counts and the total only; no list */

/* ---- table placement (Aho-Corasick transition table) ------------------- */
#define PM_PLACE_AUTO 0    /* shared memory if it fits, else hybrid */
#define PM_PLACE_SMEM 1    /* whole table in shared memory, else PM_ETOOBIG */
#define PM_PLACE_HYBRID 2  /* breadth-first prefix of rows in shared memory, rest via L2 */
#define PM_PLACE_GLOBAL 3  /* every row read through L1/L2 */

#define PM_ALGO_AC 1
#define PM_ALGO_WM 2
#define PM_ALGO_PFAC 3
#define PM_ALGO_ACV 4   /* Aho-Corasick over patterns of mixed lengths */
#define PM_ALGO_WMV 5   /* Wu-Manber over patterns of mixed lengths */

/* Tuning knobs; a zero field means "pick automatically". */
typedef struct pm_params {
    int32_t placement;        /* PM_PLACE_* */
    int32_t smem_table_bytes; /* cap on the shared-memory part of the table */
    int32_t warps_per_cta;    /* 1..32 (0 automatic); clamped to the kernel's
                                 launch bound: at most 24 (768-thread kernels)
                                 for Aho-Corasick, PFAC and Wu-Manber over
                                 ACGT-like alphabets, for mixed lengths and
                                 for the stride-2 scan, else 16 */
    int32_t ctas_per_sm;      /* persistent CTAs per SM */
    int32_t wm_prefix_len;    /* Wu-Manber B' (default 2, clamped to m) */
    int32_t host_only;        /* 1: build host tables only (no device upload);
                                 such a set can only be inspected, not scanned */
    int32_t counters;         /* AC per-terminal counters: 0 auto, 1 32-bit in
                                 shared memory, 2 16-bit in shared memory,
                                 3 64-bit in device memory */
    int32_t ids_place;        /* AC terminal-id structure: 0 auto, 1 shared
                                 memory, 2 device memory (through L1/L2),
                                 3 late: in list mode the scan keeps only a
                                 2-bit multiplicity per match entry, and the
                                 expand kernel maps match entries to terminal
                                 ids and pattern codes and counts them (frees
                                 shared memory for the table and warps);
                                 counts mode keeps the rank structure there;
                                 not for PFAC sets */
    int32_t stride;           /* AC characters per table lookup: 0 or 1 one; 2 two
                                 (a 16-entry row per state and character pair,
                                 for ACGT sets of at most 4096 rows and m <= 33;
                                 PM_ETOOBIG otherwise); pm_tune tries both */
} pm_params;

typedef struct pm_set pm_set; /* compiled pattern set; owns its device tables */

typedef struct pm_set_info {
    int32_t algo;             /* PM_ALGO_AC, PM_ALGO_WM, PM_ALGO_PFAC, PM_ALGO_ACV or PM_ALGO_WMV */
    int32_t m;
    int64_t d;
    int64_t n_distinct;       /* distinct patterns */
    /* Aho-Corasick (and PFAC) */
    int64_t n_states;         /* trie states, including terminals */
    int64_t n_rows;           /* DFA rows kept (terminal rows elided) + reset row */
    int32_t n_classes;        /* character classes (alphabet size of P) */
    int32_t row_width;        /* table columns per row */
    int32_t entry_bytes;      /* 2 or 4 */
    int32_t dna_mode;         /* 1: ACGT-like alphabet decoded arithmetically
                                 (Wu-Manber: exact 2-bit-code tables in use) */
    int32_t placement;        /* resolved PM_PLACE_* */
    int64_t smem_rows;        /* rows resident in shared memory */
    int64_t table_bytes;      /* bytes of the transition table */
    /* Wu-Manber */
    int32_t B, Bp;            /* block size B and prefix length B' */
    int64_t shift_entries;    /* 2^(5B) */
    int64_t n_zero_shift;     /* SHIFT entries equal to 0 */
    /* both */
    int64_t device_bytes;     /* device memory owned by the set */
    /* mixed lengths (PM_ALGO_ACV, PM_ALGO_WMV; m is then the longest length) */
    int32_t m_min;            /* shortest pattern length (= m for one length) */
    int32_t max_starts;       /* most patterns that can start at one position */
    int32_t stride;           /* AC characters per table lookup in use (1 or 2) */
} pm_set_info;

typedef struct pm_result {    /* library-owned; release with pm_result_free */
    int64_t d;
    int64_t n_occ;
    int64_t *counts;          /* host array of d counts */
    uint64_t *occ;            /* host array of n_occ keys (NULL if counts only) */
} pm_result;

/*
 * Compile an Aho-Corasick DFA (Section 3.1, Algorithms 1-2, merged into one
 * transition table). Builds the trie in insertion order, supply links in
 * breadth-first order, the full transition function, renumbers states
 * breadth-first, elides the rows of depth-m states and uploads the tables.
 * opt may be NULL. On success *out owns device memory until pm_set_free.
 * Device scans hold a lane's m-1 halo bytes in registers, so m <= 65 unless
 * opt->host_only is set (PM_ETOOBIG otherwise).
 */
int pm_ac_compile(const uint8_t *P, int64_t d, int32_t m,
                  const pm_params *opt, pm_set **out);

/*
 * Compile Wu-Manber tables (Section 3.2, Algorithm 4) for block size B,
 * 1 <= B <= min(m, 4). h1 and h2 shift by 5 bits and add (byte & 31), giving
 * 2^(5B) SHIFT entries; results do not depend on the hash (SHIFT is a
 * minimum over colliding blocks and every candidate is verified in full).
 */
int pm_wm_compile(const uint8_t *P, int64_t d, int32_t m, int32_t B,
                  const pm_params *opt, pm_set **out);

/*
 * Compile a PFAC set (failure-less Aho-Corasick, Lin et al.; the related work
 * the paper cites next to its own kernels): the trie of Section 3.1,
 * Algorithm 1, with no supply function. Each start position i is walked by
 * its own thread along goto edges only; a walk that reaches depth m reports
 * (i, r), one that finds no edge stops. Same results, scans, workspace and
 * outputs as an AC set (pm_scan, pm_scan_device ...); the batched scan, the
 * server, the tuner and the allocation-free scan take AC sets only.
 */
int pm_pfac_compile(const uint8_t *P, int64_t d, int32_t m,
                    const pm_params *opt, pm_set **out);

/*
 * Compile an Aho-Corasick set whose patterns have their own lengths (the
 * Section 1 definition with each pattern's length in place of m; the
 * paper's sets have one length). Pattern r is P[offsets[r] .. offsets[r+1]),
 * offsets[0] = 0, each length 1..65; P and offsets are copied. Algorithm 1's
 * trie, Algorithm 2's supply links and output propagation (Output(s) takes
 * Output(Supply(s))), merged into one DFA with a row per state; a position
 * reports every pattern ending there, each at its own start. pm_scan,
 * pm_scan_to_host (single launch) and pm_scan_device take such sets; the
 * occurrence list is sorted by (i, r) as for the other sets. The slot part
 * of the list-mode workspace grows with pm_set_info.max_starts. The batched
 * scan, the server, the tuner and the allocation-free scan take AC sets only.
 * Errors: PM_EINVAL (bad offsets, a length 0), PM_ETOOBIG (a length above
 * 65, d >= 2^25).
 */
int pm_acv_compile(const uint8_t *P, const int64_t *offsets, int64_t d,
                   const pm_params *opt, pm_set **out);

/*
 * Compile Wu-Manber tables for a set of mixed lengths (same layout of P and
 * offsets as pm_acv_compile), with m = the shortest length: Algorithm 4 over
 * every pattern's first m characters (1 <= B <= min(shortest length, 4)),
 * HASH holding every id in (PREFIX, r) order, and each candidate verified
 * over its own length. Algorithm 5 visits the windows of length m; the
 * matches at one start come out in ascending r. Byte-hash tables only (no
 * exact-code path). Same scan entry points and restrictions as
 * pm_acv_compile.
 */
int pm_wmv_compile(const uint8_t *P, const int64_t *offsets, int64_t d, int32_t B,
                   const pm_params *opt, pm_set **out);

void pm_set_free(pm_set *s);
int pm_set_get_info(const pm_set *s, pm_set_info *info);

/*
 * The launch plan the planner picks for an Aho-Corasick or PFAC set on a
 * device of the given shape: its number of SMs, the most dynamic shared
 * memory a block may opt in to, and the shared memory per SM (bytes). The
 * set's own pm_params (placement, warps, counters, ids) apply as at compile
 * time. No device is touched, so this works for host-only sets
 * (pm_params.host_only) and without a GPU: for inspecting what the planner
 * does and testing it. A set compiled for a device runs the plan of that
 * device's shape (until pm_tune replaces it). PM_EINVAL for other
 * algorithms or non-positive sizes; PM_ETOOBIG when nothing fits.
 */
typedef struct pm_plan_info {
    int32_t placement;        /* PM_PLACE_SMEM, PM_PLACE_HYBRID or PM_PLACE_GLOBAL */
    int32_t warps;            /* warps per CTA, counts-only scans */
    int32_t warps_list;       /* warps per CTA, list mode */
    int32_t ids_place;        /* terminal-id structure: 1 shared memory,
                                 2 device memory, 3 late (pm_params.ids_place) */
    int32_t counters;         /* counts-only scans' per-terminal counters:
                                 1 32-bit shared, 2 16-bit shared, 3 device */
    int32_t ctas_per_sm;
    int64_t smem_rows;        /* table rows held in shared memory */
    int64_t smem_bytes;       /* dynamic shared memory per CTA, counts only */
    int64_t smem_bytes_list;  /* the same, list mode */
} pm_plan_info;
int pm_plan_for_device(const pm_set *s, int32_t sm_count, int32_t smem_optin, int32_t smem_per_sm,
                       pm_plan_info *out);

/*
 * Scan T (n bytes) for every occurrence of the set (Section 1 definition).
 * flags: PM_HOST_TEXT or PM_DEVICE_TEXT, optionally | PM_COUNTS_ONLY.
 * Synchronous: returns when *out (host arrays, library-owned) is complete.
 * Device buffers are cached inside the set between calls, so a set must not
 * be scanned from two host threads at once.
 */
int pm_scan(const pm_set *s, const uint8_t *T, int64_t n, uint32_t flags,
            void *stream, pm_result **out);

void pm_result_free(pm_result *r);

/*
 * pm_scan with caller-owned host result buffers (page-locked buffers give
 * full-speed device-to-host copies; T may be page-locked for the same
 * reason). counts_out: int64[d]; occ_out: uint64[occ_capacity] (may be NULL
 * with PM_COUNTS_ONLY). *n_occ_out receives the total; when it exceeds
 * occ_capacity only the first occ_capacity keys are written and the call
 * returns PM_ECAPACITY. Synchronous.
 */
int pm_scan_to_host(const pm_set *s, const uint8_t *T, int64_t n, uint32_t flags,
                    int64_t *counts_out, uint64_t *occ_out, int64_t occ_capacity,
                    int64_t *n_occ_out, void *stream);

/*
 * Device-level scan with caller-owned device buffers (e.g. torch tensors),
 * enqueued on `stream`; nothing is allocated and nothing synchronises.
 *   d_text       device text, n bytes (any alignment; 16-byte aligned is fastest)
 *   d_counts     device int64[d], overwritten
 *   d_occ        device uint64[occ_capacity] (may be NULL with PM_COUNTS_ONLY)
 *   d_n_occ      device int64[1], receives the total number of occurrences
 *   d_workspace  device scratch of at least pm_scan_workspace_bytes(s, n, flags)
 * If the total exceeds occ_capacity only the first occ_capacity keys are
 * written; the call still succeeds and *d_n_occ tells the caller how much to
 * allocate for a rerun. Device-side failures (a bounded wait that gave up)
 * are reported in the workspace status word, read by pm_scan_status.
 */
int64_t pm_scan_workspace_bytes(const pm_set *s, int64_t n, uint32_t flags);

int pm_scan_device(const pm_set *s, const uint8_t *d_text, int64_t n, uint32_t flags,
                   int64_t *d_counts, uint64_t *d_occ, int64_t occ_capacity,
                   int64_t *d_n_occ, void *d_workspace, int64_t workspace_bytes,
                   void *stream);

/*
 * Allocation-free Aho-Corasick scan. The paper has no counterpart: this is
 * for callers that cannot allocate device memory when they scan -- a host
 * application that owns the GPU allocator and must account for every
 * allocation, or a latency-bound loop that reserved all of its memory up
 * front and must not call cudaMalloc (which can block on the device and
 * fail under fragmentation). It computes what pm_scan_device computes (same
 * arguments, no workspace) with its scratch in one fixed device array of
 * pm_noalloc_scratch_bytes() bytes (64 MiB) inside the library, reserved on
 * every GPU that loads the library until the process exits. Nothing is
 * allocated: no cudaMalloc, cudaFree or allocating library call.
 *   - Only plain Aho-Corasick sets (PM_EINVAL for PFAC, mixed-length and
 *     Wu-Manber sets).
 *   - Always the one-character walk, even for a set whose tuned plan takes
 *     two characters per lookup (pm_params.stride = 2): the results are the
 *     same, only the launch plan differs.
 *   - PM_ETOOBIG when the scan would need more scratch than the array holds
 *     (large texts in list mode, or very large pattern sets); nothing runs.
 *   - Each call looks up the array's device address on the current device
 *     (no allocation); the first lookup on a device may load the library's
 *     kernels, so make the first call before any stream capture begins.
 *   - Every call uses the same array, which keeps the last call's contents
 *     (the call clears what must start at zero). Calls whose work overlaps
 *     on the GPU -- other streams, other host threads -- race on it: run
 *     them one after another.
 *   - A device-side failure (a bounded wait that gave up) is recorded in the
 *     array's status word: read it with pm_noalloc_scan_status.
 */
int pm_scan_device_noalloc(const pm_set *s, const uint8_t *d_text, int64_t n, uint32_t flags,
                           int64_t *d_counts, uint64_t *d_occ, int64_t occ_capacity,
                           int64_t *d_n_occ, void *stream);
int64_t pm_noalloc_scratch_bytes(void);
/* Synchronise `stream` and read the status word of the last
 * pm_scan_device_noalloc on the current device: PM_OK, or PM_ETIMEOUT when a
 * bounded wait in the kernel gave up (the results are then incomplete). */
int pm_noalloc_scan_status(void *stream);

/*
 * Autotuner for the plain Aho-Corasick scan (the paper's kernels fix their
 * launch shape by hand; this picks it by measurement). Times `reps` scans of
 * the device text (after one warm-up each) for every distinct launch plan
 * the planner accepts over table placement (shared memory / hybrid prefix),
 * warps per CTA (auto, 16, 12, 8), per-terminal counters (32-bit or 16-bit
 * in shared memory, or device memory) and the terminal-id structure (shared
 * or device memory, or late: codes and counts taken by the expand kernel in
 * list mode), plus the two-character scan (stride 2) when the set
 * qualifies, and keeps the fastest for the set: later scans use it. In list
 * mode, late plans that differ only in their counters count as one, and the
 * one kept has the counters that fit best for counts-only scans.
 * Results never depend on the plan. Allocates its own scratch, synchronises
 * `stream`. *best_out / *best_ms (may be NULL) receive the chosen pm_params
 * and its time per scan. Wu-Manber sets tune warps per CTA only (auto, 24,
 * 20, 16, 12, 8; more than 16 for exact-code tables of ACGT sets).
 * PM_EINVAL for PFAC and mixed-length sets and for host-only sets.
 */
int pm_tune(pm_set *s, const uint8_t *d_text, int64_t n, uint32_t flags, int32_t reps,
            void *stream, pm_params *best_out, float *best_ms);

/* Synchronise `stream` and read the device status word of the last
 * pm_scan_device on this workspace: PM_OK or PM_ETIMEOUT. */
int pm_scan_status(const void *d_workspace, void *stream);

/*
 * Scan k independent (set, text) instances, synchronously; outs[j]
 * receives instance j's result (library-owned, as pm_scan gives it).
 * texts are host pointers unless flags has PM_DEVICE_TEXT. Host texts
 * against Aho-Corasick sets over an ACGT-like alphabet with m <= 65 run
 * together in the batched persistent kernel (pm_batch_*): a first launch
 * gives every instance's total, a second writes the keys into exact
 * capacities. Every other instance (device texts, PFAC, Wu-Manber, mixed
 * lengths) runs as a pm_scan call, in order. Results equal k separate
 * pm_scan calls. Allocates device scratch for the call and frees it. On an
 * error every outs[j] is NULL.
 */
int pm_scan_batch(const pm_set *const *sets, const uint8_t *const *texts,
                  const int64_t *ns, int32_t k, uint32_t flags, void *stream,
                  pm_result **outs);

/*
 * Batched device scan: k independent Aho-Corasick instances (text j against
 * set j), each computing exactly what pm_scan_device computes for it, in one
 * persistent launch. A CTA takes whole instances from a queue, largest text
 * first, and runs the instance's warp tiles (the chunk-with-halo partition of
 * Section 4.2.1) on its own warps, so no instance waits on another. The
 * paper scans one text per run; the batch and its tuner and graph are
 * additions of this library.
 *
 * pm_batch_prepare fixes the batch layout (host arrays are copied):
 *   sets      k compiled AC sets over an ACGT-like alphabet with m <= 65
 *             (else PM_EINVAL); a set may appear several times
 *   text_off, text_len  int64[k] each: instance j's text is the
 *             text_len[j] (< 2^32) bytes at text_off[j] of one device text
 *             buffer; texts may overlap (16-byte aligned starts let the tiles
 *             be copied by the bulk-copy engine)
 *   occ_off   int64[k+1]: instance j's keys go to occ[occ_off[j] ..
 *             occ_off[j+1]) (its capacity); ignored with PM_COUNTS_ONLY
 *   flags     0 or PM_COUNTS_ONLY (PM_DEVICE_TEXT is accepted and implied)
 * Counts of instance j land at counts[c_j .. c_j + d_j) with c_j the sum of
 * the d of the instances before j; pm_batch_counts_total gives the sum. The
 * sets must outlive the batch. The batch owns a small device array of
 * descriptors until pm_batch_free.
 */
typedef struct pm_batch pm_batch;
int pm_batch_prepare(const pm_set *const *sets, int32_t k, const int64_t *text_off,
                     const int64_t *text_len, const int64_t *occ_off, uint32_t flags,
                     pm_batch **out);
void pm_batch_free(pm_batch *b);
int64_t pm_batch_counts_total(const pm_batch *b);
/* Workspace for every call below (any warp count the tuner may pick): a
 * header, the device counters of instances whose counters do not fit a
 * CTA's shared memory, and, in list mode, key staging for the parts of
 * instances split across CTAs (one 8-byte key per 32 text bytes of a part,
 * at most the instance's capacity). */
int64_t pm_batch_workspace_bytes(const pm_batch *b);
int32_t pm_batch_warps(const pm_batch *b);  /* warps per CTA of the current plan */

/*
 * Enqueue the batched scan on `stream` (asynchronous, allocates nothing).
 *   d_text   the device text buffer of pm_batch_prepare
 *   d_counts int64[pm_batch_counts_total]; d_n_occ int64[k]: instance j's
 *            total, which may exceed its capacity (then only the first
 *            capacity keys are written, sorted, as in pm_scan_device)
 *   d_occ    uint64[occ_off[k]] (may be NULL with PM_COUNTS_ONLY)
 * Device-side failures are reported through pm_scan_status on d_workspace.
 */
int pm_batch_scan_device(const pm_batch *b, const uint8_t *d_text, int64_t *d_counts,
                         uint64_t *d_occ, int64_t *d_n_occ, void *d_workspace,
                         int64_t workspace_bytes, void *stream);

/*
 * Autotuner: times `reps` batched scans (after one warm-up) for each
 * candidate plan, warps per CTA (8, 12, 16; each fixes how shared memory is
 * split between per-warp buffers and the instance region) x table placement
 * (see pm_batch_set_placement), keeps the fastest and returns its time per
 * scan in *best_ms (may be NULL). Synchronises `stream`; results of every
 * candidate are identical, and the buffers hold the last candidate's. Drops
 * a captured graph.
 */
int pm_batch_tune(pm_batch *b, const uint8_t *d_text, int64_t *d_counts, uint64_t *d_occ,
                  int64_t *d_n_occ, void *d_workspace, int64_t workspace_bytes, int32_t reps,
                  void *stream, float *best_ms);
int pm_batch_set_warps(pm_batch *b, int32_t warps);  /* 1..16; drops a captured graph */
/* Table placement of instances whose tables do not all fit the CTA's shared
 * memory: 0 (default) keeps their terminal ids and counters there while each
 * takes at most a quarter of the region and gives the table's breadth-first
 * prefix the rest; 1 keeps ids and counters in device memory and gives the
 * prefix the whole region. PM_EINVAL for other values; drops a captured
 * graph. Results never depend on it. */
int pm_batch_set_placement(pm_batch *b, int32_t placement);
int32_t pm_batch_placement(const pm_batch *b);  /* the current plan's placement, or -1 */

/*
 * CUDA graph of one batched scan on these buffers (the workspace memset and
 * the persistent kernel), captured on a private stream; pm_batch_replay
 * launches it on `stream`. Buffers are baked in: replays must use them and
 * must not overlap each other. Capture synchronises nothing and runs nothing.
 */
int pm_batch_capture(pm_batch *b, const uint8_t *d_text, int64_t *d_counts, uint64_t *d_occ,
                     int64_t *d_n_occ, void *d_workspace, int64_t workspace_bytes);
int pm_batch_replay(const pm_batch *b, void *stream);

/*
 * Serving loop with continuous batching (the paper has no counterpart; it
 * scans one text per run). A server owns a device arena of
 * device_budget_bytes for the texts, counts and occurrence buffers of the
 * requests in flight, and two host threads:
 *   - a dispatcher admits queued requests in arrival order while their
 *     memory fits the arena, and launches everything admitted as one batched
 *     scan (pm_batch_scan_device's kernel) on a free stream slot; up to
 *     max_inflight batches run at once, so requests that arrive while others
 *     are on the GPU start as soon as memory and a slot free up;
 *   - a completer copies each finished batch's results to host memory
 *     (re-running, with the exact capacity, the rare request whose
 *     occurrence estimate was short), frees its memory, records latencies and
 *     wakes waiters.
 * Requests of 256 KiB or more run as whole-GPU scans (the plain kernel) on
 * the slot's stream, sharing one per-slot workspace outside the arena; the
 * rest share one batched launch.
 * A request's result equals a solo scan of the same text with the same set
 * (pm_scan): instances never share counters or outputs.
 */
typedef struct pm_server pm_server;
typedef struct pm_server_params {
    int64_t device_budget_bytes;  /* arena size (default 4 GiB) */
    int32_t max_batch;            /* requests per batched launch (default 512) */
    int32_t max_inflight;         /* batches in flight, one stream each (default 3, max 16) */
    int32_t warps_per_cta;        /* batched kernel shape, 1..16 (default 12) */
    int32_t pad;
    int64_t counter_words;        /* per-slot workspace for global per-terminal
                                     counters, in 8-byte words (default 4 Mi) */
    int64_t host_pool_bytes;      /* page-locked host pool for result arrays
                                     (default 1 GiB; < 0: none, plain memory);
                                     results may outlive the server */
} pm_server_params;
typedef struct pm_server_stats {
    int64_t completed;            /* requests finished with PM_OK */
    int64_t bytes;                /* text bytes of those requests */
    int64_t batches;              /* batched launches */
    int64_t reruns;               /* requests re-run with an exact capacity */
    int64_t peak_inflight;        /* most requests admitted at once */
    int64_t pending;              /* requests waiting for admission now */
    int64_t arena_used;           /* arena bytes held now */
    double mean_batch;            /* requests per launch */
    double p50_us, p99_us, mean_us; /* latency, submit -> result on the host */
    double gbs;                   /* text bytes / (last completion - first submit) */
    double dispatch_busy_s;       /* dispatcher time spent enqueueing batches */
    double complete_busy_s;       /* completer time spent finishing batches */
} pm_server_stats;

/* params may be NULL (all defaults). Allocates the arena and per-slot
 * buffers on the current device and starts the two threads. */
int pm_server_create(const pm_server_params *params, pm_server **out);
/*
 * Queue a scan of host text T (n bytes) against `set` (an AC set the batched
 * scan accepts, else PM_EINVAL); flags: 0 or PM_COUNTS_ONLY. T and set must
 * stay valid until pm_server_wait returns for the ticket. PM_ETOOBIG when
 * the request alone could never fit the arena. Never blocks on the GPU.
 */
int pm_server_submit(pm_server *s, const pm_set *set, const uint8_t *T, int64_t n,
                     uint32_t flags, int64_t *ticket);
/* Block until the request is done; returns its status and hands over its
 * result (library-owned; pm_result_free). Each ticket is waited on once. */
int pm_server_wait(pm_server *s, int64_t ticket, pm_result **out);
int pm_server_get_stats(pm_server *s, pm_server_stats *st);
/* Forget the statistics so far (e.g. after a warm-up); requests in flight
 * are counted when they finish. */
int pm_server_reset_stats(pm_server *s);
/* Finishes every queued and running request, then frees everything
 * (results never waited on are freed too). */
void pm_server_destroy(pm_server *s);

/*
 * Table self-check on the host, no GPU needed: walks the compiled AC table
 * (or applies the compiled WM tables) exactly as the kernels do, one thread,
 * on the host. It exists to test the compiler; pm_scan never calls it.
 */
int pm_selfcheck_host_walk(const pm_set *s, const uint8_t *T, int64_t n, pm_result **out);

const char *pm_strerror(int code);
int pm_last_cuda_error(void);  /* cudaError_t of the last PM_ECUDA, per thread */
const char *pm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PMSCAN_H */
