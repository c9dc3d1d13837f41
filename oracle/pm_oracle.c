/*
 * pm_oracle.c -- CPU oracle for multiple pattern matching.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg use it. It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (Kouzinopoulos et al., "A Hybrid Parallel Implementation of
 * the Aho-Corasick and Wu-Manber Algorithms Using NVIDIA CUDA and MPI",
 * Section 1, Definition): given a text T = t_0..t_{n-1} and d patterns
 * p^0..p^{d-1}, each of length m, report every pair (i, r) with
 * 0 <= i < n-m+1 and t_{i+j} = p^r_j for all 0 <= j < m.  (The printed
 * definition reads "t_i = p^r_j"; the index must be i+j for "occurrence" to
 * mean anything, and Algorithm 3 reports at i-m+1, which agrees.)
 *
 * Output convention shared by every routine here:
 *   occ[k]    = ((uint64_t)i << 32) | r, sorted ascending by (i, r);
 *   counts[r] = number of i with (i, r) reported;
 *   return    = total number of occurrences (may exceed cap; only the first
 *               cap entries are written, counts are always complete).
 *
 * Routines:
 *   orc_brute   -- the definition as three nested loops (Section 1).
 *   orc_dict    -- the same set, by membership of each text window in a
 *                  sorted dictionary of the patterns; multithreaded over i.
 *   orc_ac_*    -- sequential Aho-Corasick, Algorithms 1, 2 and 3 (Section
 *                  3.1): goto trie in insertion order, supply links in
 *                  breadth-first order, search that follows supply links.
 *   orc_wm_*    -- sequential Wu-Manber, Algorithms 4 and 5 (Section 3.2)
 *                  with the paper's shift-and-add hash (bitshift 2).
 *   orc_ac_dfa_scan -- the CPU baseline: the same automaton as a full DFA
 *                  over byte classes, walked by host threads over contiguous
 *                  ranges with the m-1 overlap (timed, not a parity route).
 *   orc_brute_var, orc_dict_var -- the same definition for a set whose
 *                  patterns have their own lengths len_r: every (i, r) with
 *                  i + len_r <= n and t_{i+k} = p^r_k for all k < len_r
 *                  (the paper's sets have one length m; this is the
 *                  definition with m replaced by len_r).
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   - Algorithm 1 adds pattern i to Output() of the state its path ends in.
 *     The listing names q_current, the last state *created*; for a pattern
 *     whose whole path already exists (a duplicate) no state is created, so
 *     the state reached by the walk is used.
 *   - Algorithms 4, 5, 7 and 9 write the B-character block as
 *     p_{q-B-1}..p_{q-1} and t_{i-B}..t_i, which is B+1 characters; the block
 *     used is the B characters p_{q-B}..p_{q-1} and t_{i-B+1}..t_i, the only
 *     reading under which SHIFT of a pattern's last block is m-q = 0.
 *   - Duplicate patterns are reported once per index r (the definition is
 *     "for each p^r").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_OCC(i, r) ((((uint64_t)(i)) << 32) | (uint64_t)(uint32_t)(r))

/* ------------------------------------------------------------------------ */
/* O1a: the definition, literally.                                           */
/* ------------------------------------------------------------------------ */
int64_t orc_brute(const uint8_t *T, int64_t n, const uint8_t *P, int64_t d,
                  int32_t m, uint64_t *occ, int64_t cap, int64_t *counts)
{
    int64_t total = 0;
    for (int64_t r = 0; r < d; r++) counts[r] = 0;
    if (m < 1 || n < m) return 0;
    for (int64_t i = 0; i < n - m + 1; i++) {
        for (int64_t r = 0; r < d; r++) {
            const uint8_t *p = P + r * (int64_t)m;
            int all = 1;
            for (int32_t j = 0; j < m; j++) {
                if (T[i + j] != p[j]) { all = 0; break; }
            }
            if (all) {
                if (total < cap) occ[total] = ORC_OCC(i, r);
                total++;
                counts[r]++;
            }
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* O1b: the same set by dictionary membership.                               */
/* The patterns are sorted by (bytes, r); window T[i..i+m) is located by     */
/* binary search and every equal pattern is reported in ascending r.         */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint8_t *P;
    int32_t m;
} orc_sort_ctx;

/* Order of pattern indices ra, rb: by bytes, then by index. */
static int orc_cmp_pattern_idx(const void *ctx, int64_t ra, int64_t rb)
{
    const orc_sort_ctx *c = (const orc_sort_ctx *)ctx;
    int k = memcmp(c->P + ra * c->m, c->P + rb * c->m, (size_t)c->m);
    if (k) return k;
    return (ra > rb) - (ra < rb);
}

/* Bottom-up merge sort of n indices under cmp(ctx, .) -- the context is an
 * argument, so concurrent oracle calls never share sorting state. Returns
 * -1 if its scratch cannot be allocated. */
static int orc_sort_idx(int64_t *a, int64_t n, int (*cmp)(const void *, int64_t, int64_t), const void *ctx)
{
    if (n < 2) return 0;
    int64_t *tmp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!tmp) return -1;
    int64_t *src = a, *dst = tmp;
    for (int64_t w = 1; w < n; w *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * w) {
            int64_t mid = lo + w < n ? lo + w : n;
            int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) dst[k++] = cmp(ctx, src[j], src[i]) < 0 ? src[j++] : src[i++];
            while (i < mid) dst[k++] = src[i++];
            while (j < hi) dst[k++] = src[j++];
        }
        int64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(int64_t));
    free(tmp);
    return 0;
}

typedef struct {
    const uint8_t *T;
    const uint8_t *P;
    const int64_t *order; /* pattern indices sorted by (bytes, r) */
    int64_t d;
    int32_t m;
    int64_t i0, i1;       /* window starts handled by this worker */
    uint64_t *buf;        /* worker-local occurrences */
    int64_t len, cap;
    int64_t *counts;      /* worker-local per-pattern counts */
    int failed;
} orc_dict_job;

static void *orc_dict_worker(void *arg)
{
    orc_dict_job *jb = (orc_dict_job *)arg;
    const int32_t m = jb->m;
    for (int64_t i = jb->i0; i < jb->i1; i++) {
        const uint8_t *w = jb->T + i;
        /* lower bound of w among the sorted patterns */
        int64_t lo = 0, hi = jb->d;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (memcmp(jb->P + jb->order[mid] * m, w, (size_t)m) < 0) lo = mid + 1;
            else hi = mid;
        }
        for (int64_t k = lo; k < jb->d; k++) {
            int64_t r = jb->order[k];
            if (memcmp(jb->P + r * m, w, (size_t)m) != 0) break;
            if (jb->len == jb->cap) {
                int64_t nc = jb->cap ? 2 * jb->cap : 4096;
                uint64_t *nb = (uint64_t *)realloc(jb->buf, (size_t)nc * sizeof(uint64_t));
                if (!nb) { jb->failed = 1; return NULL; }
                jb->buf = nb;
                jb->cap = nc;
            }
            jb->buf[jb->len++] = ORC_OCC(i, r);
            jb->counts[r]++;
        }
    }
    return NULL;
}

/* Returns the total, or -1 if memory ran out. */
int64_t orc_dict(const uint8_t *T, int64_t n, const uint8_t *P, int64_t d,
                 int32_t m, int32_t nthreads, uint64_t *occ, int64_t cap,
                 int64_t *counts)
{
    for (int64_t r = 0; r < d; r++) counts[r] = 0;
    if (m < 1 || n < m || d < 1) return 0;
    if (nthreads < 1) nthreads = 1;
    int64_t nwin = n - m + 1;
    if (nthreads > nwin) nthreads = (int32_t)nwin;

    int64_t *order = (int64_t *)malloc((size_t)d * sizeof(int64_t));
    orc_dict_job *jobs = (orc_dict_job *)calloc((size_t)nthreads, sizeof(orc_dict_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!order || !jobs || !tids) { free(order); free(jobs); free(tids); return -1; }
    for (int64_t r = 0; r < d; r++) order[r] = r;
    const orc_sort_ctx sctx = {P, m};
    if (orc_sort_idx(order, d, orc_cmp_pattern_idx, &sctx)) {
        free(order);
        free(jobs);
        free(tids);
        return -1;
    }

    int64_t total = 0;
    int failed = 0;
    for (int32_t t = 0; t < nthreads; t++) {
        jobs[t].T = T; jobs[t].P = P; jobs[t].order = order;
        jobs[t].d = d; jobs[t].m = m;
        jobs[t].i0 = nwin * t / nthreads;
        jobs[t].i1 = nwin * (t + 1) / nthreads;
        jobs[t].counts = (int64_t *)calloc((size_t)d, sizeof(int64_t));
        if (!jobs[t].counts) failed = 1;
    }
    if (!failed) {
        for (int32_t t = 0; t < nthreads; t++)
            pthread_create(&tids[t], NULL, orc_dict_worker, &jobs[t]);
        for (int32_t t = 0; t < nthreads; t++) pthread_join(tids[t], NULL);
        /* workers cover consecutive i-ranges, so concatenation is sorted */
        for (int32_t t = 0; t < nthreads; t++) {
            if (jobs[t].failed) failed = 1;
            for (int64_t k = 0; k < jobs[t].len; k++) {
                if (total < cap) occ[total] = jobs[t].buf[k];
                total++;
            }
            for (int64_t r = 0; r < d; r++) counts[r] += jobs[t].counts[r];
        }
    }
    for (int32_t t = 0; t < nthreads; t++) { free(jobs[t].buf); free(jobs[t].counts); }
    free(order); free(jobs); free(tids);
    return failed ? -1 : total;
}

/* ------------------------------------------------------------------------ */
/* O2: sequential Aho-Corasick, Algorithms 1-3 (Section 3.1).                */
/* Sigma is the 256 byte values. g is a dense goto table with FAIL = -1;     */
/* states are numbered in creation order, q_0 = 0.                           */
/* ------------------------------------------------------------------------ */
#define ORC_SIGMA 256
#define ORC_FAIL (-1)

typedef struct {
    int64_t nstates;
    int32_t *g;        /* nstates x 256 goto function */
    int32_t *supply;   /* supply (failure) function; supply[0] = 0 unused */
    int64_t *out_head; /* first entry of Output(q) in out_next chain, -1 none */
    int64_t *out_tail;
    int64_t *out_next; /* per pattern: next pattern in the same Output set */
    int32_t *depth;
    int32_t m;
    int64_t d;
} orc_ac;

void orc_ac_free(orc_ac *a)
{
    if (!a) return;
    free(a->g); free(a->supply); free(a->out_head); free(a->out_tail);
    free(a->out_next); free(a->depth); free(a);
}

/* Algorithm 1 (goto) followed by Algorithm 2 (supply). NULL on failure. */
orc_ac *orc_ac_build(const uint8_t *P, int64_t d, int32_t m)
{
    if (d < 1 || m < 1) return NULL;
    int64_t maxs = d * (int64_t)m + 1;
    orc_ac *a = (orc_ac *)calloc(1, sizeof(orc_ac));
    if (!a) return NULL;
    a->m = m;
    a->d = d;
    a->g = (int32_t *)malloc((size_t)maxs * ORC_SIGMA * sizeof(int32_t));
    a->supply = (int32_t *)calloc((size_t)maxs, sizeof(int32_t));
    a->out_head = (int64_t *)malloc((size_t)maxs * sizeof(int64_t));
    a->out_tail = (int64_t *)malloc((size_t)maxs * sizeof(int64_t));
    a->out_next = (int64_t *)malloc((size_t)d * sizeof(int64_t));
    a->depth = (int32_t *)calloc((size_t)maxs, sizeof(int32_t));
    if (!a->g || !a->supply || !a->out_head || !a->out_tail || !a->out_next || !a->depth) {
        orc_ac_free(a);
        return NULL;
    }

    /* Algorithm 1: create q_0 with every transition undefined */
    a->nstates = 1;
    for (int c = 0; c < ORC_SIGMA; c++) a->g[c] = ORC_FAIL;
    a->out_head[0] = a->out_tail[0] = -1;

    for (int64_t i = 0; i < d; i++) {
        const uint8_t *p = P + i * (int64_t)m;
        int32_t state = 0;
        int32_t j = 0;
        /* follow the existing path as far as it goes */
        while (j < m && a->g[(int64_t)state * ORC_SIGMA + p[j]] != ORC_FAIL) {
            state = a->g[(int64_t)state * ORC_SIGMA + p[j]];
            j++;
        }
        /* create a new state for each remaining character */
        for (int32_t l = j; l < m; l++) {
            int32_t q = (int32_t)a->nstates++;
            for (int c = 0; c < ORC_SIGMA; c++) a->g[(int64_t)q * ORC_SIGMA + c] = ORC_FAIL;
            a->out_head[q] = a->out_tail[q] = -1;
            a->depth[q] = a->depth[state] + 1;
            a->g[(int64_t)state * ORC_SIGMA + p[l]] = q;
            state = q;
        }
        /* Output(state) := Output(state) U {p^i}; appended, so ascending i */
        a->out_next[i] = -1;
        if (a->out_tail[state] < 0) a->out_head[state] = i;
        else a->out_next[a->out_tail[state]] = i;
        a->out_tail[state] = i;
    }

    /* Algorithm 2: root self-loops and depth-1 supply links */
    int32_t *queue = (int32_t *)malloc((size_t)a->nstates * sizeof(int32_t));
    if (!queue) { orc_ac_free(a); return NULL; }
    int64_t qh = 0, qt = 0;
    for (int c = 0; c < ORC_SIGMA; c++) {
        int32_t s = a->g[c];
        if (s == ORC_FAIL) {
            a->g[c] = 0;
        } else {
            a->supply[s] = 0;
            queue[qt++] = s;
        }
    }
    /* remaining states in breadth-first ("transversal") order */
    while (qh < qt) {
        int32_t cur = queue[qh++];
        for (int c = 0; c < ORC_SIGMA; c++) {
            int32_t s = a->g[(int64_t)cur * ORC_SIGMA + c];
            if (s == ORC_FAIL) continue;
            int32_t st = a->supply[cur];
            while (a->g[(int64_t)st * ORC_SIGMA + c] == ORC_FAIL) st = a->supply[st];
            a->supply[s] = a->g[(int64_t)st * ORC_SIGMA + c];
            queue[qt++] = s;
        }
    }
    free(queue);
    return a;
}

int64_t orc_ac_nstates(const orc_ac *a) { return a->nstates; }

/* g(q, c) after Algorithm 2 (root self-loops filled in); FAIL = -1 */
int32_t orc_ac_goto(const orc_ac *a, int64_t q, int32_t c)
{
    return a->g[q * ORC_SIGMA + (c & 0xff)];
}

int32_t orc_ac_supply(const orc_ac *a, int64_t q) { return a->supply[q]; }

int32_t orc_ac_depth(const orc_ac *a, int64_t q) { return a->depth[q]; }

/* first pattern index in Output(q), or -1; orc_ac_output_next walks the set */
int64_t orc_ac_output_first(const orc_ac *a, int64_t q) { return a->out_head[q]; }
int64_t orc_ac_output_next(const orc_ac *a, int64_t r) { return a->out_next[r]; }

/* Algorithm 3: one pass over T following supply links on a failed goto.   */
/* A non-empty Output(state) at i reports every pattern in it at i-m+1.    */
int64_t orc_ac_search(const orc_ac *a, const uint8_t *T, int64_t n,
                      uint64_t *occ, int64_t cap, int64_t *counts)
{
    int64_t total = 0;
    for (int64_t r = 0; r < a->d; r++) counts[r] = 0;
    int32_t state = 0;
    for (int64_t i = 0; i < n; i++) {
        int32_t ns;
        while ((ns = a->g[(int64_t)state * ORC_SIGMA + T[i]]) == ORC_FAIL)
            state = a->supply[state];
        state = ns;
        for (int64_t r = a->out_head[state]; r >= 0; r = a->out_next[r]) {
            if (total < cap) occ[total] = ORC_OCC(i - a->m + 1, r);
            total++;
            counts[r]++;
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* CPU baseline: the same automaton as a full DFA (goto and supply merged,   */
/* the "array of size |Sigma|" form of Section 3.1) over byte classes, walked */
/* by nthreads threads, each over a contiguous range of start positions plus */
/* the m-1 characters after it (Section 4.2.1's chunk-with-overlap split,    */
/* here over host threads). Not a parity route: it exists to be timed.       */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int32_t *dfa;     /* nstates x ncls */
    const uint8_t *cls;     /* byte -> class (0 = a byte in no pattern) */
    const orc_ac *a;
    int32_t ncls;
    const uint8_t *T;
    int64_t n, i0, i1;      /* start positions [i0, i1) */
    uint64_t *buf;
    int64_t len, cap;
    int64_t *counts;
    int failed;
} orc_dfa_job;

static void *orc_dfa_worker(void *arg)
{
    orc_dfa_job *jb = (orc_dfa_job *)arg;
    const int32_t m = jb->a->m;
    int64_t end = jb->i1 + m - 1;
    if (end > jb->n) end = jb->n;
    int32_t q = 0;
    for (int64_t e = jb->i0; e < end; e++) {
        q = jb->dfa[(int64_t)q * jb->ncls + jb->cls[jb->T[e]]];
        for (int64_t r = jb->a->out_head[q]; r >= 0; r = jb->a->out_next[r]) {
            if (jb->len == jb->cap) {
                int64_t nc = jb->cap ? 2 * jb->cap : 4096;
                uint64_t *nb = (uint64_t *)realloc(jb->buf, (size_t)nc * sizeof(uint64_t));
                if (!nb) { jb->failed = 1; return NULL; }
                jb->buf = nb;
                jb->cap = nc;
            }
            jb->buf[jb->len++] = ORC_OCC(e - m + 1, r);
            jb->counts[r]++;
        }
    }
    return NULL;
}

int64_t orc_ac_dfa_scan(const orc_ac *a, const uint8_t *T, int64_t n, int32_t nthreads,
                        uint64_t *occ, int64_t cap, int64_t *counts)
{
    for (int64_t r = 0; r < a->d; r++) counts[r] = 0;
    const int32_t m = a->m;
    if (n < m) return 0;
    /* byte classes: each byte that leaves the root or any state, in byte order */
    uint8_t cls[ORC_SIGMA];
    int32_t ncls = 1;
    for (int c = 0; c < ORC_SIGMA; c++) {
        int used = 0;
        for (int64_t q = 0; q < a->nstates && !used; q++) {
            int32_t t = a->g[q * ORC_SIGMA + c];
            used = t != ORC_FAIL && t != 0;
        }
        cls[c] = used ? (uint8_t)ncls++ : 0;
    }
    /* breadth-first order from the depths, then delta(q, c) = g(q, c) if
     * defined, else delta(Supply(q), c) (Supply(q) is shallower) */
    int64_t ns = a->nstates;
    int32_t *dfa = (int32_t *)malloc((size_t)ns * (size_t)ncls * sizeof(int32_t));
    int64_t *order = (int64_t *)malloc((size_t)ns * sizeof(int64_t));
    int64_t *first = (int64_t *)calloc((size_t)m + 2, sizeof(int64_t));
    if (!dfa || !order || !first) { free(dfa); free(order); free(first); return -1; }
    for (int64_t q = 0; q < ns; q++) first[a->depth[q] + 1]++;
    for (int32_t k = 1; k <= m + 1; k++) first[k] += first[k - 1];
    for (int64_t q = 0; q < ns; q++) order[first[a->depth[q]]++] = q;
    int32_t rep[ORC_SIGMA];   /* a byte of each class */
    for (int c = ORC_SIGMA - 1; c >= 0; c--) rep[cls[c]] = c;
    for (int64_t k = 0; k < ns; k++) {
        const int64_t q = order[k];
        for (int32_t c = 0; c < ncls; c++) {
            int32_t t = c == 0 ? ORC_FAIL : a->g[q * ORC_SIGMA + rep[c]];
            if (q == 0) dfa[c] = (t == ORC_FAIL) ? 0 : t;
            else dfa[q * ncls + c] = (t == ORC_FAIL) ? dfa[(int64_t)a->supply[q] * ncls + c] : t;
        }
    }
    free(order);
    free(first);

    if (nthreads < 1) nthreads = 1;
    int64_t nwin = n - m + 1;
    if (nthreads > nwin) nthreads = (int32_t)nwin;
    orc_dfa_job *jobs = (orc_dfa_job *)calloc((size_t)nthreads, sizeof(orc_dfa_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tids) { free(dfa); free(jobs); free(tids); return -1; }
    int failed = 0;
    for (int32_t t = 0; t < nthreads; t++) {
        jobs[t].dfa = dfa; jobs[t].cls = cls; jobs[t].a = a; jobs[t].ncls = ncls;
        jobs[t].T = T; jobs[t].n = n;
        jobs[t].i0 = (nwin * t) / nthreads;        /* thread t's start positions */
        jobs[t].i1 = (nwin * (t + 1)) / nthreads;
        jobs[t].counts = (int64_t *)calloc((size_t)a->d, sizeof(int64_t));
        if (!jobs[t].counts) failed = 1;
    }
    if (!failed) {
        for (int32_t t = 0; t < nthreads; t++) pthread_create(&tids[t], NULL, orc_dfa_worker, &jobs[t]);
        for (int32_t t = 0; t < nthreads; t++) pthread_join(tids[t], NULL);
    }
    int64_t total = 0;
    for (int32_t t = 0; t < nthreads; t++) {
        failed |= jobs[t].failed;
        for (int64_t k = 0; k < jobs[t].len; k++) {
            if (total < cap) occ[total] = jobs[t].buf[k];
            total++;
        }
        if (jobs[t].counts)
            for (int64_t r = 0; r < a->d; r++) counts[r] += jobs[t].counts[r];
        free(jobs[t].buf);
        free(jobs[t].counts);
    }
    free(jobs);
    free(tids);
    free(dfa);
    return failed ? -1 : total;
}

/* ------------------------------------------------------------------------ */
/* O2: sequential Wu-Manber, Algorithms 4 and 5 (Section 3.2).               */
/* h1 and h2 are the paper's shift-and-add hash: h := (h << 2) + byte.       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t m, B, Bp;
    int64_t d;
    int64_t tsize;     /* number of h1 values */
    int32_t *shift;    /* SHIFT[h] */
    int64_t *hash_head;/* HASH[h]: first pattern index, chained via hash_next */
    int64_t *hash_tail;
    int64_t *hash_next;
    int64_t *prefix;   /* PREFIX[r] */
    uint8_t *P;        /* private copy of the patterns, for verification */
} orc_wm;

static int64_t orc_wm_h(const uint8_t *s, int32_t len)
{
    int64_t h = 0;
    for (int32_t k = 0; k < len; k++) h = (h << 2) + s[k];
    return h;
}

void orc_wm_free(orc_wm *w)
{
    if (!w) return;
    free(w->shift); free(w->hash_head); free(w->hash_tail); free(w->hash_next);
    free(w->prefix); free(w->P); free(w);
}

/* Algorithm 4. Requires 1 <= B <= m and 1 <= Bp <= m. */
orc_wm *orc_wm_build(const uint8_t *P, int64_t d, int32_t m, int32_t B, int32_t Bp)
{
    if (d < 1 || m < 1 || B < 1 || B > m || Bp < 1 || Bp > m) return NULL;
    orc_wm *w = (orc_wm *)calloc(1, sizeof(orc_wm));
    if (!w) return NULL;
    w->m = m; w->B = B; w->Bp = Bp; w->d = d;
    /* largest h1 value is 255 * (4^B - 1) / 3 */
    int64_t hmax = 0;
    for (int32_t k = 0; k < B; k++) hmax = (hmax << 2) + 255;
    w->tsize = hmax + 1;
    w->shift = (int32_t *)malloc((size_t)w->tsize * sizeof(int32_t));
    w->hash_head = (int64_t *)malloc((size_t)w->tsize * sizeof(int64_t));
    w->hash_tail = (int64_t *)malloc((size_t)w->tsize * sizeof(int64_t));
    w->hash_next = (int64_t *)malloc((size_t)d * sizeof(int64_t));
    w->prefix = (int64_t *)malloc((size_t)d * sizeof(int64_t));
    w->P = (uint8_t *)malloc((size_t)(d * m));
    if (!w->shift || !w->hash_head || !w->hash_tail || !w->hash_next || !w->prefix || !w->P) {
        orc_wm_free(w);
        return NULL;
    }
    memcpy(w->P, P, (size_t)(d * m));
    for (int64_t h = 0; h < w->tsize; h++) {
        w->shift[h] = m - B + 1;
        w->hash_head[h] = w->hash_tail[h] = -1;
    }
    for (int64_t i = 0; i < d; i++) {
        const uint8_t *p = P + i * (int64_t)m;
        for (int32_t q = m; q >= B; q--) {
            int64_t h = orc_wm_h(p + (q - B), B); /* block p_{q-B}..p_{q-1} */
            int32_t shiftlen = m - q;
            if (shiftlen < w->shift[h]) w->shift[h] = shiftlen;
            if (shiftlen == 0) {
                w->hash_next[i] = -1;
                if (w->hash_tail[h] < 0) w->hash_head[h] = i;
                else w->hash_next[w->hash_tail[h]] = i;
                w->hash_tail[h] = i;
                w->prefix[i] = orc_wm_h(p, Bp);
            }
        }
    }
    return w;
}

int64_t orc_wm_tsize(const orc_wm *w) { return w->tsize; }
int32_t orc_wm_shift(const orc_wm *w, int64_t h) { return w->shift[h]; }
int64_t orc_wm_prefix(const orc_wm *w, int64_t r) { return w->prefix[r]; }
int64_t orc_wm_hash_first(const orc_wm *w, int64_t h) { return w->hash_head[h]; }
int64_t orc_wm_hash_next(const orc_wm *w, int64_t r) { return w->hash_next[r]; }

/* Algorithm 5. */
int64_t orc_wm_search(const orc_wm *w, const uint8_t *T, int64_t n,
                      uint64_t *occ, int64_t cap, int64_t *counts)
{
    int64_t total = 0;
    const int32_t m = w->m, B = w->B, Bp = w->Bp;
    for (int64_t r = 0; r < w->d; r++) counts[r] = 0;
    int64_t i = m - 1;
    while (i < n) {
        int64_t h = orc_wm_h(T + (i - B + 1), B); /* block t_{i-B+1}..t_i */
        if (w->shift[h] > 0) {
            i += w->shift[h];
        } else {
            int64_t hp = orc_wm_h(T + (i - m + 1), Bp);
            for (int64_t r = w->hash_head[h]; r >= 0; r = w->hash_next[r]) {
                if (w->prefix[r] != hp) continue;
                if (memcmp(w->P + r * (int64_t)m, T + (i - m + 1), (size_t)m) == 0) {
                    if (total < cap) occ[total] = ORC_OCC(i - m + 1, r);
                    total++;
                    counts[r]++;
                }
            }
            i += 1;
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Variable-length sets: the Section 1 definition with |p^r| = len_r.       */
/* Pattern r is the bytes P[off[r] .. off[r+1]), off[0] = 0.                */
/* ------------------------------------------------------------------------ */

/* The definition as loops over start positions and patterns (ascending),   */
/* so the output is sorted by (i, r) as it is produced.                     */
int64_t orc_brute_var(const uint8_t *T, int64_t n, const uint8_t *P, const int64_t *off,
                      int64_t d, uint64_t *occ, int64_t cap, int64_t *counts)
{
    int64_t total = 0;
    for (int64_t r = 0; r < d; r++) counts[r] = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t r = 0; r < d; r++) {
            const int64_t len = off[r + 1] - off[r];
            if (len < 1 || i + len > n) continue;
            const uint8_t *q = P + off[r];
            int64_t k = 0;
            while (k < len && q[k] == T[i + k]) k++;
            if (k < len) continue;
            if (total < cap) occ[total] = ORC_OCC(i, r);
            total++;
            counts[r]++;
        }
    }
    return total;
}

/* By dictionary membership: the patterns sorted by (length, bytes, r); for  */
/* each start i and each distinct length L, the window T[i..i+L) is located  */
/* by binary search among the length-L patterns; the ids found at i (over    */
/* all lengths) are put in ascending order before they are reported.        */
typedef struct {
    const uint8_t *P;
    const int64_t *off;
} orc_var_ctx;

/* Order of pattern ids ra, rb: by length, then bytes, then id. */
static int orc_cmp_var(const void *ctx, int64_t ra, int64_t rb)
{
    const orc_var_ctx *c = (const orc_var_ctx *)ctx;
    const int64_t la = c->off[ra + 1] - c->off[ra];
    const int64_t lb = c->off[rb + 1] - c->off[rb];
    if (la != lb) return (la > lb) - (la < lb);
    const int k = memcmp(c->P + c->off[ra], c->P + c->off[rb], (size_t)la);
    if (k) return k;
    return (ra > rb) - (ra < rb);
}

typedef struct {
    const uint8_t *T;
    int64_t n;
    const uint8_t *P;
    const int64_t *off;
    const int64_t *sorted;   /* ids by (length, bytes, r) */
    const int64_t *gfirst;   /* length groups: sorted[gfirst[g] .. gfirst[g+1]) */
    const int64_t *glen;
    int64_t ngroups, d;
    int64_t i0, i1;
    uint64_t *buf;
    int64_t len, cap;
    int64_t *counts;
    int64_t *found;          /* ids found at one start, up to d */
    int failed;
} orc_var_job;

static void *orc_dict_var_worker(void *arg)
{
    orc_var_job *jb = (orc_var_job *)arg;
    for (int64_t i = jb->i0; i < jb->i1; i++) {
        int64_t nf = 0;
        for (int64_t g = 0; g < jb->ngroups; g++) {
            const int64_t L = jb->glen[g];
            if (i + L > jb->n) continue;
            const uint8_t *win = jb->T + i;
            int64_t a = jb->gfirst[g], b = jb->gfirst[g + 1];
            while (a < b) {  /* first pattern of the group not below the window */
                const int64_t h = a + (b - a) / 2;
                if (memcmp(jb->P + jb->off[jb->sorted[h]], win, (size_t)L) >= 0) b = h;
                else a = h + 1;
            }
            for (int64_t k = a; k < jb->gfirst[g + 1]; k++) {
                const int64_t r = jb->sorted[k];
                if (memcmp(jb->P + jb->off[r], win, (size_t)L) != 0) break;
                jb->found[nf++] = r;
            }
        }
        /* ids of different lengths interleave: order them (insertion sort) */
        for (int64_t x = 1; x < nf; x++) {
            const int64_t v = jb->found[x];
            int64_t y = x;
            while (y > 0 && jb->found[y - 1] > v) { jb->found[y] = jb->found[y - 1]; y--; }
            jb->found[y] = v;
        }
        for (int64_t x = 0; x < nf; x++) {
            if (jb->len == jb->cap) {
                const int64_t nc = jb->cap ? 2 * jb->cap : 4096;
                uint64_t *nb = (uint64_t *)realloc(jb->buf, (size_t)nc * sizeof(uint64_t));
                if (!nb) { jb->failed = 1; return NULL; }
                jb->buf = nb;
                jb->cap = nc;
            }
            jb->buf[jb->len++] = ORC_OCC(i, jb->found[x]);
            jb->counts[jb->found[x]]++;
        }
    }
    return NULL;
}

/* Returns the total, or -1 if memory ran out. */
int64_t orc_dict_var(const uint8_t *T, int64_t n, const uint8_t *P, const int64_t *off,
                     int64_t d, int32_t nthreads, uint64_t *occ, int64_t cap, int64_t *counts)
{
    for (int64_t r = 0; r < d; r++) counts[r] = 0;
    if (d < 1 || n < 1) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = (int32_t)n;
    int64_t *sorted = (int64_t *)malloc((size_t)d * sizeof(int64_t));
    int64_t *gfirst = (int64_t *)malloc((size_t)(d + 1) * sizeof(int64_t));
    int64_t *glen = (int64_t *)malloc((size_t)d * sizeof(int64_t));
    orc_var_job *jobs = (orc_var_job *)calloc((size_t)nthreads, sizeof(orc_var_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!sorted || !gfirst || !glen || !jobs || !tids) {
        free(sorted); free(gfirst); free(glen); free(jobs); free(tids);
        return -1;
    }
    int64_t nz = 0;  /* empty patterns match nowhere: left out */
    for (int64_t r = 0; r < d; r++)
        if (off[r + 1] > off[r]) sorted[nz++] = r;
    const orc_var_ctx vctx = {P, off};
    if (orc_sort_idx(sorted, nz, orc_cmp_var, &vctx)) {
        free(sorted); free(gfirst); free(glen); free(jobs); free(tids);
        return -1;
    }
    int64_t ng = 0;
    for (int64_t k = 0; k < nz; k++) {
        const int64_t L = off[sorted[k] + 1] - off[sorted[k]];
        if (ng == 0 || glen[ng - 1] != L) { gfirst[ng] = k; glen[ng] = L; ng++; }
    }
    gfirst[ng] = nz;

    int64_t total = 0;
    int failed = 0;
    for (int32_t t = 0; t < nthreads; t++) {
        orc_var_job *jb = &jobs[t];
        jb->T = T; jb->n = n; jb->P = P; jb->off = off; jb->sorted = sorted;
        jb->gfirst = gfirst; jb->glen = glen; jb->ngroups = ng; jb->d = d;
        jb->i0 = n * t / nthreads;
        jb->i1 = n * (t + 1) / nthreads;
        jb->counts = (int64_t *)calloc((size_t)d, sizeof(int64_t));
        jb->found = (int64_t *)malloc((size_t)d * sizeof(int64_t));
        if (!jb->counts || !jb->found) failed = 1;
    }
    if (!failed) {
        for (int32_t t = 0; t < nthreads; t++) pthread_create(&tids[t], NULL, orc_dict_var_worker, &jobs[t]);
        for (int32_t t = 0; t < nthreads; t++) pthread_join(tids[t], NULL);
        /* workers cover consecutive start ranges: concatenation is sorted */
        for (int32_t t = 0; t < nthreads; t++) {
            if (jobs[t].failed) failed = 1;
            for (int64_t k = 0; k < jobs[t].len; k++) {
                if (total < cap) occ[total] = jobs[t].buf[k];
                total++;
            }
            for (int64_t r = 0; r < d; r++) counts[r] += jobs[t].counts[r];
        }
    }
    for (int32_t t = 0; t < nthreads; t++) { free(jobs[t].buf); free(jobs[t].counts); free(jobs[t].found); }
    free(sorted); free(gfirst); free(glen); free(jobs); free(tids);
    return failed ? -1 : total;
}
