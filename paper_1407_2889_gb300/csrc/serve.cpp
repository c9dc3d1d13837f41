// serve.cpp -- request loop with continuous batching over the batched
// Aho-Corasick scan.
//
// Requests (a pattern set already compiled on the device plus a host text)
// enter a FIFO. A dispatcher thread admits requests from the head while
// their device memory (text, counts, an occurrence buffer of estimated size)
// fits a fixed device arena, forms a batch from everything admitted, and
// launches it on a free stream slot: one copy per text, the descriptors, the
// persistent batched kernel, and a copy of the per-instance totals back. Up
// to max_inflight batches run at once on their own streams, so requests that
// arrive while others are on the GPU are admitted as soon as memory and a
// slot free up, and their copies and kernels overlap the running batches.
// A completion thread takes finished batches (a host callback on the stream
// marks them), re-runs the few instances whose occurrence estimate was too
// small with the exact capacity, copies results to host memory, frees the
// arena blocks, records each request's latency and wakes its waiter.
//
// Each request's result is computed by the same per-instance arithmetic as a
// solo scan (an instance never shares counters or outputs with another), so
// results are identical alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pm_internal.h"

namespace pm {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int64_t kAlign = 256;
// Every request shares the batched launch, where the costliest instances
// are split across CTAs; only a request whose workspace words could exceed
// a slot's runs as its own whole-GPU scan (the plain scan and expand
// kernels).

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// First-fit offset allocator with coalescing free list.
class FreeList {
 public:
    void reset(int64_t cap)
    {
        free_.clear();
        free_[0] = cap;
        cap_ = cap;
        used_ = 0;
    }
    // offset of a block of at least `bytes`, or -1
    int64_t alloc(int64_t bytes)
    {
        bytes = round_up(std::max<int64_t>(bytes, 1), kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const int64_t off = it->first, left = it->second - bytes;
            free_.erase(it);
            if (left > 0) free_[off + bytes] = left;
            used_ += bytes;
            return off;
        }
        return -1;
    }
    void free(int64_t off, int64_t bytes)
    {
        if (off < 0) return;
        bytes = round_up(std::max<int64_t>(bytes, 1), kAlign);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t capacity() const { return cap_; }
    int64_t used() const { return used_; }

 private:
    int64_t cap_ = 0, used_ = 0;
    std::map<int64_t, int64_t> free_;  // offset -> size, coalesced
};

// Device memory of the requests in flight.
class Arena {
 public:
    int init(int64_t bytes)
    {
        bytes = round_up(bytes, kAlign);
        const cudaError_t e = cudaMalloc(&base_, size_t(bytes));
        if (e != cudaSuccess) {
            set_cuda_error(int(e));
            cudaGetLastError();
            base_ = nullptr;
            return PM_ENOMEM;
        }
        fl_.reset(bytes);
        return PM_OK;
    }
    void release()
    {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    int64_t alloc(int64_t bytes) { return fl_.alloc(bytes); }
    void free(int64_t off, int64_t bytes) { fl_.free(off, bytes); }
    uint8_t *base() const { return static_cast<uint8_t *>(base_); }
    int64_t capacity() const { return fl_.capacity(); }
    int64_t used() const { return fl_.used(); }

 private:
    void *base_ = nullptr;
    FreeList fl_;
};

// Page-locked host memory for result arrays, so results leave the device at
// full link speed straight into the arrays the caller receives. Results may
// outlive the server: the pool is freed when the server and every array
// handed out are gone.
struct HostPool {
    std::mutex mu;
    uint8_t *base = nullptr;
    FreeList fl;
    std::unordered_map<int64_t, int64_t> sizes;  // offset -> bytes of live arrays
    int64_t refs = 1;                            // the server + live arrays

    // NULL when the pool is full (the caller falls back to plain memory)
    void *get(int64_t bytes)
    {
        if (!base) return nullptr;
        std::lock_guard<std::mutex> lk(mu);
        const int64_t off = fl.alloc(bytes);
        if (off < 0) return nullptr;
        sizes[off] = bytes;
        ++refs;
        return base + off;
    }
    static void drop(HostPool *p, void *ptr)
    {
        bool last = false;
        {
            std::lock_guard<std::mutex> lk(p->mu);
            if (ptr) {
                const int64_t off = static_cast<uint8_t *>(ptr) - p->base;
                auto it = p->sizes.find(off);
                if (it != p->sizes.end()) {
                    p->fl.free(off, it->second);
                    p->sizes.erase(it);
                }
            }
            last = --p->refs == 0;
        }
        if (last) {
            if (p->base) cudaFreeHost(p->base);
            delete p;
        }
    }
    static void release_result(void *ctx, void *counts, void *occ)
    {
        HostPool *p = static_cast<HostPool *>(ctx);
        if (counts) drop(p, counts);
        if (occ) drop(p, occ);
    }
};

struct Req {
    int64_t id = 0;
    const pm_set *set = nullptr;
    const uint8_t *T = nullptr;
    int64_t n = 0;
    bool list = true;
    Clock::time_point t_submit;
    int64_t text_blk = -1, text_bytes = 0;
    int64_t cnt_blk = -1, cnt_bytes = 0;
    int64_t occ_blk = -1, occ_bytes = 0, occ_cap = 0;
    int64_t ws_bytes = 0;              // workspace of a whole-GPU scan (the slot's)
    bool plain = false;
    void *occ_ext = nullptr;           // re-run buffer outside the arena
    int64_t n_occ = 0;
    int status = PM_OK;
    bool done = false;
    pm_result *res = nullptr;
    bool early = false;                // res is being filled by the batch's own copies
};

struct Slot {
    cudaStream_t st = nullptr;
    BatchDesc *h_desc = nullptr;       // pinned, batch_items_bound(max_batch) queue items
    int64_t *h_nocc = nullptr;         // pinned, max_batch
    BatchDesc *d_desc = nullptr;
    int64_t *d_nocc = nullptr;
    void *d_ws = nullptr;
    int64_t ws_words = 0;              // global counter words the workspace holds
    uint32_t *h_bstat = nullptr;       // pinned: the batched scan's status word
    void *d_pws = nullptr;             // workspace shared by the slot's whole-GPU scans
    int64_t pws_bytes = 0;
    uint32_t *h_pstat = nullptr;       // pinned, max_batch: their status words
    bool busy = false;
    std::vector<Req *> reqs;
    std::atomic<bool> ready{false};
    Clock::time_point t_launch;
};

}  // namespace
}  // namespace pm

struct pm_server {
    pm_server_params p{};
    int device = 0;
    pm::BatchShape shape;
    pm::Arena arena;
    std::vector<pm::Slot *> slots;
    std::mutex mu;
    std::condition_variable cv_dispatch, cv_complete, cv_done;
    std::deque<pm::Req *> pending;
    std::unordered_map<int64_t, pm::Req *> by_id;
    std::unordered_map<const pm_set *, double> rate;   // occurrences per text byte seen
    int64_t next_id = 1;
    bool stopping = false;
    std::thread dispatcher;
    std::vector<std::thread> completers;   // one per slot
    pm::HostPool *pool = nullptr;
    // statistics
    std::vector<double> lat_us;
    int64_t bytes_done = 0, batches = 0, batched_reqs = 0, reruns = 0, peak_inflight = 0;
    int64_t inflight_reqs = 0;
    double dispatch_busy_s = 0.0, complete_busy_s = 0.0;
    bool have_first = false;
    pm::Clock::time_point t_first, t_last;
};

namespace pm {
namespace {

void CUDART_CB on_batch_done(void *arg)
{
    // runs on a CUDA callback thread: no CUDA calls here
    auto *pr = static_cast<std::pair<pm_server *, Slot *> *>(arg);
    {
        std::lock_guard<std::mutex> lk(pr->first->mu);
        pr->second->ready.store(true);
    }
    pr->first->cv_complete.notify_all();
    delete pr;
}

int64_t est_cap(pm_server *s, const Req &r)
{
    if (!r.list) return 0;
    auto it = s->rate.find(r.set);
    const double rate = it == s->rate.end() ? 1.0 / 16.0 : it->second;
    return int64_t(double(r.n) * rate * 1.25) + 256;
}

// Arena blocks of one request; false (nothing held) when they do not fit.
bool admit(pm_server *s, Req &r)
{
    const int64_t d = r.set->ac.d;
    r.text_bytes = std::max<int64_t>(r.n, 1);
    r.cnt_bytes = d * 8;
    r.occ_cap = est_cap(s, r);
    r.occ_bytes = r.list ? std::max<int64_t>(r.occ_cap, 1) * 8 : 0;
    {
        const BatchInst I{r.set, 0, r.n, 0, 0, r.list ? r.occ_cap : 0, 0};
        r.plain = batch_words_bound(I, s->shape, r.list) > s->p.counter_words;
    }
    r.ws_bytes = r.plain ? pm_scan_workspace_bytes(r.set, r.n, r.list ? 0u : PM_COUNTS_ONLY) : 0;
    r.text_blk = s->arena.alloc(r.text_bytes);
    if (r.text_blk < 0) return false;
    r.cnt_blk = s->arena.alloc(r.cnt_bytes);
    if (r.cnt_blk < 0) {
        s->arena.free(r.text_blk, r.text_bytes);
        r.text_blk = -1;
        return false;
    }
    if (r.list) {
        r.occ_blk = s->arena.alloc(r.occ_bytes);
        if (r.occ_blk < 0) {
            s->arena.free(r.text_blk, r.text_bytes);
            s->arena.free(r.cnt_blk, r.cnt_bytes);
            r.text_blk = r.cnt_blk = -1;
            return false;
        }
    }
    return true;
}

// Arena blocks back to the free list (caller holds the lock; a buffer
// outside the arena is handed back for cudaFree after the lock is dropped:
// a CUDA call under the lock could wait on a stream callback that waits on
// the lock).
void *release(pm_server *s, Req &r)
{
    s->arena.free(r.text_blk, r.text_bytes);
    s->arena.free(r.cnt_blk, r.cnt_bytes);
    if (r.occ_blk >= 0) s->arena.free(r.occ_blk, r.occ_bytes);
    r.text_blk = r.cnt_blk = r.occ_blk = -1;
    void *ext = r.occ_ext;
    r.occ_ext = nullptr;
    return ext;
}

// Workspace words a request may add to a batch (0: it runs as a whole-GPU
// scan with its own workspace).
int64_t counter_words(pm_server *s, const Req &r)
{
    const BatchInst I{r.set, 0, r.n, 0, 0, r.list ? est_cap(s, r) : 0, 0};
    const int64_t w = batch_words_bound(I, s->shape, r.list);
    return w > s->p.counter_words ? 0 : w;
}

// A whole-GPU scan of one request, its keys going to `occ`, its total to
// d_nocc (asynchronous on the stream).
int launch_plain(pm_server *s, const Req &r, uint64_t *occ, int64_t cap, int64_t *d_nocc, void *ws,
                 cudaStream_t st)
{
    uint8_t *base = s->arena.base();
    return ac_launch(r.set->ac, r.set->dac, base + r.text_blk, r.n, r.list,
                     reinterpret_cast<int64_t *>(base + r.cnt_blk), r.list ? occ : nullptr, cap, d_nocc,
                     ws, st);
}

// The slot's whole-GPU scans run one after another on its stream and share
// one workspace; grow it when a request needs more (the slot is idle here).
int ensure_pws(Slot &sl, int64_t need)
{
    if (need <= sl.pws_bytes) return PM_OK;
    if (sl.d_pws) cudaFree(sl.d_pws);
    sl.d_pws = nullptr;
    sl.pws_bytes = 0;
    const cudaError_t e = cudaMalloc(&sl.d_pws, size_t(need));
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        cudaGetLastError();
        sl.d_pws = nullptr;
        return PM_ENOMEM;
    }
    sl.pws_bytes = need;
    return PM_OK;
}

// Enqueue the batch of slot `sl` (texts in, kernel, totals out); the caller
// holds no lock. Returns a PM code.
int launch_slot(pm_server *s, Slot &sl)
{
    const int k = int(sl.reqs.size());
    std::vector<BatchInst> inst;
    for (int j = 0; j < k; ++j) {
        const Req &r = *sl.reqs[size_t(j)];
        if (r.plain) continue;
        const int64_t occ_off = r.list ? r.occ_blk / 8 : 0;
        inst.push_back(BatchInst{r.set, r.text_blk, r.n, r.cnt_blk / 8, occ_off, r.list ? r.occ_cap : 0, j});
    }
    // queue items: costliest first, large requests split across CTAs
    std::vector<BatchDesc> items;
    int64_t spill = 0;
    const int64_t words = batch_items(inst.data(), int(inst.size()), s->shape, true, items, &spill);
    const int kb = int(items.size());
    if (words + spill > sl.ws_words || int64_t(kb) > batch_items_bound(s->p.max_batch, s->shape))
        return PM_EINVAL;  // admission keeps this from happening
    if (kb > 0) std::memcpy(sl.h_desc, items.data(), size_t(kb) * sizeof(BatchDesc));
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < k && e == cudaSuccess; ++j) {
        const Req &r = *sl.reqs[size_t(j)];
        if (r.n > 0)
            e = cudaMemcpyAsync(s->arena.base() + r.text_blk, r.T, size_t(r.n), cudaMemcpyHostToDevice, sl.st);
    }
    if (e == cudaSuccess && kb > 0)
        e = cudaMemcpyAsync(sl.d_desc, sl.h_desc, size_t(kb) * sizeof(BatchDesc), cudaMemcpyHostToDevice, sl.st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    uint8_t *base = s->arena.base();
    int rc = PM_OK;
    *sl.h_bstat = 0;
    if (kb > 0) {
        rc = batch_launch_raw(sl.d_desc, kb, base, reinterpret_cast<int64_t *>(base),
                              reinterpret_cast<uint64_t *>(base), sl.d_nocc, sl.d_ws, words, s->shape,
                              true, sl.st);
        if (rc == PM_OK) {
            e = cudaMemcpyAsync(sl.h_bstat, sl.d_ws, 4, cudaMemcpyDeviceToHost, sl.st);
            if (e != cudaSuccess) { set_cuda_error(int(e)); rc = PM_ECUDA; }
        }
    }
    int64_t pws = 0;
    for (const Req *r : sl.reqs)
        if (r->plain) pws = std::max(pws, r->ws_bytes);
    if (rc == PM_OK && pws > 0) rc = ensure_pws(sl, pws);
    for (int j = 0; j < k && rc == PM_OK; ++j) {
        const Req &r = *sl.reqs[size_t(j)];
        if (!r.plain) continue;
        rc = launch_plain(s, r, reinterpret_cast<uint64_t *>(base + r.occ_blk), r.occ_cap, sl.d_nocc + j,
                          sl.d_pws, sl.st);
        // the next scan clears the shared status word: keep this one's
        if (rc == PM_OK) {
            e = cudaMemcpyAsync(sl.h_pstat + j, sl.d_pws, 4, cudaMemcpyDeviceToHost, sl.st);
            if (e != cudaSuccess) { set_cuda_error(int(e)); rc = PM_ECUDA; }
        }
    }
    if (rc) return rc;
    // results straight into page-locked host memory behind the kernels (the
    // estimated capacity of keys), so a batch whose estimates hold needs no
    // copy after it completes; without pool room the completion copies them
    for (int j = 0; j < k && s->pool; ++j) {
        Req &r = *sl.reqs[size_t(j)];
        r.early = false;
        const int64_t d = r.set->ac.d, cap = r.list ? r.occ_cap : 0;
        void *pc = s->pool->get(d * 8);
        void *po = r.list ? s->pool->get(std::max<int64_t>(cap, 1) * 8) : nullptr;
        pm_result *res = (pc && (po || !r.list))
                             ? make_result_owned(d, 0, static_cast<int64_t *>(pc), static_cast<uint64_t *>(po),
                                                 &HostPool::release_result, s->pool)
                             : nullptr;
        if (!res) { HostPool::release_result(s->pool, pc, po); continue; }
        e = cudaMemcpyAsync(res->counts, base + r.cnt_blk, size_t(r.cnt_bytes), cudaMemcpyDeviceToHost, sl.st);
        if (e == cudaSuccess && cap > 0)
            e = cudaMemcpyAsync(res->occ, base + r.occ_blk, size_t(cap) * 8, cudaMemcpyDeviceToHost, sl.st);
        r.res = res;
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        r.early = true;
    }
    e = cudaMemcpyAsync(sl.h_nocc, sl.d_nocc, size_t(k) * 8, cudaMemcpyDeviceToHost, sl.st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    return PM_OK;
}

void finish(pm_server *s, Req &r, int status)
{
    // caller holds the lock
    r.status = status;
    r.done = true;
    const auto now = Clock::now();
    if (status == PM_OK) {
        s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_submit).count());
        s->bytes_done += r.n;
        s->t_last = now;
    }
}

void dispatcher_main(pm_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        Slot *free_slot = nullptr;
        for (Slot *sl : s->slots)
            if (!sl->busy) { free_slot = sl; break; }
        if (s->stopping && s->pending.empty()) break;
        if (!free_slot || s->pending.empty()) {
            s->cv_dispatch.wait(lk);
            continue;
        }
        // admit from the head while memory, batch size and counters allow
        std::vector<Req *> batch;
        int64_t words = 0;
        while (!s->pending.empty() && int(batch.size()) < s->p.max_batch) {
            Req *r = s->pending.front();
            const int64_t w = counter_words(s, *r);
            if (words + w > free_slot->ws_words && !batch.empty()) break;
            if (!admit(s, *r)) break;
            words += w;
            batch.push_back(r);
            s->pending.pop_front();
        }
        if (batch.empty()) {
            bool any_busy = false;
            for (Slot *sl : s->slots) any_busy = any_busy || sl->busy;
            if (!any_busy) {
                // nothing holds memory and the head still does not fit (its
                // estimate grew since it was accepted): it never will
                Req *r = s->pending.front();
                s->pending.pop_front();
                finish(s, *r, PM_ENOMEM);
                s->cv_done.notify_all();
                continue;
            }
            // the head does not fit while batches hold memory: wait for one
            s->cv_dispatch.wait(lk);
            continue;
        }
        free_slot->busy = true;
        free_slot->ready.store(false);
        free_slot->reqs = batch;
        free_slot->t_launch = Clock::now();
        s->inflight_reqs += int64_t(batch.size());
        s->peak_inflight = std::max(s->peak_inflight, s->inflight_reqs);
        s->batches += 1;
        s->batched_reqs += int64_t(batch.size());
        lk.unlock();
        const auto tb0 = Clock::now();
        int rc = launch_slot(s, *free_slot);
        if (rc == PM_OK) {
            auto *arg = new (std::nothrow) std::pair<pm_server *, Slot *>(s, free_slot);
            cudaError_t e = arg ? cudaLaunchHostFunc(free_slot->st, on_batch_done, arg) : cudaErrorMemoryAllocation;
            if (e != cudaSuccess) {
                delete arg;
                set_cuda_error(int(e));
                rc = PM_ECUDA;
            }
        }
        lk.lock();
        s->dispatch_busy_s += std::chrono::duration<double>(Clock::now() - tb0).count();
        if (rc != PM_OK) {
            // the stream may still hold copies: drain it, then fail the batch
            lk.unlock();
            cudaStreamSynchronize(free_slot->st);
            cudaGetLastError();
            lk.lock();
            for (Req *r : free_slot->reqs) {
                release(s, *r);  // nothing outside the arena before a re-run
                if (r->res) pm_result_free(r->res);
                r->res = nullptr;
                r->early = false;
                finish(s, *r, rc);
            }
            s->inflight_reqs -= int64_t(free_slot->reqs.size());
            free_slot->reqs.clear();
            free_slot->busy = false;
            s->cv_done.notify_all();
        }
    }
}

// One instance again with the exact capacity, its keys going to `occ`
// (arena or not): a batch of one whose occurrence base is that buffer.
// Synchronous on the slot's stream; the slot's batch has finished.
int rerun_one(pm_server *s, Slot &sl, Req &r, uint64_t *occ)
{
    cudaError_t e = cudaSuccess;
    int rc = PM_OK;
    if (r.plain) {
        rc = ensure_pws(sl, r.ws_bytes);
        if (rc == PM_OK) rc = launch_plain(s, r, occ, r.occ_cap, sl.d_nocc, sl.d_pws, sl.st);
    } else {
        // split across CTAs when the parts' words fit the slot's workspace
        BatchInst I{r.set, r.text_blk, r.n, r.cnt_blk / 8, 0, r.occ_cap, 0};
        std::vector<BatchDesc> items;
        int64_t spill = 0;
        int64_t words = batch_items(&I, 1, s->shape, true, items, &spill);
        if (words + spill > sl.ws_words) {
            items.assign(1, BatchDesc());
            words = batch_fill(&I, 1, s->shape, items.data());
        }
        std::memcpy(sl.h_desc, items.data(), items.size() * sizeof(BatchDesc));
        e = cudaMemcpyAsync(sl.d_desc, sl.h_desc, items.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice, sl.st);
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        uint8_t *base = s->arena.base();
        rc = batch_launch_raw(sl.d_desc, int(items.size()), base, reinterpret_cast<int64_t *>(base), occ,
                              sl.d_nocc, sl.d_ws, words, s->shape, true, sl.st);
    }
    if (rc) return rc;
    e = cudaMemcpyAsync(sl.h_nocc, sl.d_nocc, 8, cudaMemcpyDeviceToHost, sl.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sl.st);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    if (pm_scan_status(r.plain ? sl.d_pws : sl.d_ws, sl.st) != PM_OK) return PM_ETIMEOUT;
    return sl.h_nocc[0] == r.n_occ ? PM_OK : PM_ECUDA;  // same scan, same total
}

// Finish one completed slot: re-runs, host copies, bookkeeping.
void complete_slot(pm_server *s, Slot &sl, std::unique_lock<std::mutex> &lk)
{
    const int k = int(sl.reqs.size());
    std::vector<Req *> over;
    for (int j = 0; j < k; ++j) {
        Req &r = *sl.reqs[size_t(j)];
        r.n_occ = sl.h_nocc[j];
        if (r.list && r.n_occ > r.occ_cap) over.push_back(&r);
    }
    int rc = PM_OK;
    lk.unlock();
    if (*sl.h_bstat != 0) rc = PM_ETIMEOUT;
    for (int j = 0; j < k; ++j)
        if (rc == PM_OK && sl.reqs[size_t(j)]->plain && sl.h_pstat[j] != 0) rc = PM_ETIMEOUT;
    if (!over.empty() && rc == PM_OK) {
        // exact capacity for the instances whose estimate was short: a new
        // arena block, else a buffer of its own
        lk.lock();
        for (Req *r : over) {
            if (r->res) pm_result_free(r->res);  // its early copy was too short
            r->res = nullptr;
            r->early = false;
            s->arena.free(r->occ_blk, r->occ_bytes);
            r->occ_bytes = r->n_occ * 8;
            r->occ_cap = r->n_occ;
            r->occ_blk = s->arena.alloc(r->occ_bytes);
        }
        s->reruns += int64_t(over.size());
        lk.unlock();
        for (Req *r : over) {
            if (rc != PM_OK) break;
            if (r->occ_blk < 0) {
                const cudaError_t e = cudaMalloc(&r->occ_ext, size_t(r->occ_bytes));
                if (e != cudaSuccess) { cudaGetLastError(); r->occ_ext = nullptr; rc = PM_ENOMEM; break; }
            }
            uint64_t *o = r->occ_ext ? static_cast<uint64_t *>(r->occ_ext)
                                     : reinterpret_cast<uint64_t *>(s->arena.base() + r->occ_blk);
            rc = rerun_one(s, sl, *r, o);
        }
    }
    // results to host memory
    std::vector<int> rcs(static_cast<size_t>(k), rc);
    for (int j = 0; j < k; ++j) {
        Req &r = *sl.reqs[size_t(j)];
        if (rcs[size_t(j)] != PM_OK) continue;
        if (r.early) {  // already in host memory
            r.res->n_occ = r.n_occ;
            continue;
        }
        const int64_t d = r.set->ac.d, no = r.list ? r.n_occ : 0;
        void *pc = s->pool->get(d * 8);
        void *po = r.list ? s->pool->get(std::max<int64_t>(no, 1) * 8) : nullptr;
        if (pc && (po || !r.list)) {
            r.res = make_result_owned(d, r.n_occ, static_cast<int64_t *>(pc), static_cast<uint64_t *>(po),
                                      &HostPool::release_result, s->pool);
            if (!r.res) HostPool::release_result(s->pool, pc, po);
        } else {
            HostPool::release_result(s->pool, pc, po);
            r.res = make_result(d, no, r.list);  // pool full: plain host arrays
        }
        if (!r.res) { rcs[size_t(j)] = PM_ENOMEM; continue; }
        r.res->n_occ = r.n_occ;
        cudaError_t e = cudaMemcpyAsync(r.res->counts, s->arena.base() + r.cnt_blk, size_t(r.cnt_bytes),
                                        cudaMemcpyDeviceToHost, sl.st);
        if (e == cudaSuccess && r.list && r.n_occ > 0) {
            const uint8_t *o = r.occ_ext ? static_cast<uint8_t *>(r.occ_ext) : s->arena.base() + r.occ_blk;
            e = cudaMemcpyAsync(r.res->occ, o, size_t(r.n_occ) * 8, cudaMemcpyDeviceToHost, sl.st);
        }
        if (e != cudaSuccess) { set_cuda_error(int(e)); rcs[size_t(j)] = PM_ECUDA; }
    }
    if (cudaStreamSynchronize(sl.st) != cudaSuccess) {
        cudaGetLastError();
        for (int &x : rcs) if (x == PM_OK) x = PM_ECUDA;
    }
    lk.lock();
    std::vector<void *> ext;
    for (int j = 0; j < k; ++j) {
        Req &r = *sl.reqs[size_t(j)];
        if (rcs[size_t(j)] != PM_OK && r.res) {
            pm_result_free(r.res);
            r.res = nullptr;
        }
        if (r.list && rcs[size_t(j)] == PM_OK && r.n > 0) {
            const double obs = double(r.n_occ) / double(r.n);
            auto it = s->rate.find(r.set);
            const double prev = it == s->rate.end() ? obs : it->second;
            s->rate[r.set] = std::max(obs, 0.98 * prev);
        }
        if (void *x = release(s, r)) ext.push_back(x);
        finish(s, r, rcs[size_t(j)]);
    }
    s->inflight_reqs -= int64_t(k);
    sl.reqs.clear();
    sl.busy = false;
    s->cv_done.notify_all();
    s->cv_dispatch.notify_all();
    if (!ext.empty()) {
        lk.unlock();
        for (void *x : ext) cudaFree(x);
        lk.lock();
    }
}

// One completion thread per slot, so batches that finish together are
// finished in parallel (their copies run on their own streams).
void completer_main(pm_server *s, Slot *sl)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        if (sl->busy && sl->ready.load()) {
            sl->ready.store(false);
            const auto tb0 = Clock::now();
            complete_slot(s, *sl, lk);
            s->complete_busy_s += std::chrono::duration<double>(Clock::now() - tb0).count();
            continue;
        }
        if (s->stopping && !sl->busy && s->pending.empty()) break;
        s->cv_complete.wait_for(lk, std::chrono::milliseconds(50));
    }
}

void destroy(pm_server *s)
{
    for (Slot *sl : s->slots) {
        if (sl->st) cudaStreamDestroy(sl->st);
        if (sl->h_desc) cudaFreeHost(sl->h_desc);
        if (sl->h_nocc) cudaFreeHost(sl->h_nocc);
        if (sl->h_pstat) cudaFreeHost(sl->h_pstat);
        if (sl->h_bstat) cudaFreeHost(sl->h_bstat);
        if (sl->d_pws) cudaFree(sl->d_pws);
        if (sl->d_desc) cudaFree(sl->d_desc);
        if (sl->d_nocc) cudaFree(sl->d_nocc);
        if (sl->d_ws) cudaFree(sl->d_ws);
        delete sl;
    }
    s->slots.clear();
    s->arena.release();
    if (s->pool) HostPool::drop(s->pool, nullptr);  // the server's reference
    s->pool = nullptr;
    for (auto &kv : s->by_id) {
        if (kv.second->res) pm_result_free(kv.second->res);
        delete kv.second;
    }
    s->by_id.clear();
    delete s;
}

}  // namespace
}  // namespace pm

using namespace pm;

extern "C" {

int pm_server_create(const pm_server_params *params, pm_server **out)
{
    if (!out) return PM_EINVAL;
    pm_server_params p{};
    if (params) p = *params;
    if (p.device_budget_bytes <= 0) p.device_budget_bytes = int64_t(4) << 30;
    if (p.max_batch <= 0) p.max_batch = 512;
    if (p.max_inflight <= 0) p.max_inflight = 3;
    if (p.warps_per_cta <= 0) p.warps_per_cta = 12;
    if (p.counter_words <= 0) p.counter_words = int64_t(4) << 20;
    if (p.host_pool_bytes == 0) p.host_pool_bytes = int64_t(1) << 30;
    if (p.max_inflight > 16 || p.max_batch > (1 << 20)) return PM_EINVAL;
    pm_server *s = new (std::nothrow) pm_server();
    if (!s) return PM_ENOMEM;
    s->p = p;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) { set_cuda_error(int(e)); cudaGetLastError(); delete s; return PM_ENODEV; }
    int rc = batch_shape(p.warps_per_cta, s->shape);
    if (!rc) rc = batch_prepare_launch(s->shape);
    if (!rc) rc = s->arena.init(p.device_budget_bytes);
    if (!rc) {
        s->pool = new (std::nothrow) HostPool();
        if (!s->pool) rc = PM_ENOMEM;
    }
    if (!rc && p.host_pool_bytes > 0) {
        const int64_t hb = round_up(p.host_pool_bytes, kAlign);
        void *hp = nullptr;
        if (cudaMallocHost(&hp, size_t(hb)) == cudaSuccess) {
            s->pool->base = static_cast<uint8_t *>(hp);
            s->pool->fl.reset(hb);
        } else {
            cudaGetLastError();  // no page-locked pool: results use plain memory
        }
    }
    for (int i = 0; i < p.max_inflight && !rc; ++i) {
        Slot *sl = new (std::nothrow) Slot();
        if (!sl) { rc = PM_ENOMEM; break; }
        s->slots.push_back(sl);
        sl->ws_words = p.counter_words;
        e = cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking);
        const size_t items = size_t(batch_items_bound(p.max_batch, s->shape));
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&sl->h_desc), items * sizeof(BatchDesc));
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&sl->h_nocc), size_t(p.max_batch) * 8);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&sl->h_pstat), size_t(p.max_batch) * 4);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&sl->h_bstat), 4);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&sl->d_desc), items * sizeof(BatchDesc));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&sl->d_nocc), size_t(p.max_batch) * 8);
        if (e == cudaSuccess) e = cudaMalloc(&sl->d_ws, size_t(batch_ws_bytes(p.counter_words)));
        if (e != cudaSuccess) {
            set_cuda_error(int(e));
            cudaGetLastError();
            rc = e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA;
        }
    }
    if (rc) { destroy(s); return rc; }
    try {
        s->dispatcher = std::thread(dispatcher_main, s);
        for (Slot *sl : s->slots) s->completers.emplace_back(completer_main, s, sl);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
        }
        s->cv_dispatch.notify_all();
        s->cv_complete.notify_all();
        if (s->dispatcher.joinable()) s->dispatcher.join();
        for (auto &t : s->completers) if (t.joinable()) t.join();
        destroy(s);
        return PM_ENOMEM;
    }
    *out = s;
    return PM_OK;
}

int pm_server_submit(pm_server *s, const pm_set *set, const uint8_t *T, int64_t n, uint32_t flags,
                     int64_t *ticket)
{
    if (!s || !ticket || n < 0 || (n > 0 && !T)) return PM_EINVAL;
    if (flags & ~(PM_HOST_TEXT | PM_COUNTS_ONLY)) return PM_EINVAL;
    if (!batch_supports(set)) return PM_EINVAL;
    if (n >= (int64_t(1) << 32)) return PM_ETOOBIG;
    Req *r = new (std::nothrow) Req();
    if (!r) return PM_ENOMEM;
    r->set = set;
    r->T = T;
    r->n = n;
    r->list = !(flags & PM_COUNTS_ONLY);
    int64_t need = round_up(std::max<int64_t>(n, 1), kAlign) + round_up(set->ac.d * 8, kAlign) +
                   (r->list ? round_up((est_cap(s, *r) + 1) * 8, kAlign) : 0);
    if (need > s->arena.capacity() || counter_words(s, *r) > s->p.counter_words) {
        delete r;
        return PM_ETOOBIG;  // could never be admitted
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) { delete r; return PM_EINVAL; }
        r->id = s->next_id++;
        r->t_submit = Clock::now();
        if (!s->have_first) { s->have_first = true; s->t_first = r->t_submit; }
        s->by_id[r->id] = r;
        s->pending.push_back(r);
        *ticket = r->id;
    }
    s->cv_dispatch.notify_all();
    return PM_OK;
}

int pm_server_wait(pm_server *s, int64_t ticket, pm_result **out)
{
    if (!s || !out) return PM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->by_id.find(ticket);
    if (it == s->by_id.end()) return PM_EINVAL;
    Req *r = it->second;
    s->cv_done.wait(lk, [&] { return r->done; });
    const int rc = r->status;
    *out = r->res;
    r->res = nullptr;
    s->by_id.erase(ticket);
    delete r;
    return rc;
}

int pm_server_get_stats(pm_server *s, pm_server_stats *st)
{
    if (!s || !st) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof(*st));
    st->completed = int64_t(s->lat_us.size());
    st->bytes = s->bytes_done;
    st->batches = s->batches;
    st->mean_batch = s->batches ? double(s->batched_reqs) / double(s->batches) : 0.0;
    st->reruns = s->reruns;
    st->peak_inflight = s->peak_inflight;
    st->pending = int64_t(s->pending.size());
    st->arena_used = s->arena.used();
    st->dispatch_busy_s = s->dispatch_busy_s;
    st->complete_busy_s = s->complete_busy_s;
    if (!s->lat_us.empty()) {
        std::vector<double> v = s->lat_us;
        auto pct = [&](double q) {
            const size_t i = std::min(v.size() - 1, size_t(q * double(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + long(i), v.end());
            return v[i];
        };
        st->p50_us = pct(0.50);
        st->p99_us = pct(0.99);
        double sum = 0.0;
        for (double x : s->lat_us) sum += x;
        st->mean_us = sum / double(s->lat_us.size());
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        st->gbs = span > 0.0 ? double(s->bytes_done) / span / 1e9 : 0.0;
    }
    return PM_OK;
}

int pm_server_reset_stats(pm_server *s)
{
    if (!s) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_us.clear();
    s->bytes_done = 0;
    s->batches = s->batched_reqs = s->reruns = 0;
    s->peak_inflight = s->inflight_reqs;
    s->dispatch_busy_s = s->complete_busy_s = 0.0;
    s->have_first = false;
    return PM_OK;
}

void pm_server_destroy(pm_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_dispatch.notify_all();
    s->cv_complete.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    for (auto &t : s->completers) if (t.joinable()) t.join();
    destroy(s);
}

}  // extern "C"
