// capi.cpp -- the C ABI of libpmscan (declared in include/pmscan.h): set
// compilation and upload, device-level and host-convenience scans, results,
// errors. No C++ exception crosses this boundary.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pm {

static thread_local int g_last_cuda = 0;
void set_cuda_error(int e) { g_last_cuda = e; }

int64_t warp_tiles(int64_t n) { return n <= 0 ? 0 : (n + kWarpTile - 1) / kWarpTile; }


// The dynamic shared memory a kernel may use is a per-device attribute of
// the kernel: raise it once per (device, kernel) to the largest launch seen,
// under a lock (launchers run on several host threads).
int kernel_smem_attr(const void *fn, int64_t bytes)
{
    static std::mutex mu;
    static std::vector<std::pair<std::pair<int, const void *>, int64_t>> seen;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    std::lock_guard<std::mutex> lk(mu);
    int64_t *have = nullptr;
    for (auto &x : seen)
        if (x.first.first == dev && x.first.second == fn) have = &x.second;
    if (have && *have >= bytes) return PM_OK;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) { set_cuda_error(int(e)); cudaGetLastError(); return PM_ECUDA; }
    if (have) *have = bytes;
    else seen.push_back({{dev, fn}, bytes});
    return PM_OK;
}

int device_props(DeviceProps &p)
{
    static std::mutex mu;
    static DeviceProps cache[64];
    static bool have[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        cudaGetLastError();
        return PM_ENODEV;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && have[dev]) {
        p = cache[dev];
        return PM_OK;
    }
    DeviceProps q;
    e = cudaDeviceGetAttribute(&q.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&q.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&q.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&q.l2_bytes, cudaDevAttrL2CacheSize, dev);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        cudaGetLastError();
        return PM_ENODEV;
    }
    if (dev >= 0 && dev < 64) {
        cache[dev] = q;
        have[dev] = true;
    }
    p = q;
    return PM_OK;
}

namespace {

// Copy `bytes` to a fresh device allocation padded to a multiple of 16.
int upload(void **dst, const void *src, size_t bytes, int64_t &total)
{
    size_t padded = (bytes + 15) & ~size_t(15);
    if (padded == 0) padded = 16;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, padded);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA;
    }
    e = cudaMemset(p, 0, padded);
    if (e == cudaSuccess && bytes) e = cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        cudaFree(p);
        return PM_ECUDA;
    }
    *dst = p;
    total += int64_t(padded);
    return PM_OK;
}

void free_dev(void *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

void release_device(pm_set *s)
{
    void *ptrs[] = {s->dac.table, s->dac.flag_mask, s->dac.flag_rank, s->dac.canon, s->dac.tmul, s->dac.emul,
                    s->dac.grp_off, s->dac.grp_ids, s->dac.cls,
                    s->dwm.shift, s->dwm.hoff, s->dwm.hids, s->dwm.hpfx, s->dwm.pats,
                    s->dwm.shift2, s->dwm.dir, s->dwm.ccode, s->dwm.cr,
                    s->dwm.hcode, s->dwm.grp_off, s->dwm.grp_ids, s->dwm.poff, s->dwm.fcode, s->dwm.flen,
                    s->dacv.table, s->dacv.cls, s->dacv.omask, s->dacv.orank, s->dacv.out_off, s->dacv.out_ent,
                    s->dac2.table2,
                    s->c_text, s->c_ws, s->c_out, s->c_counts};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (s->c_pin) cudaFreeHost(s->c_pin);
    s->c_pin = nullptr;
    s->dac = DevAc();
    s->dwm = DevWm();
    s->dacv = DevAcv();
    s->dac2 = DevAc2();
    s->c_text = s->c_ws = s->c_out = s->c_counts = nullptr;
    s->c_text_cap = s->c_ws_cap = s->c_out_cap = 0;
}

int upload_ac(pm_set *s)
{
    const AcTables &t = s->ac;
    DevAc &d = s->dac;
    int64_t &tot = s->device_bytes;
    const int eb = t.dna ? t.entry_bytes : 4;
    int rc;
    // the device copy of an ACGT table may hold (next_row << 2) | match, the
    // table index of the next row's first entry (see DevAc::pre)
    auto dev_entry = [&](uint32_t e) { return d.pre ? (((e >> 1) << 2) | (e & 1u)) : e; };
    if (eb == 2) {
        std::vector<uint16_t> t16(t.table.size());
        for (size_t i = 0; i < t.table.size(); ++i) t16[i] = uint16_t(dev_entry(t.table[i]));
        rc = upload(&d.table, t16.data(), t16.size() * 2, tot);
    } else if (d.pre) {
        std::vector<uint32_t> t32(t.table.size());
        for (size_t i = 0; i < t.table.size(); ++i) t32[i] = dev_entry(t.table[i]);
        rc = upload(&d.table, t32.data(), t32.size() * 4, tot);
    } else {
        rc = upload(&d.table, t.table.data(), t.table.size() * 4, tot);
    }
    if (!rc)
        rc = upload(reinterpret_cast<void **>(&d.flag_mask), t.flag_mask.data(), t.flag_mask.size() * 4, tot);
    if (!rc) {
        if (eb == 2) {
            std::vector<uint16_t> r16v(t.flag_rank.begin(), t.flag_rank.end());
            std::vector<uint16_t> c16v(t.canon.size());
            for (size_t i = 0; i < t.canon.size(); ++i)
                c16v[i] = uint16_t((t.canon[i] & 0x80000000u) ? (0x8000u | (t.canon[i] & 0x7FFFu)) : t.canon[i]);
            rc = upload(&d.flag_rank, r16v.data(), r16v.size() * 2, tot);
            if (!rc) rc = upload(&d.canon, c16v.data(), c16v.size() * 2, tot);
        } else {
            rc = upload(&d.flag_rank, t.flag_rank.data(), t.flag_rank.size() * 4, tot);
            if (!rc) rc = upload(&d.canon, t.canon.data(), t.canon.size() * 4, tot);
        }
    }
    if (!rc) {
        // late ids: min(multiplicity - 1, 3) of each terminal, 2 bits (counts
        // mode), and the same per match entry (list mode)
        auto mult2 = [&](size_t c) -> uint32_t {
            if (!(t.canon[c] & 0x80000000u)) return 0u;
            const uint32_t g = t.canon[c] & 0x7FFFFFFFu;
            return std::min<uint32_t>(t.grp_off[g + 1] - t.grp_off[g] - 1u, 3u);
        };
        std::vector<uint32_t> bits((t.canon.size() + 15) / 16 + 1, 0u);
        for (size_t c = 0; c < t.canon.size(); ++c) bits[c >> 4] |= mult2(c) << ((c & 15) * 2);
        rc = upload(reinterpret_cast<void **>(&d.tmul), bits.data(), bits.size() * 4, tot);
        const size_t nw = t.flag_mask.size();
        std::vector<uint32_t> ebits(2 * nw + 1, 0u);
        for (size_t k = 0; k < nw * 32; ++k) {
            const uint32_t mw = t.flag_mask[k >> 5], b = uint32_t(k & 31);
            if (!((mw >> b) & 1u)) continue;
            const size_t c = t.flag_rank[k >> 5] + uint32_t(__builtin_popcount(mw & ((1u << b) - 1u)));
            ebits[k >> 4] |= mult2(c) << ((k & 15) * 2);
        }
        if (!rc) rc = upload(reinterpret_cast<void **>(&d.emul), ebits.data(), ebits.size() * 4, tot);
    }
    if (!rc)
        rc = upload(reinterpret_cast<void **>(&d.grp_off), t.grp_off.data(), t.grp_off.size() * 4, tot);
    if (!rc)
        rc = upload(reinterpret_cast<void **>(&d.grp_ids), t.grp_ids.data(), t.grp_ids.size() * 4, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.cls), t.cls, 256, tot);
    return rc;
}

int upload_acv(pm_set *s)
{
    const AcvTables &v = s->acv;
    const AcTables &t = v.ac;
    DevAcv &d = s->dacv;
    int64_t &tot = s->device_bytes;
    int rc;
    // index entries (next_row << 2) | flag for ACGT sets (see DevAc::pre)
    auto dev_entry = [&](uint32_t e) { return d.pre ? (((e >> 1) << 2) | (e & 1u)) : e; };
    if (d.entry_bytes == 2) {
        std::vector<uint16_t> t16(t.table.size());
        for (size_t i = 0; i < t.table.size(); ++i) t16[i] = uint16_t(dev_entry(t.table[i]));
        rc = upload(&d.table, t16.data(), t16.size() * 2, tot);
    } else {
        std::vector<uint32_t> t32(t.table.size());
        for (size_t i = 0; i < t.table.size(); ++i) t32[i] = dev_entry(t.table[i]);
        rc = upload(&d.table, t32.data(), t32.size() * 4, tot);
    }
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.cls), t.cls, 256, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.omask), v.omask.data(), v.omask.size() * 4, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.orank), v.orank.data(), v.orank.size() * 4, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.out_off), v.out_off.data(), v.out_off.size() * 4, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.out_ent), v.out_ent.data(), v.out_ent.size() * 4, tot);
    return rc;
}

int upload_wm(pm_set *s)
{
    const WmTables &t = s->wm;
    DevWm &d = s->dwm;
    int64_t &tot = s->device_bytes;
    int rc = upload(reinterpret_cast<void **>(&d.shift), t.shift.data(), t.shift.size(), tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.hoff), t.hoff.data(), t.hoff.size() * 4, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.hids), t.hids.data(), t.hids.size() * 4, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.hpfx), t.hpfx.data(), t.hpfx.size() * 2, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.pats), t.pats.data(), t.pats.size(), tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.hcode), t.hcode.data(), t.hcode.size() * 4, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.grp_off), t.grp_off.data(), t.grp_off.size() * 4, tot);
    if (!rc) rc = upload(reinterpret_cast<void **>(&d.grp_ids), t.grp_ids.data(), t.grp_ids.size() * 4, tot);
    if (!rc && t.var) rc = upload(reinterpret_cast<void **>(&d.poff), t.poff.data(), t.poff.size() * 8, tot);
    if (!rc && t.var && t.dna) {
        rc = upload(reinterpret_cast<void **>(&d.fcode), t.fcode.data(), t.fcode.size() * 8, tot);
        if (!rc) rc = upload(reinterpret_cast<void **>(&d.flen), t.flen.data(), t.flen.size(), tot);
    }
    if (!rc && t.dna) {
        rc = upload(reinterpret_cast<void **>(&d.shift2), t.shift2.data(), t.shift2.size(), tot);
        if (!rc) rc = upload(reinterpret_cast<void **>(&d.dir), t.dir.data(), t.dir.size() * 4, tot);
        if (!rc) rc = upload(reinterpret_cast<void **>(&d.ccode), t.ccode.data(), t.ccode.size() * 8, tot);
        if (!rc) rc = upload(reinterpret_cast<void **>(&d.cr), t.cr.data(), t.cr.size() * 4, tot);
    }
    return rc;
}

int finish_compile(pm_set *s, pm_set **out)
{
    if (s->host_only) {
        *out = s;
        return PM_OK;
    }
    DeviceProps dp;
    int rc = device_props(dp);
    const bool ac_like = s->algo == PM_ALGO_AC || s->algo == PM_ALGO_PFAC;
    if (!rc) {
        if (s->algo == PM_ALGO_ACV) rc = acv_plan(s->acv, s->params, dp, s->dacv);
        else rc = ac_like ? ac_plan(s->ac, s->params, dp, s->dac) : wm_plan(s->wm, s->params, dp, s->dwm);
    }
    if (!rc && s->algo == PM_ALGO_PFAC) s->dac.pre = 0;  // PFAC walks the plain entry format
    if (!rc) rc = s->algo == PM_ALGO_ACV ? upload_acv(s) : ac_like ? upload_ac(s) : upload_wm(s);
    if (!rc && s->algo == PM_ALGO_AC && !s->ac.table2.empty()) {
        // two characters per lookup: uploaded whenever the set is eligible
        // (the tuner may pick it); used when pm_params.stride is 2
        rc = upload(&s->dac2.table2, s->ac.table2.data(), s->ac.table2.size() * 2, s->device_bytes);
        if (!rc && s->params.stride == 2) {
            rc = ac2_plan(s->ac, s->params, dp, s->dac2);
            s->dac2.use = rc == PM_OK;
        }
    }
    if (rc) {
        release_device(s);
        delete s;
        return rc;
    }
    *out = s;
    return PM_OK;
}

// grow a cached device buffer to at least `bytes`
int ensure(void *&p, int64_t &cap, int64_t bytes)
{
    if (p && cap >= bytes) return PM_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    int64_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&p, size_t(want));
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        cudaGetLastError();
        p = nullptr;
        return e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA;
    }
    cap = want;
    return PM_OK;
}

// A result and how its arrays were allocated; the public struct comes first
// so a pm_result* is also a ResultBox*.
struct ResultBox {
    pm_result pub;
    int pinned;
    ResultRelease release;  // arrays owned by an allocator of the caller's
    void *ctx;
};

void free_array(void *p, int pinned)
{
    if (!p) return;
    if (pinned) cudaFreeHost(p);
    else std::free(p);
}

// pinned = page-locked host arrays (device-to-host copies at full link speed)
pm_result *new_result(int64_t d, int64_t n_occ, bool list, bool pinned)
{
    ResultBox *b = static_cast<ResultBox *>(std::calloc(1, sizeof(ResultBox)));
    if (!b) return nullptr;
    pm_result *r = &b->pub;
    b->pinned = pinned ? 1 : 0;
    r->d = d;
    r->n_occ = n_occ;
    const size_t cb = size_t(d > 0 ? d : 1) * sizeof(int64_t);
    const size_t ob = size_t(n_occ > 0 ? n_occ : 1) * 8;
    if (pinned) {
        void *c = nullptr, *o = nullptr;
        if (cudaMallocHost(&c, cb) == cudaSuccess) r->counts = static_cast<int64_t *>(c);
        if (list && cudaMallocHost(&o, ob) == cudaSuccess) r->occ = static_cast<uint64_t *>(o);
        cudaGetLastError();
    } else {
        r->counts = static_cast<int64_t *>(std::calloc(cb / 8, 8));
        if (list) r->occ = static_cast<uint64_t *>(std::malloc(ob));
    }
    if (!r->counts || (list && !r->occ)) {
        free_array(r->counts, b->pinned);
        free_array(r->occ, b->pinned);
        std::free(b);
        return nullptr;
    }
    return r;
}

int64_t set_d(const pm_set *s)
{
    if (s->algo == PM_ALGO_WM || s->algo == PM_ALGO_WMV) return s->wm.d;
    return s->algo == PM_ALGO_ACV ? s->acv.ac.d : s->ac.d;
}

}  // namespace

pm_result *make_result(int64_t d, int64_t n_occ, bool list) { return new_result(d, n_occ, list, false); }

pm_result *make_result_owned(int64_t d, int64_t n_occ, int64_t *counts, uint64_t *occ,
                             ResultRelease release, void *ctx)
{
    ResultBox *b = static_cast<ResultBox *>(std::calloc(1, sizeof(ResultBox)));
    if (!b) return nullptr;
    b->pub.d = d;
    b->pub.n_occ = n_occ;
    b->pub.counts = counts;
    b->pub.occ = occ;
    b->release = release;
    b->ctx = ctx;
    return &b->pub;
}
}  // namespace pm

using namespace pm;

extern "C" {

const char *pm_version(void) { return "pmscan 1.0 (sm_103a)"; }

const char *pm_strerror(int code)
{
    switch (code) {
    case PM_OK: return "ok";
    case PM_EINVAL: return "invalid argument";
    case PM_ENOMEM: return "out of memory";
    case PM_ECUDA: return "CUDA runtime error";
    case PM_ETOOBIG: return "input or table too large";
    case PM_ETIMEOUT: return "a bounded device wait gave up";
    case PM_ECAPACITY: return "occurrence buffer too small";
    case PM_ENODEV: return "no usable CUDA device";
    default: return "unknown error";
    }
}

int pm_last_cuda_error(void) { return g_last_cuda; }

static bool params_ok(const pm_params *p)
{
    if (!p) return true;
    return p->placement >= 0 && p->placement <= PM_PLACE_GLOBAL && p->smem_table_bytes >= 0 &&
           p->warps_per_cta >= 0 && p->warps_per_cta <= 32 && p->ctas_per_sm >= 0 &&
           p->ctas_per_sm <= 8 && p->wm_prefix_len >= 0 && p->wm_prefix_len <= 3 &&
           p->counters >= 0 && p->counters <= 3 && p->ids_place >= 0 && p->ids_place <= 3 &&
           p->stride >= 0 && p->stride <= 2;
}

int pm_ac_compile(const uint8_t *P, int64_t d, int32_t m, const pm_params *opt, pm_set **out)
{
    if (!out || !P || d < 1 || m < 1 || !params_ok(opt)) return PM_EINVAL;
    pm_set *s = new (std::nothrow) pm_set();
    if (!s) return PM_ENOMEM;
    s->algo = PM_ALGO_AC;
    if (opt) s->params = *opt;
    s->host_only = s->params.host_only != 0;
    int rc = build_ac(P, d, m, s->ac);
    if (!rc) {
        build_ac2(s->ac);  // the two-character table of an eligible set
        if (s->params.stride == 2 && s->ac.table2.empty()) rc = PM_ETOOBIG;
    }
    if (rc) {
        delete s;
        return rc;
    }
    return finish_compile(s, out);
}

int pm_pfac_compile(const uint8_t *P, int64_t d, int32_t m, const pm_params *opt, pm_set **out)
{
    if (!out || !P || d < 1 || m < 1 || !params_ok(opt)) return PM_EINVAL;
    pm_set *s = new (std::nothrow) pm_set();
    if (!s) return PM_ENOMEM;
    s->algo = PM_ALGO_PFAC;
    if (opt) s->params = *opt;
    s->host_only = s->params.host_only != 0;
    int rc = build_pfac(P, d, m, s->ac);
    if (rc) {
        delete s;
        return rc;
    }
    return finish_compile(s, out);
}

int pm_acv_compile(const uint8_t *P, const int64_t *offsets, int64_t d, const pm_params *opt, pm_set **out)
{
    if (!out || !P || !offsets || d < 1 || !params_ok(opt)) return PM_EINVAL;
    pm_set *s = new (std::nothrow) pm_set();
    if (!s) return PM_ENOMEM;
    s->algo = PM_ALGO_ACV;
    if (opt) s->params = *opt;
    s->host_only = s->params.host_only != 0;
    int rc = build_acv(P, offsets, d, s->acv);
    if (rc) {
        delete s;
        return rc;
    }
    return finish_compile(s, out);
}

int pm_wmv_compile(const uint8_t *P, const int64_t *offsets, int64_t d, int32_t B, const pm_params *opt,
                   pm_set **out)
{
    if (!out || !P || !offsets || d < 1 || B < 1 || !params_ok(opt)) return PM_EINVAL;
    pm_set *s = new (std::nothrow) pm_set();
    if (!s) return PM_ENOMEM;
    s->algo = PM_ALGO_WMV;
    if (opt) s->params = *opt;
    s->host_only = s->params.host_only != 0;
    const int bp = s->params.wm_prefix_len > 0 ? s->params.wm_prefix_len : 2;
    int rc = build_wmv(P, offsets, d, B, bp, s->wm);
    if (rc) {
        delete s;
        return rc;
    }
    return finish_compile(s, out);
}

int pm_wm_compile(const uint8_t *P, int64_t d, int32_t m, int32_t B, const pm_params *opt,
                  pm_set **out)
{
    if (!out || !P || d < 1 || m < 1 || B < 1 || B > m || !params_ok(opt)) return PM_EINVAL;
    pm_set *s = new (std::nothrow) pm_set();
    if (!s) return PM_ENOMEM;
    s->algo = PM_ALGO_WM;
    if (opt) s->params = *opt;
    s->host_only = s->params.host_only != 0;
    int bp = s->params.wm_prefix_len > 0 ? s->params.wm_prefix_len : 2;
    if (bp > m) bp = m;
    int rc = build_wm(P, d, m, B, bp, s->wm);
    if (rc) {
        delete s;
        return rc;
    }
    return finish_compile(s, out);
}

void pm_set_free(pm_set *s)
{
    if (!s) return;
    release_device(s);
    delete s;
}

int pm_plan_for_device(const pm_set *s, int32_t sm_count, int32_t smem_optin, int32_t smem_per_sm,
                       pm_plan_info *out)
{
    if (!s || !out || sm_count <= 0 || smem_optin <= 0 || smem_per_sm <= 0) return PM_EINVAL;
    if (s->algo != PM_ALGO_AC && s->algo != PM_ALGO_PFAC) return PM_EINVAL;
    DeviceProps dp;
    dp.sm_count = sm_count;
    dp.smem_optin = smem_optin;
    dp.smem_per_sm = smem_per_sm;
    DevAc d;
    const int rc = ac_plan(s->ac, s->params, dp, d);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    out->placement = d.placement;
    out->warps = d.warps;
    out->warps_list = d.warps_list;
    out->ids_place = d.ids_smem == 1 ? 1 : d.ids_smem == 2 ? 3 : 2;
    out->counters = d.hist_smem == 1 ? 1 : d.hist_smem == 2 ? 2 : 3;
    out->ctas_per_sm = d.ctas_per_sm;
    out->smem_rows = d.smem_entries >> s->ac.lw;
    out->smem_bytes = d.smem_bytes;
    out->smem_bytes_list = d.smem_bytes_list;
    return PM_OK;
}

int pm_set_get_info(const pm_set *s, pm_set_info *info)
{
    if (!s || !info) return PM_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->algo = s->algo;
    info->device_bytes = s->device_bytes;
    if (s->algo == PM_ALGO_ACV) {
        const AcTables &t = s->acv.ac;
        info->m = t.m;
        info->m_min = s->acv.m_min;
        info->max_starts = s->acv.K;
        info->d = t.d;
        info->n_distinct = t.n_distinct;
        info->n_states = t.n_states;
        info->n_rows = t.n_rows;
        info->n_classes = t.n_classes;
        info->row_width = 1 << t.lw;
        info->entry_bytes = s->host_only ? (t.dna && t.n_rows <= (1 << 14) ? 2 : 4) : s->dacv.entry_bytes;
        info->dna_mode = t.dna ? 1 : 0;
        info->placement = s->dacv.placement;
        info->smem_rows = s->dacv.smem_entries >> t.lw;
        info->table_bytes = (t.n_rows << t.lw) * info->entry_bytes;
        return PM_OK;
    }
    info->max_starts = 1;
    info->stride = (s->algo == PM_ALGO_AC && s->dac2.use) ? 2 : 1;
    if (s->algo == PM_ALGO_AC || s->algo == PM_ALGO_PFAC) {
        const AcTables &t = s->ac;
        info->m = t.m;
        info->m_min = t.m;
        info->d = t.d;
        info->n_distinct = t.n_distinct;
        info->n_states = t.n_states;
        info->n_rows = t.n_rows;
        info->n_classes = t.n_classes;
        info->row_width = 1 << t.lw;
        info->entry_bytes = t.dna ? t.entry_bytes : 4;
        info->dna_mode = t.dna ? 1 : 0;
        info->placement = s->dac.placement;
        info->smem_rows = s->dac.smem_entries >> t.lw;
        info->table_bytes = (t.n_rows << t.lw) * info->entry_bytes;
    } else {
        const WmTables &t = s->wm;
        info->m = t.m;
        info->d = t.d;
        info->B = t.B;
        info->Bp = t.Bp;
        info->shift_entries = int64_t(t.shift.size());
        info->n_zero_shift = t.n_zero_shift;
        info->n_distinct = t.n_distinct;
        info->m_min = t.m;
        if (t.var) {
            info->m = t.m_max;
            info->max_starts = t.K;
        }
        info->dna_mode = t.dna ? 1 : 0;  // exact 2-bit-code tables in use
    }
    return PM_OK;
}

static int64_t set_ws_bytes(const pm_set *s, int64_t n, bool list)
{
    if (s->algo == PM_ALGO_ACV) return acv_workspace_bytes(s->acv, n, list);
    if (s->algo == PM_ALGO_AC || s->algo == PM_ALGO_PFAC) return ac_workspace_bytes(s->ac, n, list);
    return wm_workspace_bytes(s->wm, n, list);
}

int64_t pm_scan_workspace_bytes(const pm_set *s, int64_t n, uint32_t flags)
{
    if (!s || n < 0) return -1;
    return set_ws_bytes(s, n, !(flags & PM_COUNTS_ONLY));
}

int pm_scan_device(const pm_set *s, const uint8_t *d_text, int64_t n, uint32_t flags,
                   int64_t *d_counts, uint64_t *d_occ, int64_t occ_capacity, int64_t *d_n_occ,
                   void *d_workspace, int64_t workspace_bytes, void *stream)
{
    if (!s || n < 0 || !d_counts || !d_n_occ || !d_workspace) return PM_EINVAL;
    if (s->host_only) return PM_EINVAL;
    if (n > 0 && !d_text) return PM_EINVAL;
    if (n >= (int64_t(1) << 32)) return PM_ETOOBIG;
    const bool list = !(flags & PM_COUNTS_ONLY);
    if (list && occ_capacity > 0 && !d_occ) return PM_EINVAL;
    if (occ_capacity < 0) return PM_EINVAL;
    if (workspace_bytes < set_ws_bytes(s, n, list)) return PM_EINVAL;
    if (s->algo == PM_ALGO_AC && s->dac2.use)
        return ac2_launch(s->ac, s->dac, s->dac2, d_text, n, list, d_counts, d_occ, occ_capacity, d_n_occ,
                          d_workspace, stream);
    if (s->algo == PM_ALGO_AC)
        return ac_launch(s->ac, s->dac, d_text, n, list, d_counts, d_occ, occ_capacity, d_n_occ,
                         d_workspace, stream);
    if (s->algo == PM_ALGO_PFAC)
        return pfac_launch(s->ac, s->dac, d_text, n, list, d_counts, d_occ, occ_capacity, d_n_occ,
                           d_workspace, stream);
    if (s->algo == PM_ALGO_ACV)
        return acv_launch(s->acv, s->dacv, d_text, n, list, d_counts, d_occ, occ_capacity, d_n_occ,
                          d_workspace, stream);
    return wm_launch(s->wm, s->dwm, d_text, n, list, d_counts, d_occ, occ_capacity, d_n_occ,
                     d_workspace, stream);
}

int pm_scan_device_noalloc(const pm_set *s, const uint8_t *d_text, int64_t n, uint32_t flags,
                           int64_t *d_counts, uint64_t *d_occ, int64_t occ_capacity,
                           int64_t *d_n_occ, void *stream)
{
    if (!s || n < 0 || !d_counts || !d_n_occ) return PM_EINVAL;
    if (s->host_only || s->algo != PM_ALGO_AC) return PM_EINVAL;
    if (n > 0 && !d_text) return PM_EINVAL;
    if (n >= (int64_t(1) << 32)) return PM_ETOOBIG;
    const bool list = !(flags & PM_COUNTS_ONLY);
    if (occ_capacity < 0 || (list && occ_capacity > 0 && !d_occ)) return PM_EINVAL;
    return ac_launch_noalloc(s->ac, s->dac, d_text, n, list, d_counts, d_occ, occ_capacity,
                             d_n_occ, stream);
}

int64_t pm_noalloc_scratch_bytes(void) { return ac_noalloc_limit_bytes(); }

int pm_noalloc_scan_status(void *stream) { return ac_noalloc_status(stream); }

// Wu-Manber sets: warps per CTA (more than 16 only for exact-code tables, in
// the 768-thread kernels), timed on the caller's text like the AC tuner.
static int tune_wm(pm_set *s, const uint8_t *d_text, int64_t n, bool list, int32_t reps, cudaStream_t st,
                   pm_params *best_out, float *best_ms)
{
    DeviceProps dp;
    int rc = device_props(dp);
    if (rc) return rc;
    const WmTables &t = s->wm;
    void *ws = nullptr, *counts = nullptr, *nocc = nullptr, *occ = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int64_t n_occ = 0;
    auto cleanup = [&]() {
        for (void *p : {ws, counts, nocc, occ})
            if (p) cudaFree(p);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&ws, size_t(wm_workspace_bytes(t, n, list)));
    if (e == cudaSuccess) e = cudaMalloc(&counts, size_t(t.d) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&nocc, 8);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && list) {
        rc = wm_launch(t, s->dwm, d_text, n, false, static_cast<int64_t *>(counts), nullptr, 0,
                       static_cast<int64_t *>(nocc), ws, st);
        if (!rc) e = cudaMemcpyAsync(&n_occ, nocc, 8, cudaMemcpyDeviceToHost, st);
        if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (!rc && e == cudaSuccess) e = cudaMalloc(&occ, size_t(std::max<int64_t>(n_occ, 1)) * 8);
    }
    if (e != cudaSuccess || rc) {
        if (e != cudaSuccess) set_cuda_error(int(e));
        cudaGetLastError();
        cleanup();
        return rc ? rc : (e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA);
    }
    const DevWm saved = s->dwm;
    DevWm best = saved;
    pm_params best_p = s->params;
    float best_t = -1.0f;
    std::vector<std::pair<int, int>> tried;   // (warps, hist_smem)
    for (int w : {0, 24, 20, 16, 12, 8}) {
        pm_params p = s->params;
        p.warps_per_cta = w;
        DevWm plan = saved;
        if (wm_plan(t, p, dp, plan) != PM_OK) continue;
        bool dup = false;
        for (const auto &x : tried) dup = dup || (x.first == plan.warps && x.second == plan.hist_smem);
        if (dup) continue;
        tried.push_back({plan.warps, plan.hist_smem});
        auto run = [&]() {
            return wm_launch(t, plan, d_text, n, list, static_cast<int64_t *>(counts), static_cast<uint64_t *>(occ),
                             n_occ, static_cast<int64_t *>(nocc), ws, st);
        };
        rc = run();
        if (!rc) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && !rc && e == cudaSuccess; ++r) rc = run();
        if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { set_cuda_error(int(e)); rc = PM_ECUDA; }
        if (!rc && pm_scan_status(ws, st) != PM_OK) rc = PM_ETIMEOUT;
        if (rc) break;
        ms /= float(reps);
        if (best_t < 0.0f || ms < best_t) { best_t = ms; best = plan; best_p = p; }
    }
    cleanup();
    if (rc) return rc;
    if (best_t < 0.0f) return PM_ETOOBIG;
    s->dwm = best;
    s->params = best_p;
    if (best_out) *best_out = best_p;
    if (best_ms) *best_ms = best_t;
    return PM_OK;
}

int pm_tune(pm_set *s, const uint8_t *d_text, int64_t n, uint32_t flags, int32_t reps,
            void *stream, pm_params *best_out, float *best_ms)
{
    if (!s || s->host_only || !d_text || n <= 0) return PM_EINVAL;
    if (s->algo == PM_ALGO_WM) {
        if (n >= (int64_t(1) << 32)) return PM_ETOOBIG;
        return tune_wm(s, d_text, n, !(flags & PM_COUNTS_ONLY), reps < 1 ? 1 : reps,
                       static_cast<cudaStream_t>(stream), best_out, best_ms);
    }
    if (s->algo != PM_ALGO_AC) return PM_EINVAL;
    if (n >= (int64_t(1) << 32)) return PM_ETOOBIG;
    if (reps < 1) reps = 1;
    const bool list = !(flags & PM_COUNTS_ONLY);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DeviceProps dp;
    int rc = device_props(dp);
    if (rc) return rc;
    const AcTables &t = s->ac;
    void *ws = nullptr, *counts = nullptr, *nocc = nullptr, *occ = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int64_t n_occ = 0;
    auto cleanup = [&]() {
        if (ws) cudaFree(ws);
        if (counts) cudaFree(counts);
        if (nocc) cudaFree(nocc);
        if (occ) cudaFree(occ);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&ws, size_t(ac_workspace_bytes(t, n, list)));
    if (e == cudaSuccess) e = cudaMalloc(&counts, size_t(t.d) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&nocc, 8);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && list) {
        // size the occurrence buffer with one counts-only scan
        rc = ac_launch(t, s->dac, d_text, n, false, static_cast<int64_t *>(counts), nullptr, 0,
                       static_cast<int64_t *>(nocc), ws, st);
        if (!rc) e = cudaMemcpyAsync(&n_occ, nocc, 8, cudaMemcpyDeviceToHost, st);
        if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (!rc && e == cudaSuccess) e = cudaMalloc(&occ, size_t(std::max<int64_t>(n_occ, 1)) * 8);
    }
    if (e != cudaSuccess || rc) {
        if (e != cudaSuccess) set_cuda_error(int(e));
        cudaGetLastError();
        cleanup();
        return rc ? rc : (e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA);
    }
    // candidate plans: the current one, then placement x warps x counters x ids
    std::vector<pm_params> cand;
    cand.push_back(s->params);
    cand.back().stride = 1;
    for (int place : {PM_PLACE_AUTO, PM_PLACE_HYBRID})
        for (int w : {0, 24, 20, 16, 12, 8})
            for (int c : {0, 1, 2, 3})
                for (int idp : {0, 1, 2, 3}) {
                    pm_params p = s->params;
                    p.stride = 1;
                    p.placement = place;
                    p.warps_per_cta = w;
                    p.counters = c;
                    p.ids_place = idp;
                    p.smem_table_bytes = 0;
                    cand.push_back(p);
                }
    struct Tried { DevAc plan; pm_params params; float ms; };
    std::vector<Tried> tried;
    const DevAc saved = s->dac;
    for (const pm_params &p : cand) {
        DevAc plan = saved;
        if (ac_plan(t, p, dp, plan) != PM_OK) continue;
        bool dup = false;
        // a late-ids plan's list mode does not count in the scan kernel, so
        // plans differing only in counters are one candidate there; the
        // first one tried (automatic counters: the best that fit for counts
        // mode) is kept
        const bool late_list = list && plan.ids_smem == 2;
        for (const Tried &x : tried) {
            if (late_list && x.plan.ids_smem == 2) {  // only the list-mode launch matters
                dup = dup || (x.plan.warps_list == plan.warps_list && x.plan.variant_list == plan.variant_list &&
                              x.plan.smem_entries == plan.smem_entries);
                continue;
            }
            dup = dup || (x.plan.warps == plan.warps && x.plan.warps_list == plan.warps_list &&
                          x.plan.variant_list == plan.variant_list &&
                          x.plan.hist_smem == plan.hist_smem &&
                          x.plan.ids_smem == plan.ids_smem && x.plan.smem_entries == plan.smem_entries &&
                          x.plan.variant == plan.variant && x.plan.ctas_per_sm == plan.ctas_per_sm);
        }
        if (dup) continue;
        auto run = [&]() {
            return ac_launch(t, plan, d_text, n, list, static_cast<int64_t *>(counts),
                             static_cast<uint64_t *>(occ), n_occ, static_cast<int64_t *>(nocc), ws, st);
        };
        rc = run();  // warm-up
        if (!rc) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && !rc && e == cudaSuccess; ++r) rc = run();
        if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { set_cuda_error(int(e)); rc = PM_ECUDA; }
        if (!rc && pm_scan_status(ws, stream) != PM_OK) rc = PM_ETIMEOUT;
        if (rc) break;
        tried.push_back(Tried{plan, p, ms / float(reps)});
    }
    // two characters per lookup, when the set is eligible
    float ms2 = -1.0f;
    DevAc2 plan2 = s->dac2;
    pm_params p2 = s->params;
    p2.stride = 2;
    p2.warps_per_cta = 0;
    if (!rc && plan2.table2 && ac2_plan(t, p2, dp, plan2) == PM_OK) {
        auto run2 = [&]() {
            return ac2_launch(t, saved, plan2, d_text, n, list, static_cast<int64_t *>(counts),
                              static_cast<uint64_t *>(occ), n_occ, static_cast<int64_t *>(nocc), ws, st);
        };
        rc = run2();
        if (!rc) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && !rc && e == cudaSuccess; ++r) rc = run2();
        if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { set_cuda_error(int(e)); rc = PM_ECUDA; }
        if (!rc && pm_scan_status(ws, stream) != PM_OK) rc = PM_ETIMEOUT;
        if (!rc) ms2 = ms / float(reps);
    }
    cleanup();
    if (rc) return rc;
    if (tried.empty() && ms2 < 0.0f) return PM_ETOOBIG;
    size_t bi = 0;
    for (size_t i = 1; i < tried.size(); ++i)
        if (tried[i].ms < tried[bi].ms) bi = i;
    if (ms2 >= 0.0f && (tried.empty() || ms2 < tried[bi].ms)) {
        s->dac = saved;
        plan2.use = true;
        s->dac2 = plan2;
        s->params = p2;
        if (best_out) *best_out = p2;
        if (best_ms) *best_ms = ms2;
        return PM_OK;
    }
    s->dac = tried[bi].plan;  // same device tables, new launch plan
    s->dac2.use = false;
    s->params = tried[bi].params;
    s->params.stride = 1;
    if (best_out) *best_out = s->params;
    if (best_ms) *best_ms = tried[bi].ms;
    return PM_OK;
}

int pm_scan_status(const void *d_workspace, void *stream)
{
    if (!d_workspace) return PM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, d_workspace, sizeof(status), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        return PM_ECUDA;
    }
    return status ? PM_ETIMEOUT : PM_OK;
}

}  // extern "C"

namespace pm {
namespace {
// pm_scan_batch's batched part: the host texts of instances `js` copied into
// one device buffer (16-byte aligned starts), a counts pass that gives every
// instance's total, then the list pass into exact capacities, and each
// instance's counts and keys back into its own library-owned result.
int scan_batch_host(const pm_set *const *sets, const uint8_t *const *texts, const int64_t *ns,
                    const std::vector<int32_t> &js, uint32_t flags, void *stream, pm_result **outs)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool list = !(flags & PM_COUNTS_ONLY);
    const int32_t kb = int32_t(js.size());
    std::vector<const pm_set *> bs(size_t(kb), nullptr);
    std::vector<int64_t> off(size_t(kb), 0), len(size_t(kb), 0), occ_off(size_t(kb) + 1, 0);
    int64_t total = 0;
    for (int32_t i = 0; i < kb; ++i) {
        bs[size_t(i)] = sets[js[size_t(i)]];
        off[size_t(i)] = total;
        len[size_t(i)] = ns[js[size_t(i)]];
        total += (len[size_t(i)] + 15) & ~int64_t(15);
    }
    void *d_text = nullptr, *d_counts = nullptr, *d_nocc = nullptr, *d_ws = nullptr, *d_occ = nullptr;
    pm_batch *b = nullptr;
    auto cleanup = [&]() {
        pm_batch_free(b);
        for (void *p : {d_text, d_counts, d_nocc, d_ws, d_occ})
            if (p) cudaFree(p);
    };
    auto cuda_fail = [&](cudaError_t e) {
        set_cuda_error(int(e));
        cudaGetLastError();
        cleanup();
        return e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA;
    };
    int rc = pm_batch_prepare(bs.data(), kb, off.data(), len.data(), occ_off.data(), list ? 0u : PM_COUNTS_ONLY, &b);
    if (rc) { cleanup(); return rc; }
    const int64_t d_total = pm_batch_counts_total(b);
    int64_t ws_bytes = pm_batch_workspace_bytes(b);
    cudaError_t e = cudaMalloc(&d_text, size_t(std::max<int64_t>(total, 16)));
    if (e == cudaSuccess) e = cudaMalloc(&d_counts, size_t(std::max<int64_t>(d_total, 1)) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_nocc, size_t(kb) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_ws, size_t(ws_bytes));
    for (int32_t i = 0; i < kb && e == cudaSuccess; ++i)
        if (len[size_t(i)] > 0)
            e = cudaMemcpyAsync(static_cast<uint8_t *>(d_text) + off[size_t(i)], texts[js[size_t(i)]],
                                size_t(len[size_t(i)]), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
    // pass 1: every instance's total (list mode with no capacity writes no key)
    rc = pm_batch_scan_device(b, static_cast<const uint8_t *>(d_text), static_cast<int64_t *>(d_counts), nullptr,
                              static_cast<int64_t *>(d_nocc), d_ws, ws_bytes, stream);
    if (!rc) rc = pm_scan_status(d_ws, stream);
    if (rc) { cleanup(); return rc; }
    std::vector<int64_t> nocc(size_t(kb), 0);
    e = cudaMemcpyAsync(nocc.data(), d_nocc, size_t(kb) * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (list) {
        // pass 2: the keys, into exact capacities
        for (int32_t i = 0; i < kb; ++i) occ_off[size_t(i) + 1] = occ_off[size_t(i)] + nocc[size_t(i)];
        pm_batch_free(b);
        b = nullptr;
        rc = pm_batch_prepare(bs.data(), kb, off.data(), len.data(), occ_off.data(), 0u, &b);
        if (rc) { cleanup(); return rc; }
        if (pm_batch_workspace_bytes(b) > ws_bytes) {  // key staging of split instances
            cudaFree(d_ws);
            d_ws = nullptr;
            ws_bytes = pm_batch_workspace_bytes(b);
            e = cudaMalloc(&d_ws, size_t(ws_bytes));
            if (e != cudaSuccess) return cuda_fail(e);
        }
        e = cudaMalloc(&d_occ, size_t(std::max<int64_t>(occ_off[size_t(kb)], 1)) * 8);
        if (e != cudaSuccess) return cuda_fail(e);
        rc = pm_batch_scan_device(b, static_cast<const uint8_t *>(d_text), static_cast<int64_t *>(d_counts),
                                  static_cast<uint64_t *>(d_occ), static_cast<int64_t *>(d_nocc), d_ws, ws_bytes,
                                  stream);
        if (!rc) rc = pm_scan_status(d_ws, stream);
        if (rc) { cleanup(); return rc; }
    }
    int64_t coff = 0;
    for (int32_t i = 0; i < kb && e == cudaSuccess; ++i) {
        const int32_t j = js[size_t(i)];
        const int64_t d = bs[size_t(i)]->ac.d;
        pm_result *r = make_result(d, list ? nocc[size_t(i)] : 0, list);
        if (!r) { cleanup(); return PM_ENOMEM; }
        outs[j] = r;
        if (!list) r->n_occ = nocc[size_t(i)];
        e = cudaMemcpyAsync(r->counts, static_cast<int64_t *>(d_counts) + coff, size_t(d) * 8,
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && list && nocc[size_t(i)] > 0)
            e = cudaMemcpyAsync(r->occ, static_cast<uint64_t *>(d_occ) + occ_off[size_t(i)],
                                size_t(nocc[size_t(i)]) * 8, cudaMemcpyDeviceToHost, st);
        coff += d;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    cleanup();
    return PM_OK;
}
}  // namespace
}  // namespace pm

namespace pm {
namespace {
// Runs a scan of host or device text into the set's cached device buffers.
// On success d_counts/d_occ point at the device results and n_occ is known.
int scan_cached(pm_set *s, const uint8_t *T, int64_t n, uint32_t flags, void *stream,
                int64_t **d_counts_out, int64_t *n_occ_out)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool list = !(flags & PM_COUNTS_ONLY);
    const int64_t d = set_d(s);
    int rc;
    const uint8_t *d_text = T;
    if (!(flags & PM_DEVICE_TEXT) && n > 0) {
        rc = ensure(s->c_text, s->c_text_cap, n);
        if (rc) return rc;
        cudaError_t e = cudaMemcpyAsync(s->c_text, T, size_t(n), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        d_text = static_cast<const uint8_t *>(s->c_text);
    }
    const int64_t wsb = set_ws_bytes(s, n, list);
    rc = ensure(s->c_ws, s->c_ws_cap, wsb);
    if (rc) return rc;
    if (!s->c_counts) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, size_t(d + 2) * 8);
        if (e != cudaSuccess) { set_cuda_error(int(e)); cudaGetLastError(); return PM_ENOMEM; }
        s->c_counts = p;
    }
    int64_t *d_counts = static_cast<int64_t *>(s->c_counts);
    int64_t *d_nocc = d_counts + d;
    int64_t n_occ = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        int64_t cap = 0;
        if (list) {
            int64_t want = attempt == 0 ? (s->c_out_cap / 8 > 0 ? s->c_out_cap / 8 : (n / 16 + 1024)) : n_occ;
            if (want < 1) want = 1;
            rc = ensure(s->c_out, s->c_out_cap, want * 8);
            if (rc) return rc;
            cap = s->c_out_cap / 8;
        }
        rc = pm_scan_device(s, d_text, n, flags, d_counts, static_cast<uint64_t *>(s->c_out), cap,
                            d_nocc, s->c_ws, wsb, stream);
        if (rc) return rc;
        rc = pm_scan_status(s->c_ws, stream);
        if (rc) return rc;
        cudaError_t e = cudaMemcpy(&n_occ, d_nocc, 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
        if (!list || n_occ <= cap) break;
    }
    *d_counts_out = d_counts;
    *n_occ_out = n_occ;
    return PM_OK;
}
}  // namespace
}  // namespace pm

extern "C" {

int pm_scan(const pm_set *cs, const uint8_t *T, int64_t n, uint32_t flags, void *stream,
            pm_result **out)
{
    if (!cs || !out || n < 0 || (n > 0 && !T)) return PM_EINVAL;
    if (cs->host_only) return PM_EINVAL;
    if (n >= (int64_t(1) << 32)) return PM_ETOOBIG;
    pm_set *s = const_cast<pm_set *>(cs);  // device caches only
    const bool list = !(flags & PM_COUNTS_ONLY);
    const int64_t d = set_d(s);
    int64_t *d_counts = nullptr, n_occ = 0;
    int rc = scan_cached(s, T, n, flags, stream, &d_counts, &n_occ);
    if (rc) return rc;
    pm_result *r = new_result(d, n_occ, list, false);
    if (!r) return PM_ENOMEM;
    cudaError_t e = cudaMemcpy(r->counts, d_counts, size_t(d) * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && list && n_occ > 0)
        e = cudaMemcpy(r->occ, s->c_out, size_t(n_occ) * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_cuda_error(int(e));
        pm_result_free(r);
        return PM_ECUDA;
    }
    *out = r;
    return PM_OK;
}

}  // extern "C"

namespace pm {
namespace {
// pm_scan_to_host of a long host text with an Aho-Corasick or PFAC set, in
// pieces split with an m-1 halo (each piece owns the windows that start in
// it, as Section 4.3 splits the text over nodes): the copy of piece c+1 runs
// while piece c is scanned, and the keys of each piece leave for the host as
// soon as its running total is known. `done` false: take the plain path.
int scan_to_host_pieces(pm_set *s, const uint8_t *T, int64_t n, uint32_t flags, int64_t *counts_out,
                        uint64_t *occ_out, int64_t occ_capacity, int64_t *n_occ_out, void *stream,
                        bool &done)
{
    done = false;
    constexpr int64_t kMinPiece = int64_t(64) << 20;
    if ((s->algo != PM_ALGO_AC && s->algo != PM_ALGO_PFAC) || (flags & PM_DEVICE_TEXT) || n < 2 * kMinPiece)
        return PM_OK;
    const AcTables &t = s->ac;
    const bool list = !(flags & PM_COUNTS_ONLY);
    const int64_t d = t.d, m = t.m;
    int64_t K = std::min<int64_t>(16, n / kMinPiece);
    const int64_t piece = ((n + K - 1) / K + 15) & ~int64_t(15);  // 16-byte aligned starts
    K = (n + piece - 1) / piece;
    int rc = ensure(s->c_text, s->c_text_cap, n);
    if (!rc) rc = ensure(s->c_ws, s->c_ws_cap, ac_workspace_bytes(t, piece + m - 1, list));
    if (!rc && list) {
        int64_t want = std::max<int64_t>(s->c_out_cap / 8, n / 16 + 1024);
        rc = ensure(s->c_out, s->c_out_cap, want * 8);
    }
    if (rc) return rc;
    if (!s->c_counts) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, size_t(d + 2) * 8);
        if (e != cudaSuccess) { set_cuda_error(int(e)); cudaGetLastError(); return PM_ENOMEM; }
        s->c_counts = p;
    }
    if (!s->c_pin) {
        cudaError_t e = cudaMallocHost(&s->c_pin, 16 * 8);
        if (e != cudaSuccess) { set_cuda_error(int(e)); cudaGetLastError(); s->c_pin = nullptr; return PM_ENOMEM; }
    }
    int64_t *d_counts = static_cast<int64_t *>(s->c_counts);
    int64_t *d_nocc = d_counts + d;
    unsigned long long *run = reinterpret_cast<unsigned long long *>(d_counts + d + 1);
    int64_t *pin = static_cast<int64_t *>(s->c_pin);
    uint8_t *text = static_cast<uint8_t *>(s->c_text);
    uint64_t *occ = static_cast<uint64_t *>(s->c_out);
    const int64_t cap_dev = list ? s->c_out_cap / 8 : 0;
    cudaStream_t sc = static_cast<cudaStream_t>(stream), si = nullptr, so = nullptr;
    std::vector<cudaEvent_t> ev(size_t(2 * K), nullptr);
    auto cleanup = [&]() {
        if (si) cudaStreamDestroy(si);
        if (so) cudaStreamDestroy(so);
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&si, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&so, cudaStreamNonBlocking);
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(run, 0, 8, sc);
    // the first copy must not overtake work already queued on the caller's stream
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], sc);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(si, ev[0], 0);
    for (int64_t c = 0; c < K && e == cudaSuccess && !rc; ++c) {
        const int64_t off = c * piece, len = std::min(piece, n - off);
        const int64_t nc = std::min(len + m - 1, n - off);
        e = cudaMemcpyAsync(text + off, T + off, size_t(nc), cudaMemcpyHostToDevice, si);
        if (e == cudaSuccess) e = cudaEventRecord(ev[size_t(2 * c)], si);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sc, ev[size_t(2 * c)], 0);
        if (e != cudaSuccess) break;
        rc = ac_launch_piece(t, s->dac, s->algo == PM_ALGO_PFAC, text + off, nc, list, d_counts, occ, cap_dev,
                             d_nocc, s->c_ws, sc, c == 0, c == 0 ? nullptr : run, (unsigned long long)off);
        if (rc) break;
        if (list) e = cudaMemcpyAsync(run, d_nocc, 8, cudaMemcpyDeviceToDevice, sc);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pin + c, d_nocc, 8, cudaMemcpyDeviceToHost, sc);
        if (e == cudaSuccess) e = cudaEventRecord(ev[size_t(2 * c + 1)], sc);
    }
    int64_t prev = 0, total = 0;
    for (int64_t c = 0; c < K && e == cudaSuccess && !rc; ++c) {
        e = cudaEventSynchronize(ev[size_t(2 * c + 1)]);
        if (e != cudaSuccess) break;
        total = pin[c];
        if (!list) continue;
        const int64_t hi = std::min(total, std::min(occ_capacity, cap_dev));
        if (hi > prev) {
            e = cudaMemcpyAsync(occ_out + prev, occ + prev, size_t(hi - prev) * 8, cudaMemcpyDeviceToHost, so);
            prev = hi;
        }
    }
    if (e == cudaSuccess && !rc) e = cudaMemcpyAsync(counts_out, d_counts, size_t(d) * 8, cudaMemcpyDeviceToHost, sc);
    if (e == cudaSuccess && !rc) e = cudaStreamSynchronize(so);
    if (e == cudaSuccess && !rc) e = cudaStreamSynchronize(sc);
    cleanup();
    if (e != cudaSuccess) { set_cuda_error(int(e)); cudaGetLastError(); return PM_ECUDA; }
    if (rc) return rc;
    rc = pm_scan_status(s->c_ws, stream);
    if (rc) return rc;
    if (list && total > cap_dev) {
        // the device buffer was short: the plain path sizes it exactly
        s->c_out_cap = 0;
        int rc2 = ensure(s->c_out, s->c_out_cap, total * 8);
        return rc2;  // done stays false
    }
    *n_occ_out = total;
    done = true;
    return (list && total > occ_capacity) ? PM_ECAPACITY : PM_OK;
}
}  // namespace
}  // namespace pm

extern "C" {

int pm_scan_to_host(const pm_set *cs, const uint8_t *T, int64_t n, uint32_t flags,
                    int64_t *counts_out, uint64_t *occ_out, int64_t occ_capacity,
                    int64_t *n_occ_out, void *stream)
{
    if (!cs || !counts_out || !n_occ_out || n < 0 || (n > 0 && !T) || occ_capacity < 0)
        return PM_EINVAL;
    const bool list = !(flags & PM_COUNTS_ONLY);
    if (list && occ_capacity > 0 && !occ_out) return PM_EINVAL;
    if (cs->host_only) return PM_EINVAL;
    if (n >= (int64_t(1) << 32)) return PM_ETOOBIG;
    pm_set *s = const_cast<pm_set *>(cs);
    const int64_t d = set_d(s);
    bool done = false;
    int rc = scan_to_host_pieces(s, T, n, flags, counts_out, occ_out, occ_capacity, n_occ_out, stream, done);
    if (done || rc) return rc;
    int64_t *d_counts = nullptr, n_occ = 0;
    rc = scan_cached(s, T, n, flags, stream, &d_counts, &n_occ);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(counts_out, d_counts, size_t(d) * 8, cudaMemcpyDeviceToHost);
    const int64_t k = list ? (n_occ < occ_capacity ? n_occ : occ_capacity) : 0;
    if (e == cudaSuccess && k > 0) e = cudaMemcpy(occ_out, s->c_out, size_t(k) * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_cuda_error(int(e)); return PM_ECUDA; }
    *n_occ_out = n_occ;
    return (list && n_occ > occ_capacity) ? PM_ECAPACITY : PM_OK;
}

void pm_result_free(pm_result *r)
{
    if (!r) return;
    ResultBox *b = reinterpret_cast<ResultBox *>(r);
    if (b->release) {
        b->release(b->ctx, r->counts, r->occ);
    } else {
        free_array(r->counts, b->pinned);
        free_array(r->occ, b->pinned);
    }
    std::free(b);
}

int pm_scan_batch(const pm_set *const *sets, const uint8_t *const *texts, const int64_t *ns,
                  int32_t k, uint32_t flags, void *stream, pm_result **outs)
{
    if (!sets || !texts || !ns || !outs || k < 0) return PM_EINVAL;
    if (flags & ~(PM_HOST_TEXT | PM_DEVICE_TEXT | PM_COUNTS_ONLY)) return PM_EINVAL;
    for (int32_t j = 0; j < k; ++j) outs[j] = nullptr;
    for (int32_t j = 0; j < k; ++j)
        if (!sets[j] || ns[j] < 0 || (ns[j] > 0 && !texts[j])) return PM_EINVAL;
    // Host texts against Aho-Corasick sets the batched kernel takes go
    // through one persistent launch; the other instances (device texts,
    // Wu-Manber, PFAC, mixed lengths) through pm_scan, one after another.
    std::vector<int32_t> batched, single;
    for (int32_t j = 0; j < k; ++j) {
        const bool fits = !(flags & PM_DEVICE_TEXT) && batch_supports(sets[j]) && ns[j] < (int64_t(1) << 32);
        (fits ? batched : single).push_back(j);
    }
    if (batched.size() < 2) {
        single.insert(single.end(), batched.begin(), batched.end());
        batched.clear();
    }
    auto fail = [&](int rc) {
        for (int32_t q = 0; q < k; ++q) {
            pm_result_free(outs[q]);
            outs[q] = nullptr;
        }
        return rc;
    };
    if (!batched.empty()) {
        const int rc = scan_batch_host(sets, texts, ns, batched, flags, stream, outs);
        if (rc) return fail(rc);
    }
    for (const int32_t j : single) {
        const int rc = pm_scan(sets[j], texts[j], ns[j], flags, stream, &outs[j]);
        if (rc) return fail(rc);
    }
    return PM_OK;
}

int pm_selfcheck_host_walk(const pm_set *s, const uint8_t *T, int64_t n, pm_result **out)
{
    if (!s || !out || n < 0 || (n > 0 && !T)) return PM_EINVAL;
    try {
        std::vector<uint64_t> occ;
        std::vector<int64_t> counts;
        if (s->algo == PM_ALGO_AC && s->params.stride == 2) host_walk_ac2(s->ac, T, n, occ, counts);
        else if (s->algo == PM_ALGO_AC) host_walk_ac(s->ac, T, n, occ, counts);
        else if (s->algo == PM_ALGO_PFAC) host_walk_pfac(s->ac, T, n, occ, counts);
        else if (s->algo == PM_ALGO_ACV) host_walk_acv(s->acv, T, n, occ, counts);
        else if (s->algo == PM_ALGO_WMV) host_walk_wmv(s->wm, T, n, occ, counts);
        else host_walk_wm(s->wm, T, n, occ, counts);
        pm_result *r = new_result(int64_t(counts.size()), int64_t(occ.size()), true, false);
        if (!r) return PM_ENOMEM;
        if (!occ.empty()) std::memcpy(r->occ, occ.data(), occ.size() * 8);
        std::memcpy(r->counts, counts.data(), counts.size() * 8);
        *out = r;
        return PM_OK;
    } catch (const std::bad_alloc &) {
        return PM_ENOMEM;
    }
}

}  // extern "C"
