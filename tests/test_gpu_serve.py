"""GPU tests of the serving loop: results alone and in the mix are identical.

Requests of mixed sizes and sets (list and counts-only) are submitted from
several threads at staggered times, so batches form while others run; every
result must equal, bit for bit, the solo scan of the same text with the same
set (and the oracle on a sample). Tight memory budgets (admission waits),
short occurrence estimates (exact-capacity re-runs) and rejected requests
are covered too.
"""
import os
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1407_2889_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU-only machines, never run there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1407_2889_gb300 import pmscan as pm  # noqa: E402

THREADS = os.cpu_count() or 4
BASE_N = 8 << 20


@pytest.fixture(scope="module")
def base():
    return synth.est_text(BASE_N, 11)


@pytest.fixture(scope="module")
def sets(base):
    shapes = [(50, 8), (400, 12), (3000, 8), (1200, 24), (5000, 16), (800, 40)]
    out = []
    for j, (d, m) in enumerate(shapes):
        P = synth.batch_patterns(base, (j * 977 * 4096) % (BASE_N - (1 << 20)), 1 << 20, d, m, 700 + j)
        out.append((P, pm.PatternSet.ac(P)))
    return out


def _requests(k, seed, n_hi=1 << 19, nsets=6):
    u = synth.uniform01(seed, synth.SID_MISC, 4 * k).reshape(k, 4)
    reqs = []
    for j in range(k):
        n = int(round(1024 * (n_hi / 1024) ** u[j, 0]))
        off = int(u[j, 1] * (BASE_N - n))
        reqs.append((int(u[j, 2] * nsets) % nsets, off, n, bool(u[j, 3] < 0.2)))
    return reqs


def _run_mixed(srv, base, sets, reqs, nthreads=4):
    tickets = [None] * len(reqs)
    errors = []

    def submitter(idx):
        rng = np.random.default_rng(idx)
        try:
            for j in range(idx, len(reqs), nthreads):
                si, off, n, co = reqs[j]
                tickets[j] = srv.submit(sets[si][1], base[off:off + n], counts_only=co)
                if rng.random() < 0.3:
                    time.sleep(float(rng.random()) * 2e-3)
        except Exception as e:  # surfaced below
            errors.append(e)

    th = [threading.Thread(target=submitter, args=(i,)) for i in range(nthreads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    return [srv.wait(t) for t in tickets]


def _solo(base, sets, reqs):
    out = []
    for si, off, n, co in reqs:
        occ, cnt = sets[si][1].scan(base[off:off + n], counts_only=co)
        out.append((occ, cnt))
    return out


def _same(got, want, j):
    assert np.array_equal(got[1], want[1]), f"request {j}: counts differ"
    assert np.array_equal(got[0], want[0]), f"request {j}: occurrences differ"


def test_results_alone_and_in_the_mix(base, sets):
    reqs = _requests(300, 31)
    solo = _solo(base, sets, reqs)
    # pin the solo path to the oracle on a sample of requests
    for j in range(0, len(reqs), 15):
        si, off, n, co = reqs[j]
        wo, wc = oracle.dictionary(base[off:off + n], sets[si][0], threads=THREADS)
        assert np.array_equal(solo[j][1], wc)
        if not co:
            assert np.array_equal(solo[j][0], wo)
    srv = pm.Server(budget_bytes=256 << 20, max_batch=64, max_inflight=3)
    try:
        got = _run_mixed(srv, base, sets, reqs)
        for j, (g, w) in enumerate(zip(got, solo)):
            _same(g, w, j)
        st = srv.stats()
        assert st["completed"] == len(reqs)
        assert st["bytes"] == sum(r[2] for r in reqs)
        assert 0 < st["p50_us"] <= st["p99_us"]
        assert st["batches"] >= 1 and st["mean_batch"] >= 1.0
        assert st["arena_used"] == 0 and st["pending"] == 0
    finally:
        srv.close()


def test_tight_budget_admission_waits(base, sets):
    reqs = _requests(60, 32, n_hi=1 << 18)
    solo = _solo(base, sets, reqs)
    srv = pm.Server(budget_bytes=3 << 20, max_batch=8, max_inflight=2)
    try:
        got = _run_mixed(srv, base, sets, reqs, nthreads=3)
        for j, (g, w) in enumerate(zip(got, solo)):
            _same(g, w, j)
        with pytest.raises(pm.PmError) as e:  # larger than the whole arena
            srv.submit(sets[0][1], base[: 4 << 20])
        assert e.value.code == pm.PM_ETOOBIG
    finally:
        srv.close()


def test_short_estimate_reruns_with_exact_capacity(base):
    T = np.full(300000, ord("A"), np.uint8)
    T[::997] = ord("C")
    P = np.full((4, 8), ord("A"), np.uint8)  # four equal patterns: every window matches 4 times
    s = pm.PatternSet.ac(P)
    want = s.scan(T)
    srv = pm.Server(budget_bytes=64 << 20)
    try:
        t = srv.submit(s, T)
        got = srv.wait(t)
        _same(got, want, 0)
        assert srv.stats()["reruns"] >= 1
    finally:
        srv.close()


def test_rejected_requests(base, sets):
    srv = pm.Server(budget_bytes=16 << 20)
    try:
        wm = pm.PatternSet.wm(sets[0][0], 2)
        with pytest.raises(pm.PmError) as e:
            srv.submit(wm, base[:4096])
        assert e.value.code == pm.PM_EINVAL
        # empty and shorter-than-m texts are ordinary requests
        t0 = srv.submit(sets[0][1], base[:0])
        t1 = srv.submit(sets[0][1], base[:5])
        for t in (t0, t1):
            occ, cnt = srv.wait(t)
            assert occ.size == 0 and cnt.sum() == 0
    finally:
        srv.close()


def test_results_outlive_the_server(base, sets):
    """Result arrays come from the server's page-locked pool; a result freed
    after pm_server_destroy is still intact (the pool lives until then)."""
    import ctypes
    L = pm.lib()
    T = base[: 1 << 20]
    want = sets[2][1].scan(T)
    srv = pm.Server(budget_bytes=64 << 20, host_pool_bytes=64 << 20)
    t = srv.submit(sets[2][1], T)
    rp = ctypes.POINTER(pm.pm_result)()
    assert L.pm_server_wait(srv.h, t, ctypes.byref(rp)) == pm.PM_OK
    srv._keep.clear()
    srv.close()
    r = rp.contents
    cnt = np.ctypeslib.as_array(r.counts, shape=(r.d,)).copy()
    occ = np.ctypeslib.as_array(r.occ, shape=(r.n_occ,)).copy() if r.n_occ else np.zeros(0, np.uint64)
    L.pm_result_free(rp)
    _same((occ, cnt), want, 0)



@pytest.mark.parametrize("counter_words", [0, 30000])
def test_large_requests_split_or_plain(base, sets, counter_words):
    """Requests of several MiB among small ones: the batched launch splits
    them across CTAs (parts staging their keys); with a small per-slot
    workspace the ones whose words could not fit run as whole-GPU scans.
    Either way every result equals the solo scan."""
    reqs = _requests(40, 33, n_hi=1 << 16)
    for j, (si, off, n) in enumerate([(2, 0, 8 << 20), (1, 1 << 20, 5 << 20), (4, 123, 3 << 20),
                                      (0, 777, 2 << 20), (3, 4096, 6 << 20)]):
        reqs.insert(3 * j, (si, off, n, j == 3))
    solo = _solo(base, sets, reqs)
    srv = pm.Server(budget_bytes=512 << 20, max_batch=32, max_inflight=2, counter_words=counter_words)
    try:
        got = _run_mixed(srv, base, sets, reqs, nthreads=2)
        for j, (g, w) in enumerate(zip(got, solo)):
            _same(g, w, j)
        assert srv.stats()["completed"] == len(reqs)
    finally:
        srv.close()
