"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Every comparison is bit-exact: occurrence keys (i << 32 | r) element by
element and per-pattern counts. Small cases span several warp tiles and a
ragged tail; the workload sizes compare against the oracle in full where it
finishes in seconds, and at the full 1 GiB size in the launch configuration
bench.py times, on sampled windows plus properties checked on every output
(each reported pair is an occurrence, order, counts, and the exact total
from an independent window-key count done with plain torch ops).
"""
import os

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


def _ac(P, **kw):
    return pm.PatternSet.ac(P, kw or None)


def _wm(P, B, **kw):
    return pm.PatternSet.wm(P, B, kw or None)


def _same(got, want, what=""):
    go, gc = got
    wo, wc = want
    assert go.size == wo.size, f"{what}: {go.size} occurrences, oracle {wo.size}"
    assert np.array_equal(go, wo), f"{what}: occurrence lists differ"
    assert np.array_equal(gc, wc), f"{what}: counts differ"


def _random_case(rng, alphabet, n_max=20000, m_max=20, d_max=60):
    n = int(rng.integers(0, n_max))
    m = int(rng.integers(1, m_max + 1))
    d = int(rng.integers(1, d_max))
    A = np.frombuffer(alphabet, np.uint8)
    T = A[rng.integers(0, A.size, n)]
    P = A[rng.integers(0, A.size, (d, m))]
    for r in range(d):
        if n >= m and rng.random() < 0.6:
            s = int(rng.integers(0, n - m + 1))
            P[r] = T[s:s + m]
    if d > 2 and rng.random() < 0.5:
        P[-1] = P[0]
    return T, np.ascontiguousarray(P)


# ---------------------------------------------------------------------------
# small cases: random alphabets, lengths, duplicates, ragged tails
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("alphabet", [b"ACGT", b"ACGTN\n", b"AC", b"acgt", b"xyzw#", bytes(range(1, 250, 3))])
def test_ac_random_small(alphabet):
    rng = np.random.default_rng(alphabet[0] * 7 + len(alphabet))
    for case in range(25):
        T, P = _random_case(rng, alphabet, m_max=65 if case % 3 == 0 else 20)
        want = oracle.brute(T, P)
        s = _ac(P)
        _same(s.scan(T), want, f"AC case {case} n={T.size} m={P.shape[1]} d={P.shape[0]}")
        _same(s.scan(torch.from_numpy(T).cuda()), want, "AC device text")
        occ, cnt = s.scan(T, counts_only=True)
        assert occ.size == 0 and np.array_equal(cnt, want[1])
        s.close()


@pytest.mark.parametrize("alphabet", [b"ACGT", b"ACGTN\n", b"AC", b"xyzw#", bytes(range(1, 250, 3))])
def test_pfac_random_small(alphabet):
    rng = np.random.default_rng(alphabet[0] * 11 + len(alphabet))
    for case in range(20):
        T, P = _random_case(rng, alphabet, m_max=65 if case % 3 == 0 else 20)
        want = oracle.brute(T, P)
        s = pm.PatternSet.pfac(P)
        _same(s.scan(T), want, f"PFAC case {case} n={T.size} m={P.shape[1]} d={P.shape[0]}")
        occ, cnt = s.scan(torch.from_numpy(T).cuda(), counts_only=True)
        assert occ.size == 0 and np.array_equal(cnt, want[1])
        s.close()


def test_pfac_est_sets_and_every_position_matching(est_text_full):
    T = est_text_full[: 32 << 20]
    for d, m in ((1000, 8), (8000, 8), (20000, 16), (8000, 32)):
        _, P = synth.est_case(d, m, text=est_text_full)
        want = oracle.dictionary(T, P, threads=THREADS)
        # the default ACGT plans run 24 warps per CTA; 12 and 20 are pinned
        for kw in ({},) + (({"warps_per_cta": 12}, {"warps_per_cta": 20}) if d == 8000 else ()):
            s = pm.PatternSet.pfac(P, kw or None)
            _same(s.scan(T), want, f"PFAC d={d} m={m} {kw}")
            s.close()
    A = np.full(300000, ord("A"), np.uint8)
    s = pm.PatternSet.pfac(np.full((3, 8), ord("A"), np.uint8))
    _same(s.scan(A), oracle.dictionary(A, np.full((3, 8), ord("A"), np.uint8)), "PFAC all hits")
    s.close()


@pytest.mark.parametrize("B", [1, 2, 3, 4])
def test_wm_random_small(B):
    rng = np.random.default_rng(1000 + B)
    for case in range(25):
        T, P = _random_case(rng, b"ACGTN\n", m_max=40)
        if P.shape[1] < B:
            continue
        want = oracle.brute(T, P)
        s = _wm(P, B)
        _same(s.scan(T), want, f"WM B={B} case {case} n={T.size} m={P.shape[1]}")
        occ, cnt = s.scan(T, counts_only=True)
        assert np.array_equal(cnt, want[1])
        s.close()


def test_wm_byte_path_groups_and_overflow():
    """Sets outside the ACGT-like form take the byte-hash walk; equal
    patterns enter HASH once under a group code (every id reported, in
    ascending order), and a lane whose pool overflows walks its staged bytes
    again."""
    rng = np.random.default_rng(77)
    A = np.frombuffer(b"ACGTN", np.uint8)
    T = A[rng.integers(0, 5, 300000)]
    P = A[rng.integers(0, 5, (300, 6))]
    for r in range(0, 300, 3):  # a third copied from the text
        s0 = int(rng.integers(0, T.size - 6))
        P[r] = T[s0:s0 + 6]
    P[1] = P[0]
    P[2] = P[0]
    P[5] = P[4]
    want = oracle.dictionary(T, P, threads=THREADS)
    for B in (2, 3):
        s = _wm(P, B)
        info = s.info()
        assert info["dna_mode"] == 0 and info["n_distinct"] < P.shape[0]
        _same(s.scan(T), want, f"byte path B={B}")
        occ, cnt = s.scan(T, counts_only=True)
        assert np.array_equal(cnt, want[1])
        s.close()
    Tn = np.full(40000, ord("N"), np.uint8)
    Pn = np.array([list(b"NNNNNNNN"), list(b"NNNNNNNN"), list(b"ANNNNNNN")], np.uint8)
    s = _wm(Pn, 2)
    _same(s.scan(Tn), oracle.brute(Tn, Pn), "all-N, every window a match")
    s.close()


def test_edge_cases():
    P = np.frombuffer(b"ACGTACGT", np.uint8).reshape(1, 8)
    for n in [0, 1, 7, 8, 9, 15, 16, 17, 2559, 2560, 2561, 2567, 5120 + 3]:
        T = synth.uniform_dna(n, 11)
        T[: min(n, 8)] = P[0, : min(n, 8)]
        want = oracle.brute(T, P)
        for s in (_ac(P), _wm(P, 3)):
            _same(s.scan(T), want, f"n={n}")
            s.close()


def test_every_position_matches_overflow_path():
    """A^n against A^m (and a duplicate): each lane sees 80 matches, more than
    its 40-entry pool, so the overflow re-walk writes directly."""
    T = np.full(50000, ord("A"), np.uint8)
    T[777] = ord("C")
    P = np.array([list(b"AAAAAAAA"), list(b"AAAAAAAA"), list(b"CAAAAAAA")], np.uint8)
    want = oracle.brute(T, P)
    assert want[0].size > 90000
    for s in (_ac(P), _wm(P, 2)):
        _same(s.scan(T), want, "all-A")
        occ, cnt = s.scan(T, counts_only=True)
        assert np.array_equal(cnt, want[1])
        s.close()


def test_unaligned_device_text():
    T = synth.est_text(300000, 5)
    P = synth.mixed_patterns(T, 300, 8, 5)
    d = torch.from_numpy(T).cuda()
    for off in (1, 3, 8, 15):
        sub = d[off:]
        want = oracle.dictionary(T[off:], P, threads=THREADS)
        for s in (_ac(P), _wm(P, 3)):
            _same(s.scan(sub), want, f"offset {off}")
            s.close()


@pytest.mark.parametrize("kw", [
    {"placement": pm.PM_PLACE_HYBRID, "smem_table_bytes": 4096},
    {"placement": pm.PM_PLACE_GLOBAL},
    {"warps_per_cta": 8},
    {"warps_per_cta": 12},
    {"ctas_per_sm": 2, "warps_per_cta": 4},
    {"ids_place": 3, "placement": pm.PM_PLACE_HYBRID, "smem_table_bytes": 4096},
    {"ids_place": 3, "warps_per_cta": 8, "counters": 2},
])
def test_placements_and_launch_shapes_agree(kw):
    T = synth.est_text(1 << 21, 6)
    P = synth.mixed_patterns(T, 2000, 12, 6)
    want = oracle.dictionary(T, P, threads=THREADS)
    s = _ac(P, **kw)
    _same(s.scan(T), want, str(kw))
    s.close()


@pytest.mark.parametrize("counters", [1, 2, 3])
@pytest.mark.parametrize("ids_place", [1, 2, 3])
def test_counter_and_id_placements_agree(counters, ids_place):
    """Per-terminal counters (32-bit / 16-bit shared, device memory) and the
    terminal-id structure (shared / device / late: codes and counts taken in
    the expand kernel in list mode) give identical results; the 16-bit
    counters overflow into the device counter many times here, and the run
    of one letter puts a group of two equal patterns on every position."""
    T = synth.est_text(4 << 20, 21)
    P = synth.mixed_patterns(T, 3000, 8, 21)
    P = np.concatenate([P, P[:7]])
    want = oracle.dictionary(T, P, threads=THREADS)
    s = _ac(P, counters=counters, ids_place=ids_place)
    _same(s.scan(T), want, f"counters={counters} ids={ids_place}")
    s.close()
    n = 8 << 20
    A = np.full(n, ord("A"), np.uint8)
    s = _ac(np.full((2, 8), ord("A"), np.uint8), counters=counters, ids_place=ids_place)
    occ, cnt = s.scan(A, counts_only=True)
    assert cnt.tolist() == [n - 7, n - 7]
    k = 1 << 20
    occ, cnt = s.scan(A[:k])
    assert cnt.tolist() == [k - 7, k - 7]
    pos = np.repeat(np.arange(k - 7, dtype=np.uint64), 2)
    assert np.array_equal(occ, (pos << np.uint64(32)) | np.tile(np.array([0, 1], np.uint64), k - 7))
    s.close()


def test_autotuner_keeps_results():
    T = synth.est_text(16 << 20, 22)
    P = synth.mixed_patterns(T, 8000, 8, 22)
    want = oracle.dictionary(T, P, threads=THREADS)
    s = _ac(P)
    params, ms = s.tune(torch.from_numpy(T).cuda(), reps=2)
    assert ms > 0 and params["counters"] in (0, 1, 2, 3)
    _same(s.scan(T), want, f"tuned {params}")
    _same(s.scan(T, counts_only=True), (np.zeros(0, np.uint64), want[1]), "tuned counts")
    s.close()
    w = _wm(P, 3)
    params, ms = w.tune(torch.from_numpy(T).cuda(), reps=1)
    assert ms > 0 and params["warps_per_cta"] in (0, 8, 12, 16, 20, 24)
    _same(w.scan(T), want, f"WM tuned {params}")
    w.close()
    pf = pm.PatternSet.pfac(P)
    with pytest.raises(pm.PmError):
        pf.tune(torch.from_numpy(T[:4096]).cuda())
    pf.close()


def test_device_api_capacity_and_status():
    T = synth.uniform_dna(1 << 20, 0)
    P = synth.mixed_patterns(T, 100, 8, 0)
    want_occ, want_cnt = oracle.brute(T, P)
    s = _ac(P)
    d_text = torch.from_numpy(T).cuda()
    ws = torch.zeros(s.workspace_bytes(T.size), dtype=torch.uint8, device="cuda")
    counts = torch.zeros(100, dtype=torch.int64, device="cuda")
    nocc = torch.zeros(1, dtype=torch.int64, device="cuda")
    cap = want_occ.size // 2
    occ = torch.zeros(cap, dtype=torch.int64, device="cuda")
    pm.pm_scan_device(s.h, d_text, T.size, 0, counts, occ, cap, nocc, ws, ws.numel())
    assert pm.pm_scan_status(ws) == pm.PM_OK
    assert int(nocc.item()) == want_occ.size  # the total is exact even when truncated
    assert np.array_equal(occ.cpu().numpy().view(np.uint64), want_occ[:cap])
    assert np.array_equal(counts.cpu().numpy(), want_cnt)
    s.close()


def test_small_uniform_workload():
    """1 MiB uniform ACGT, d=100, m=8 (50 copied from the text, 50 random);
    AC and WM with B=2, bit-exact against the brute-force definition."""
    T, P = synth.small_uniform_case()
    want = oracle.brute(T, P)
    for s in (_ac(P), _wm(P, 2)):
        _same(s.scan(T), want, "1 MiB uniform")
        s.close()


# ---------------------------------------------------------------------------
# EST-shaped workloads
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def est_text_full():
    return synth.est_text(synth.EST_N, 1)


@pytest.mark.parametrize("d", synth.EST_D)
@pytest.mark.parametrize("m", synth.EST_M)
def test_est_sets_on_64mib_prefix(est_text_full, d, m):
    """Each (d, m) set of the EST workload, patterns drawn from the full text,
    scanned over a 64 MiB prefix and compared with the oracle in full."""
    _, P = synth.est_case(d, m, text=est_text_full)
    T = est_text_full[: 64 << 20]
    want = oracle.dictionary(T, P, threads=THREADS)
    s = _ac(P)
    if (d, m) == (20000, 8):  # late ids keep its 136 KB table whole in shared memory
        assert s.info()["placement"] == pm.PM_PLACE_SMEM
    _same(s.scan(T), want, f"AC d={d} m={m}")
    s.close()
    if d <= 8000 or m >= 16:   # WM at m=8, d=20000 checks every window; prefix kept short
        s = _wm(P, 3)
        Tw = T if d <= 8000 else T[: 16 << 20]
        wantw = want if d <= 8000 else oracle.dictionary(Tw, P, threads=THREADS)
        _same(s.scan(Tw), wantw, f"WM d={d} m={m}")
        s.close()


def _window_keys_total(d_text: "torch.Tensor", P: np.ndarray):
    """Exact occurrence total and per-pattern counts of m=8 patterns by plain
    torch ops: each window of 8 ACGT bytes -> 16-bit key -> multiplicity."""
    m = P.shape[1]
    assert m == 8
    lut = torch.full((256,), -1, dtype=torch.int64, device=d_text.device)
    for c, b in enumerate(b"ACGT"):
        lut[b] = c
    code = lut[d_text.long()]
    n = code.numel()
    key = torch.zeros(n - m + 1, dtype=torch.int64, device=d_text.device)
    bad = torch.zeros(n - m + 1, dtype=torch.bool, device=d_text.device)
    for j in range(m):
        cj = code[j:n - m + 1 + j]
        bad |= cj < 0
        key = key * 4 + cj.clamp(min=0)
    pk = np.zeros(P.shape[0], np.int64)
    for j in range(m):
        pk = pk * 4 + np.array([b"ACGT".index(bytes([x])) for x in P[:, j]])
    mult = torch.zeros(1 << 16, dtype=torch.int64, device=d_text.device)
    mult.index_add_(0, torch.from_numpy(pk).cuda(), torch.ones(P.shape[0], dtype=torch.int64, device="cuda"))
    hist = torch.bincount(key[~bad], minlength=1 << 16)
    total = int((hist * mult).sum().item())
    per_pattern = hist[torch.from_numpy(pk).cuda()].cpu().numpy()
    return total, per_pattern


def test_full_size_headline_in_bench_configuration(est_text_full):
    """1 GiB EST text, d=8000, m=8, AC list mode through pm_scan_device with the
    default plan -- the launch bench.py times."""
    T = est_text_full
    _, P = synth.est_case(8000, 8, text=T)
    s = _ac(P)
    d_text = torch.from_numpy(T).cuda()
    n = T.size
    ws = torch.zeros(s.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    counts = torch.zeros(P.shape[0], dtype=torch.int64, device="cuda")
    nocc = torch.zeros(1, dtype=torch.int64, device="cuda")
    cap = n // 4
    occ = torch.zeros(cap, dtype=torch.int64, device="cuda")
    pm.pm_scan_device(s.h, d_text, n, 0, counts, occ, cap, nocc, ws, ws.numel())
    assert pm.pm_scan_status(ws) == pm.PM_OK
    total = int(nocc.item())
    assert 0 < total <= cap
    occ = occ[:total]

    # exact total and counts from an independent computation over every window
    want_total, want_counts = _window_keys_total(d_text, P)
    assert total == want_total
    assert np.array_equal(counts.cpu().numpy(), want_counts)

    # every reported pair is an occurrence; keys strictly increasing
    u = occ.view(torch.int64)
    assert bool((u[1:] > u[:-1]).all())
    i = (u >> 32)
    r = (u & 0xFFFFFFFF)
    Pd = torch.from_numpy(P).cuda()
    for j in range(8):
        assert bool((d_text[i + j] == Pd[r, j]).all())

    # sampled windows against the oracle, element by element
    rng = np.random.default_rng(8000)
    occ_np = occ.cpu().numpy().view(np.uint64)
    starts = occ_np >> np.uint64(32)
    W = 1 << 18
    for a in rng.integers(0, n - W, 24):
        a = int(a)
        wo, _ = oracle.dictionary(T[a:a + W + 7], P, threads=THREADS)
        wi, wr = oracle.unpack(wo)
        keep = wi < W
        want = ((wi[keep] + a).astype(np.uint64) << np.uint64(32)) | wr[keep].astype(np.uint64)
        lo = np.searchsorted(starts, a)
        hi = np.searchsorted(starts, a + W)
        assert np.array_equal(occ_np[lo:hi], want), f"window at {a}"
    s.close()


@pytest.mark.parametrize("d", [100000, 500000])
def test_large_sets_full_text(est_text_full, d):
    """Large pattern sets (m=32): the AC table (u32, 2.3M / 11M rows) only
    fits shared memory as a breadth-first prefix; the rest is read through
    L2/HBM. Full 1 GiB text against the oracle in full; WM with B=4 (2^20
    SHIFT entries) on a prefix (on ACGT text every 4-byte block ends some
    pattern when d is this large, so WM verifies at every position)."""
    T = est_text_full
    P = synth.large_set(d, T)
    s = _ac(P)
    info = s.info()
    assert info["entry_bytes"] == 4 and info["placement"] == pm.PM_PLACE_HYBRID
    assert info["smem_rows"] < info["n_rows"]
    want = oracle.dictionary(T, P, threads=THREADS)
    _same(s.scan(torch.from_numpy(T).cuda()), want, f"AC d={d}")
    s.close()
    nw = (16 << 20) if d == 100000 else (2 << 20)
    w = _wm(P, 4)
    assert w.info()["shift_entries"] == 1 << 20
    _same(w.scan(T[:nw]), oracle.dictionary(T[:nw], P, threads=THREADS), f"WM B=4 d={d}")
    w.close()


def test_scan_to_host_in_pieces(est_text_full):
    """Long host texts go through pm_scan_to_host in pieces (copies
    overlapping scans, keys leaving per piece); results equal one scan of the
    whole text, also with a short capacity, in counts-only mode and for PFAC."""
    T = est_text_full[: (200 << 20) + 12345]
    _, P = synth.est_case(1000, 8, text=est_text_full)
    want_occ, want_cnt = oracle.dictionary(T, P, threads=THREADS)
    pinned = torch.from_numpy(T).pin_memory()
    for make in (_ac, pm.PatternSet.pfac, lambda P: _ac(P, ids_place=3)):
        s = make(P)
        counts = torch.zeros(P.shape[0], dtype=torch.int64).pin_memory()
        occ = torch.zeros(want_occ.size + 7, dtype=torch.int64).pin_memory()
        for rep in range(2):
            counts.zero_()
            total = pm.pm_scan_to_host(s.h, pinned, counts, occ)
            assert total == want_occ.size
            assert np.array_equal(occ.numpy()[:total].view(np.uint64), want_occ)
            assert np.array_equal(counts.numpy(), want_cnt)
        short = torch.zeros(want_occ.size // 3, dtype=torch.int64).pin_memory()
        with pytest.raises(pm.PmError) as e:
            pm.pm_scan_to_host(s.h, pinned, counts, short)
        assert e.value.code == pm.PM_ECAPACITY
        assert np.array_equal(short.numpy().view(np.uint64), want_occ[: short.numel()])
        counts.zero_()
        assert pm.pm_scan_to_host(s.h, pinned, counts, None, pm.PM_COUNTS_ONLY) == want_occ.size
        assert np.array_equal(counts.numpy(), want_cnt)
        s.close()


def test_scan_to_host_pinned_buffers_and_capacity():
    T = synth.est_text(1 << 21, 9)
    P = synth.mixed_patterns(T, 500, 8, 9)
    want_occ, want_cnt = oracle.dictionary(T, P, threads=THREADS)
    s = _ac(P)
    pinned = torch.from_numpy(T).pin_memory()
    counts = torch.zeros(500, dtype=torch.int64).pin_memory()
    occ = torch.zeros(want_occ.size, dtype=torch.int64).pin_memory()
    total = pm.pm_scan_to_host(s.h, pinned, counts, occ)
    assert total == want_occ.size
    assert np.array_equal(occ.numpy().view(np.uint64), want_occ)
    assert np.array_equal(counts.numpy(), want_cnt)
    small = torch.zeros(10, dtype=torch.int64)
    with pytest.raises(pm.PmError) as e:
        pm.pm_scan_to_host(s.h, T, counts, small)
    assert e.value.code == pm.PM_ECAPACITY
    assert np.array_equal(small.numpy().view(np.uint64), want_occ[:10])
    s.close()


def test_stride2_scan_matches_oracle():
    """Two characters per lookup: random ACGT sets over texts with N and
    newline bytes (matches whose window holds one are dropped), odd and even
    m up to 33, duplicates, list and counts modes, unaligned device text, a
    text where every position matches (pool overflow), and the tuner."""
    rng = np.random.default_rng(1200)
    A = np.frombuffer(b"ACGT", np.uint8)
    for case in range(24):
        m = int(rng.choice([1, 2, 3, 7, 8, 9, 16, 17, 33]))
        d = int(rng.integers(1, 200))
        n = int(rng.integers(0, 300000))
        T = np.frombuffer(b"ACGTN\n", np.uint8)[rng.choice(6, n, p=[.2425, .2425, .2425, .2425, .02, .01])]
        P = A[rng.integers(0, 4, (d, m))]
        for r in range(d):
            if n >= m and rng.random() < 0.6:
                s0 = int(rng.integers(0, n - m + 1))
                if all(x in b"ACGT" for x in T[s0:s0 + m].tobytes()):
                    P[r] = T[s0:s0 + m]
        if d > 2:
            P[-1] = P[0]
        P = np.ascontiguousarray(P)
        try:
            s = _ac(P, stride=2)
        except pm.PmError as e:
            assert e.code == pm.PM_ETOOBIG
            continue
        assert s.info()["stride"] == 2
        want = oracle.dictionary(T, P, threads=THREADS)
        _same(s.scan(T), want, f"stride 2, case {case}, m={m}, n={n}")
        _, cnt = s.scan(T, counts_only=True)
        assert np.array_equal(cnt, want[1])
        if n > 5:
            d_T = torch.from_numpy(T).cuda()
            _same(s.scan(d_T[3:]), oracle.dictionary(T[3:], P, threads=THREADS), f"stride 2 unaligned {case}")
        s.close()
    T = np.full(60000, ord("A"), np.uint8)
    T[999] = ord("N")
    P = np.array([list(b"AAAAAAAA"), list(b"AAAAAAAA"), list(b"CAAAAAAA")], np.uint8)
    s = _ac(P, stride=2)
    _same(s.scan(T), oracle.brute(T, P), "stride 2, every position")
    s.close()


def test_stride2_est_and_tuner(est_text_full):
    T = est_text_full[: 64 << 20]
    _, P = synth.est_case(1000, 8, text=est_text_full)
    want = oracle.dictionary(T, P, threads=THREADS)
    d_T = torch.from_numpy(T).cuda()
    for kw in ({"stride": 2}, {"stride": 1}, {}):
        s = _ac(P, **kw)
        _same(s.scan(d_T), want, f"EST 64 MiB {kw}")
        if not kw:
            params, ms = s.tune(d_T, reps=1)
            assert params["stride"] in (1, 2) and s.info()["stride"] == params["stride"]
            _same(s.scan(d_T), want, "after tuning")
        s.close()


def test_late_ids_large_set_and_hot_terminal():
    """Late ids (the expand kernel maps terminal ids to codes and counts
    them) on a set whose canon and 32-bit counters do not fit the expand
    CTA's shared memory, so it counts in 16-bit halves: a 300 KB run of one
    letter inside one output segment takes one terminal (a group of three
    equal patterns) past 0x8000 many times. List mode, counts-only mode and
    a short capacity all equal the oracle."""
    T = synth.est_text(64 << 20, 31).copy()
    T[5_000_000:5_300_000] = ord("A")
    P = synth.random_patterns(24000, 8, 31)
    P = np.concatenate([P, np.full((3, 8), ord("A"), np.uint8)])
    want = oracle.dictionary(T, P, threads=THREADS)
    s = _ac(P, ids_place=3)
    _same(s.scan(T), want, "late ids, 16-bit expand counters")
    _same(s.scan(T, counts_only=True), (np.zeros(0, np.uint64), want[1]), "late ids counts only")
    d = torch.from_numpy(T).cuda()
    cap = want[0].size // 2
    counts = torch.zeros(P.shape[0], dtype=torch.int64, device="cuda")
    occ = torch.zeros(cap, dtype=torch.int64, device="cuda")
    nocc = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.zeros(s.workspace_bytes(T.size), dtype=torch.uint8, device="cuda")
    pm.pm_scan_device(s.h, d, T.size, 0, counts, occ, cap, nocc, ws, ws.numel(), None)
    torch.cuda.synchronize()
    assert pm.pm_scan_status(ws, None) == pm.PM_OK
    assert int(nocc.item()) == want[0].size
    assert np.array_equal(occ.cpu().numpy().view(np.uint64), want[0][:cap])
    assert np.array_equal(counts.cpu().numpy(), want[1])
    s.close()


def test_late_ids_large_groups_and_device_id_structure():
    """Late ids in list mode on a u32 table (more than 32,767 patterns) with
    groups of four to six equal patterns, whose multiplicity the scan takes
    from the id structure in device memory; the id structure and counters
    do not fit the expand CTA's shared memory either, so it looks terminals
    up in device memory too. List and counts-only against the oracle."""
    T = synth.est_text(16 << 20, 53).copy()
    T[2_000_000:2_100_000] = ord("C")
    P = synth.random_patterns(60000, 8, 53)
    P = np.concatenate([P, np.full((6, 8), ord("C"), np.uint8), P[:4], P[:4], P[:4]])
    want = oracle.dictionary(T, P, threads=THREADS)
    for kw in ({"ids_place": 3}, {"ids_place": 3, "warps_per_cta": 8}):
        s = _ac(P, **kw)
        assert s.info()["entry_bytes"] == 4
        _same(s.scan(T), want, f"{kw}")
        _same(s.scan(T, counts_only=True), (np.zeros(0, np.uint64), want[1]), f"{kw} counts")
        s.close()


@pytest.mark.parametrize("kw", [{"warps_per_cta": 24}, {"warps_per_cta": 20}, {"warps_per_cta": 17},
                                {"warps_per_cta": 24, "ids_place": 3}, {"warps_per_cta": 22, "ids_place": 3},
                                {"ids_place": 3}, {"warps_per_cta": 24, "counters": 2}])
def test_more_than_16_warps(kw):
    """Plans of more than 16 warps per CTA (the 768-thread kernels of u16
    ACGT tables wholly in shared memory), with late ids too, whose counts
    mode may use fewer warps than list mode: list, counts-only and a short
    capacity equal the oracle; a run of one letter fills every pool, and
    its pattern is a group of five equal ones."""
    T = synth.est_text(6 << 20, 43).copy()
    T[1_000_000:1_040_000] = ord("A")
    P = synth.mixed_patterns(T, 1500, 9, 43)
    P = np.concatenate([P, P[:11], np.full((5, 9), ord("A"), np.uint8)])
    want = oracle.dictionary(T, P, threads=THREADS)
    s = _ac(P, **kw)
    assert s.info()["placement"] == pm.PM_PLACE_SMEM
    _same(s.scan(T), want, f"{kw}")
    _same(s.scan(T, counts_only=True), (np.zeros(0, np.uint64), want[1]), f"{kw} counts")
    d = torch.from_numpy(T).cuda()
    cap = want[0].size // 3
    counts = torch.zeros(P.shape[0], dtype=torch.int64, device="cuda")
    occ = torch.zeros(cap, dtype=torch.int64, device="cuda")
    nocc = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.zeros(s.workspace_bytes(T.size), dtype=torch.uint8, device="cuda")
    pm.pm_scan_device(s.h, d, T.size, 0, counts, occ, cap, nocc, ws, ws.numel(), None)
    assert pm.pm_scan_status(ws, None) == pm.PM_OK
    assert int(nocc.item()) == want[0].size
    assert np.array_equal(occ.cpu().numpy().view(np.uint64), want[0][:cap])
    s.close()


@pytest.mark.parametrize("kw", [
    {"placement": pm.PM_PLACE_HYBRID, "smem_table_bytes": 16384, "warps_per_cta": 24},
    {"placement": pm.PM_PLACE_HYBRID, "smem_table_bytes": 8192, "warps_per_cta": 20, "ids_place": 3},
    {"placement": pm.PM_PLACE_HYBRID, "warps_per_cta": 18, "counters": 2},
])
@pytest.mark.parametrize("m", [9, 20])
def test_more_than_16_warps_hybrid(kw, m):
    """The 768-thread kernels with the table partly in device memory: u16
    tables (m = 9) and u32 tables (m = 20: more than 32,768 rows), list and
    counts-only, against the oracle."""
    T = synth.est_text(4 << 20, 47)
    P = synth.mixed_patterns(T, 3000, m, 47)
    P = np.concatenate([P, P[:5]])
    want = oracle.dictionary(T, P, threads=THREADS)
    s = _ac(P, **kw)
    inf = s.info()
    assert inf["placement"] == pm.PM_PLACE_HYBRID and inf["entry_bytes"] == (2 if m == 9 else 4)
    _same(s.scan(T), want, f"{kw} m={m}")
    _same(s.scan(T, counts_only=True), (np.zeros(0, np.uint64), want[1]), f"{kw} m={m} counts")
    s.close()


@pytest.mark.parametrize("w", [17, 20, 24])
@pytest.mark.parametrize("m", [8, 20])
def test_wm_more_than_16_warps(w, m):
    """Wu-Manber exact-code plans of more than 16 warps per CTA (the
    768-thread kernels), fixed and mixed lengths, list and counts-only,
    against the oracle."""
    T = synth.est_text(4 << 20, 53)
    P = synth.mixed_patterns(T, 1200, m, 53)
    P = np.concatenate([P, P[:7]])
    want = oracle.dictionary(T, P, threads=THREADS)
    s = _wm(P, 3, warps_per_cta=w)
    assert s.info()["dna_mode"] == 1
    _same(s.scan(T), want, f"WM m={m} warps={w}")
    _same(s.scan(T, counts_only=True), (np.zeros(0, np.uint64), want[1]), f"WM m={m} warps={w} counts")
    s.close()
    Pv = synth.mixed_length_patterns(T, 600, 8, 16, 53)
    sv = pm.PatternSet.wmv(Pv, 3, {"warps_per_cta": w})
    _same(sv.scan(T), oracle.dictionary_var(T, Pv, threads=THREADS), f"WM mixed lengths warps={w}")
    sv.close()
