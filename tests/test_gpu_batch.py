"""GPU parity of the batched scan: many (text, set) instances in one launch.

Each instance's result must equal, bit for bit, the oracle's result for
that instance alone (and the plain single-scan kernel's), whatever warps per
CTA the tuner picks, replayed from a captured CUDA graph or not. Instances
mix text lengths (empty, shorter than m, one warp tile, ragged), unaligned
starts, sets shared between instances, duplicate patterns, sets whose table
fits the CTA's shared memory and sets that only fit its prefix (16- and
32-bit entries), and lanes whose hit pool overflows.
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
BASE_N = 8 << 20
A_RUN = 20000  # a run of 'A' bytes appended to the base text


@pytest.fixture(scope="module")
def base():
    t = synth.est_text(BASE_N, 7)
    return np.concatenate([t, np.full(A_RUN, ord("A"), np.uint8)])


@pytest.fixture(scope="module")
def d_base(base):
    return torch.from_numpy(base).cuda()


def _mixed_instances(base, k=40, seed=900):
    """Seeded instance shapes plus hand-made edge instances.

    Returns (sets, patterns, off, length) with sets[j] compiled from
    patterns[j]; some sets are shared by several instances."""
    off, ln, d, m = synth.batch_plan(k, BASE_N, seed=seed, n_range=(1 << 10, 1 << 20),
                                     d_range=(10, 2000), m_range=(8, 64))
    Ps = [synth.batch_patterns(base[:BASE_N], int(off[j]), int(ln[j]), int(d[j]), int(m[j]), seed + j)
          for j in range(k)]
    offs, lens = list(off), list(ln)
    # edge instances
    P_dup = Ps[0].copy()
    P_dup[-1] = P_dup[0]                      # a duplicate pattern
    extra = [
        (Ps[1], int(off[1]), 0),              # empty text
        (Ps[2], int(off[2]), int(m[2]) - 1),  # shorter than m
        (Ps[3], 4096, 2560),                  # exactly one warp tile
        (Ps[4], 123459, 70001),               # unaligned start, ragged tail
        (P_dup, int(off[0]), int(ln[0])),     # duplicates
        (np.full((3, 8), ord("A"), np.uint8), BASE_N + 5, A_RUN - 5),  # every step a hit
    ]
    for P, o, n in extra:
        Ps.append(P)
        offs.append(o)
        lens.append(n)
    sets = [pm.PatternSet.ac(P) for P in Ps]
    # a set shared by two instances
    sets.append(sets[5])
    Ps.append(Ps[5])
    offs.append(int(off[6]))
    lens.append(int(ln[6]))
    return sets, Ps, np.array(offs, np.int64), np.array(lens, np.int64)


def _oracle_results(base, Ps, off, ln):
    return [oracle.dictionary(base[o:o + n], P, threads=THREADS) for P, o, n in zip(Ps, off, ln)]


def _check(results, want, what):
    assert len(results) == len(want)
    for j, ((o, c, tot), (wo, wc)) in enumerate(zip(results, want)):
        assert tot == wo.size, f"{what}: instance {j} total {tot}, oracle {wo.size}"
        assert np.array_equal(o, wo), f"{what}: instance {j} occurrence list differs"
        assert np.array_equal(c, wc), f"{what}: instance {j} counts differ"


@pytest.fixture(scope="module")
def mixed(base):
    sets, Ps, off, ln = _mixed_instances(base)
    return sets, Ps, off, ln, _oracle_results(base, Ps, off, ln)


def test_batch_matches_oracle_per_instance(d_base, mixed):
    sets, Ps, off, ln, want = mixed
    b = pm.Batch.exact(sets, d_base, off, ln)
    b.scan()
    assert b.status() == pm.PM_OK
    _check(b.results(), want, "batched list mode")
    c = pm.Batch(sets, d_base, off, ln, None)
    c.scan()
    assert c.status() == pm.PM_OK
    for j, ((_, cnt, tot), (wo, wc)) in enumerate(zip(c.results(), want)):
        assert tot == wo.size and np.array_equal(cnt, wc), f"counts-only instance {j}"


def test_batch_every_warp_count_and_graph_replay(d_base, mixed):
    sets, Ps, off, ln, want = mixed
    b = pm.Batch.exact(sets, d_base, off, ln)
    for w in (8, 12, 16, 4):
        for placement in (0, 1):
            b.set_warps(w)
            b.set_placement(placement)
            assert b.placement == placement
            b.scan()
            assert b.status() == pm.PM_OK
            _check(b.results(), want, f"{w} warps per CTA, placement {placement}")
    with pytest.raises(pm.PmError):
        b.set_placement(2)
    ms = b.tune(reps=2)
    assert ms > 0 and b.warps in (8, 12, 16) and b.placement in (0, 1)
    b.capture()
    for rep in range(2):
        b.occ.fill_(-1)
        b.counts.fill_(-1)
        b.replay()
        assert b.status() == pm.PM_OK
        _check(b.results(), want, f"graph replay {rep}")


def test_batch_equals_plain_single_scans(d_base, mixed):
    sets, Ps, off, ln, _ = mixed
    b = pm.Batch.exact(sets, d_base, off, ln)
    b.scan()
    got = b.results()
    for j, (s, o, n) in enumerate(zip(sets, off, ln)):
        po, pc = s.scan(d_base[int(o):int(o) + int(n)])
        assert np.array_equal(got[j][0], po) and np.array_equal(got[j][1], pc), f"instance {j}"


def test_batch_capacity_short(d_base, base, mixed):
    sets, Ps, off, ln, want = mixed
    tot = np.array([w[0].size for w in want])
    caps = tot // 2  # every instance gets half of what it needs
    b = pm.Batch(sets, d_base, off, ln, caps)
    b.scan()
    assert b.status() == pm.PM_OK
    for j, (o, c, t) in enumerate(b.results()):
        assert t == tot[j]
        assert np.array_equal(o, want[j][0][: caps[j]]), f"instance {j}: prefix differs"
        assert np.array_equal(c, want[j][1])


def test_batch_large_tables_hybrid(d_base, base):
    """Sets whose tables exceed the CTA's shared memory (only their
    breadth-first prefix is resident) with 16- and 32-bit entries."""
    cases = [(5000, 64, 0), (20000, 8, 1 << 20), (3000, 33, 3 << 20), (30000, 16, 5 << 20)]
    sets, Ps, off, ln = [], [], [], []
    for j, (d, m, o) in enumerate(cases):
        P = synth.batch_patterns(base[:BASE_N], o, 1 << 20, d, m, 950 + j)
        Ps.append(P)
        sets.append(pm.PatternSet.ac(P))
        off.append(o)
        ln.append((1 << 20) + 4099)
    info = [s.info() for s in sets]
    assert {i["entry_bytes"] for i in info} == {2, 4}
    want = _oracle_results(base, Ps, off, ln)
    b = pm.Batch.exact(sets, d_base, np.array(off), np.array(ln))
    for w in (8, 16):
        b.set_warps(w)
        b.scan()
        assert b.status() == pm.PM_OK
        _check(b.results(), want, f"large tables, {w} warps")


def test_batch_rejects_unsupported_sets(d_base):
    P = synth.random_patterns(10, 8, 1)
    wm = pm.PatternSet.wm(P, 2)
    with pytest.raises(pm.PmError) as e:
        pm.Batch([wm], d_base, [0], [100], [10])
    assert e.value.code == pm.PM_EINVAL
    with pytest.raises(pm.PmError) as e:  # device AC scans take m <= 65
        pm.PatternSet.ac(synth.random_patterns(4, 66, 2))
    assert e.value.code == pm.PM_ETOOBIG
    host_only = pm.PatternSet.ac(synth.random_patterns(4, 8, 2), {"host_only": 1})
    with pytest.raises(pm.PmError):
        pm.Batch([host_only], d_base, [0], [1000], [10])
    other = pm.PatternSet.ac(np.frombuffer(b"ABCDEFGH", np.uint8).reshape(1, 8))
    with pytest.raises(pm.PmError):
        pm.Batch([other], d_base, [0], [1000], [10])
    # an empty batch is fine
    e0 = pm.Batch([], d_base, [], [], [])
    e0.scan()
    assert e0.results() == []


@pytest.mark.parametrize("flags", [0, "counts", "device"])
def test_pm_scan_batch_host_call_against_oracle(base, d_base, flags):
    """pm_scan_batch (the host-pointer batch call of the C ABI): texts of
    mixed sizes -- empty, shorter than m, one byte past a warp tile, ragged,
    a run of one letter -- against AC, WM and PFAC sets, a set shared by two
    instances and a set with a duplicate pattern; every result equals the
    oracle's for that instance alone."""
    rng_lens = [0, 5, 2561, 100_003, 1 << 20, 777_777, 4096, A_RUN + 64]
    starts = [0, 3, 8191, 123_457, 1_000_000, 5_000_001, 7_777_777, BASE_N - 64]
    texts = [base[s:s + n] for s, n in zip(starts, rng_lens)]
    P8 = synth.mixed_patterns(base[: 1 << 20], 400, 8, 61)
    P8 = np.concatenate([P8, P8[:3], np.full((1, 8), ord("A"), np.uint8)])  # duplicates, an A-run pattern
    P12 = synth.mixed_patterns(base[1 << 20: 2 << 20], 150, 12, 62)
    sets = [pm.PatternSet.ac(P8), pm.PatternSet.wm(P12, 3), pm.PatternSet.pfac(P12), pm.PatternSet.ac(P12)]
    pats = [P8, P12, P12, P12]
    which = [0, 1, 2, 3, 0, 3, 1, 0]  # sets 0 and 3 are shared by several instances
    handles = [sets[w].h for w in which]
    fl = pm.PM_COUNTS_ONLY if flags == "counts" else pm.PM_DEVICE_TEXT if flags == "device" else pm.PM_HOST_TEXT
    args = [torch.from_numpy(np.ascontiguousarray(t)).cuda() for t in texts] if flags == "device" else texts
    res = pm.pm_scan_batch(handles, args, fl)
    assert len(res) == len(texts)
    for j, (t, w) in enumerate(zip(texts, which)):
        want_occ, want_cnt = oracle.dictionary(t, pats[w], threads=THREADS)
        occ, cnt = res[j]
        assert np.array_equal(cnt, want_cnt), f"instance {j}: counts"
        if flags == "counts":
            assert occ.size == 0, f"instance {j}: counts only gives no list"
        else:
            assert np.array_equal(occ, want_occ), f"instance {j}: occurrences"
    for s in sets:
        s.close()


def test_batch_splits_large_instances(d_base, base):
    """Large instances among many small ones are split into parts taken by
    different CTAs (each part counts, then writes after the parts before
    it): results per instance equal the oracle's in list mode, counts-only
    mode and with short capacities, including an instance that is one long
    run of a letter (every lane's pool overflows in every part)."""
    big = 4 << 20
    a_run = np.full(big, ord("A"), np.uint8)
    text = np.concatenate([base, a_run])
    d_text = torch.from_numpy(text).cuda()
    a_off = base.size
    Ps, off, ln = [], [], []
    for j in range(3):  # three large EST slices
        o = (j * 2_500_000) & ~15
        P = synth.batch_patterns(base[:BASE_N], o, big, 300 + 200 * j, 8 + 8 * j, 970 + j)
        Ps.append(P), off.append(o), ln.append(min(big, BASE_N - o))
    Ps.append(np.concatenate([np.full((2, 8), ord("A"), np.uint8), synth.random_patterns(20, 8, 9)]))
    off.append(a_off), ln.append(big)
    for j in range(60):  # many small ones
        o = 7_000_000 + 4096 * j
        P = synth.batch_patterns(base[:BASE_N], o, 4096, 50, 8 + (j % 5), 990 + j)
        Ps.append(P), off.append(o), ln.append(1000 + 37 * j)
    sets = [pm.PatternSet.ac(P) for P in Ps]
    want = [oracle.dictionary(text[o:o + n], P, threads=THREADS) for P, o, n in zip(Ps, off, ln)]
    off, ln = np.array(off, np.int64), np.array(ln, np.int64)
    b = pm.Batch.exact(sets, d_text, off, ln)
    for w in (8, 16):
        b.set_warps(w)
        b.scan()
        assert b.status() == pm.PM_OK
        _check(b.results(), want, f"split instances, {w} warps")
    b.capture()
    for rep in range(2):
        b.occ.fill_(-1)
        b.counts.fill_(-1)
        b.replay()
        assert b.status() == pm.PM_OK
        _check(b.results(), want, f"split instances, graph replay {rep}")
    c = pm.Batch(sets, d_text, off, ln, None)
    c.scan()
    assert c.status() == pm.PM_OK
    for j, ((_, cnt, tot), (wo, wc)) in enumerate(zip(c.results(), want)):
        assert tot == wo.size and np.array_equal(cnt, wc), f"counts-only instance {j}"
    tot = np.array([w[0].size for w in want])
    caps = tot // 3
    s = pm.Batch(sets, d_text, off, ln, caps)
    s.scan()
    assert s.status() == pm.PM_OK
    for j, (o, cnt, t) in enumerate(s.results()):
        assert t == tot[j] and np.array_equal(o, want[j][0][: caps[j]]), f"short capacity instance {j}"
