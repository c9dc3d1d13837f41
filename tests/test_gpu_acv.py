"""GPU parity of the mixed-length scans: Aho-Corasick (pm_acv_compile) and
Wu-Manber with m = the shortest length (pm_wmv_compile).

Every result must equal, bit for bit, the oracle's definition with each
pattern's own length: random sets over several alphabets (prefixes,
suffixes and duplicates of one another), an EST-shaped text, edge sizes, a
text where every position starts many patterns (pool overflow and the
in-place sort of large tiles), short output capacity, and a set of more
than 2^20 patterns (8-byte slot entries).
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


def _same(got, want, what=""):
    assert got[0].size == want[0].size, f"{what}: {got[0].size} occurrences, oracle {want[0].size}"
    assert np.array_equal(got[0], want[0]), f"{what}: occurrences differ"
    assert np.array_equal(got[1], want[1]), f"{what}: counts differ"


def _case(rng, alphabet, n_hi, max_len, d_hi=80):
    A = np.frombuffer(alphabet, np.uint8)
    n = int(rng.integers(0, n_hi))
    T = A[rng.integers(0, A.size, n)]
    P = []
    for _ in range(int(rng.integers(1, d_hi))):
        L = int(rng.integers(1, max_len + 1))
        if n >= L and rng.random() < 0.6:
            s0 = int(rng.integers(0, n - L + 1))
            P.append(bytes(T[s0:s0 + L]))
        else:
            P.append(bytes(A[rng.integers(0, A.size, L)]))
    P.append(P[0][: max(1, len(P[0]) // 2)])
    P.append(P[-2][-max(1, len(P[-2]) // 2):])
    P.append(P[0])
    return T, P


@pytest.mark.parametrize("alphabet,max_len", [(b"ACGT", 16), (b"ACGT", 40), (b"ACGT", 65), (b"ACGTN", 12),
                                              (b"ab", 20)])
def test_acv_random_sets(alphabet, max_len):
    rng = np.random.default_rng(500 + max_len + len(alphabet))
    for case in range(12):
        T, P = _case(rng, alphabet, 200000, max_len)
        want = oracle.dictionary_var(T, P, threads=THREADS)
        s = pm.PatternSet.acv(P)
        _same(s.scan(T), want, f"case {case}")
        _same(s.scan(torch.from_numpy(T).cuda()), want, f"case {case} device text")
        _, cnt = s.scan(T, counts_only=True)
        assert np.array_equal(cnt, want[1])
        s.close()


def test_acv_est_text():
    T = synth.est_text(16 << 20, 1)
    rng = np.random.default_rng(21)
    P = []
    for r in range(3000):
        L = int(rng.integers(6, 25))
        if r % 2 == 0:
            while True:
                s0 = int(rng.integers(0, T.size - L))
                w = bytes(T[s0:s0 + L])
                if set(w) <= set(b"ACGT"):
                    break
            P.append(w)
        else:
            P.append(bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, L)]))
    want = oracle.dictionary_var(T, P, threads=THREADS)
    s = pm.PatternSet.acv(P)
    assert s.info()["dna_mode"] == 1
    _same(s.scan(torch.from_numpy(T).cuda()), want, "EST 16 MiB")
    s.close()


def test_acv_edges():
    P = [b"ACGTACGT", b"A", b"GTA", b"ACGTACGTACGTACGTACG"]
    s = pm.PatternSet.acv(P)
    for n in [0, 1, 2, 7, 8, 9, 80, 2559, 2560, 2561, 2567, 5120 + 3, 100003]:
        T = synth.uniform_dna(n, 13)
        want = oracle.brute_var(T, P) if n < 6000 else oracle.dictionary_var(T, P, threads=THREADS)
        _same(s.scan(T), want, f"n={n}")
    # unaligned device text
    T = synth.uniform_dna(300001, 14)
    d_T = torch.from_numpy(T).cuda()
    for off in (1, 3, 7):
        _same(s.scan(d_T[off:]), oracle.dictionary_var(T[off:], P, threads=THREADS), f"offset {off}")
    s.close()


def test_acv_many_patterns_per_position_overflow():
    """A^n against A^1..A^12 (and a duplicate): every position starts 13
    patterns, so lanes overflow their pools and tiles exceed the staged sort."""
    T = np.full(60000, ord("A"), np.uint8)
    T[31337] = ord("C")
    P = [b"A" * L for L in range(1, 13)] + [b"AAAA", b"CAAA"]
    want = oracle.dictionary_var(T, P, threads=THREADS)
    s = pm.PatternSet.acv(P)
    assert s.info()["max_starts"] == 13
    _same(s.scan(T), want, "all-A")
    _, cnt = s.scan(T, counts_only=True)
    assert np.array_equal(cnt, want[1])
    s.close()


def test_acv_capacity_short_and_device_api():
    rng = np.random.default_rng(8)
    T, P = _case(rng, b"ACGT", 400000, 10, d_hi=200)
    want = oracle.dictionary_var(T, P, threads=THREADS)
    s = pm.PatternSet.acv(P)
    n = T.size
    d_T = torch.from_numpy(T).cuda()
    ws = torch.zeros(s.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    counts = torch.zeros(len(P), dtype=torch.int64, device="cuda")
    nocc = torch.zeros(1, dtype=torch.int64, device="cuda")
    cap = max(1, want[0].size // 2)
    occ = torch.zeros(cap, dtype=torch.int64, device="cuda")
    st = torch.cuda.Stream()
    pm.pm_scan_device(s.h, d_T, n, 0, counts, occ, cap, nocc, ws, ws.numel(), st)
    assert pm.pm_scan_status(ws, st) == pm.PM_OK
    assert int(nocc.item()) == want[0].size
    assert np.array_equal(occ.cpu().numpy().view(np.uint64), want[0][:cap])
    assert np.array_equal(counts.cpu().numpy(), want[1])
    s.close()


def test_acv_more_than_2_20_patterns():
    """d > 2^20: slot entries take 8 bytes."""
    rng = np.random.default_rng(31)
    T = synth.uniform_dna(1 << 20, 15)
    d = (1 << 20) + 1000
    A = np.frombuffer(b"ACGT", np.uint8)
    lens = rng.integers(12, 14, d)
    P = [bytes(A[rng.integers(0, 4, int(L))]) for L in lens]
    for r in range(0, d, 7):  # some copied from the text
        s0 = int(rng.integers(0, T.size - 14))
        P[r] = bytes(T[s0:s0 + int(lens[r])])
    want = oracle.dictionary_var(T, P, threads=THREADS)
    s = pm.PatternSet.acv(P)
    _same(s.scan(T), want, "d > 2^20")
    s.close()


@pytest.mark.parametrize("alphabet,lo,hi,B", [(b"ACGT", 4, 16, 3), (b"ACGT", 8, 40, 3), (b"ACGTN", 3, 12, 2),
                                              (b"ab", 2, 20, 1)])
def test_wmv_random_sets(alphabet, lo, hi, B):
    rng = np.random.default_rng(800 + hi + B)
    A = np.frombuffer(alphabet, np.uint8)
    for case in range(10):
        n = int(rng.integers(0, 200000))
        T = A[rng.integers(0, A.size, n)]
        P = []
        for _ in range(int(rng.integers(1, 120))):
            L = int(rng.integers(lo, hi + 1))
            if n >= L and rng.random() < 0.6:
                s0 = int(rng.integers(0, n - L + 1))
                P.append(bytes(T[s0:s0 + L]))
            else:
                P.append(bytes(A[rng.integers(0, A.size, L)]))
        P.append(P[0][: max(lo, len(P[0]) - 2)])
        P.append(P[0])
        want = oracle.dictionary_var(T, P, threads=THREADS)
        s = pm.PatternSet.wmv(P, B)
        _same(s.scan(T), want, f"case {case}")
        _, cnt = s.scan(T, counts_only=True)
        assert np.array_equal(cnt, want[1])
        s.close()


def test_wmv_est_text_and_overflow():
    T = synth.est_text(16 << 20, 1)
    P = synth.mixed_length_patterns(T, 2000, 8, 24, 311)
    want = oracle.dictionary_var(T, P, threads=THREADS)
    s = pm.PatternSet.wmv(P, 3)
    _same(s.scan(torch.from_numpy(T).cuda()), want, "EST 16 MiB")
    s.close()
    A = np.full(60000, ord("A"), np.uint8)
    A[4242] = ord("C")
    Pa = [b"A" * L for L in range(2, 13)] + [b"AAAA", b"CAAA"]
    s = pm.PatternSet.wmv(Pa, 2)
    assert s.info()["max_starts"] == 12
    _same(s.scan(A), oracle.dictionary_var(A, Pa, threads=THREADS), "all-A")
    s.close()
