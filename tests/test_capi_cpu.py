"""The C-ABI library without a GPU: it loads, exports every symbol the header
declares, rejects bad arguments, refuses to compute without a device, and
its compiled tables (walked on the host by the self-check) give the
oracle's occurrence sets."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1407_2889_gb300 import pmscan as pm
from paper_1407_2889_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST = {"host_only": 1}


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "pmscan.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z_]+)\s*\(", src)))


def test_header_and_exports_agree():
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    L = pm.lib()
    for name in declared:
        assert hasattr(L, name), f"{name} declared but not exported"
    assert sorted(pm.EXPORTED) == declared


def test_version_and_errors():
    assert "sm_103a" in pm.pm_version()
    L = pm.lib()
    for code in range(8):
        assert L.pm_strerror(code)


def test_invalid_arguments():
    with pytest.raises(pm.PmError) as e:
        pm.pm_ac_compile(np.zeros((0, 4), np.uint8), HOST)
    assert e.value.code == pm.PM_EINVAL
    with pytest.raises(pm.PmError) as e:
        pm.pm_ac_compile(np.zeros((3, 0), np.uint8), HOST)
    assert e.value.code == pm.PM_EINVAL
    with pytest.raises(pm.PmError) as e:
        pm.pm_wm_compile(["ACGT"], 5, HOST)
    assert e.value.code == pm.PM_EINVAL
    with pytest.raises(pm.PmError) as e:
        pm.pm_ac_compile(np.zeros((2, 256), np.uint8), HOST)
    assert e.value.code == pm.PM_ETOOBIG
    h = pm.pm_ac_compile(["ACGT"], HOST)
    try:  # a host-only set can be inspected, never scanned
        with pytest.raises(pm.PmError) as e:
            pm.pm_scan(h, np.frombuffer(b"ACGTACGT", np.uint8))
        assert e.value.code == pm.PM_EINVAL
    finally:
        pm.pm_set_free(h)


def test_no_device_no_compute():
    """Without a GPU the library refuses to compile for the device: there is
    no CPU fallback."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present")
    except ImportError:
        pass
    with pytest.raises(pm.PmError) as e:
        pm.pm_ac_compile(["ACGT"])
    assert e.value.code in (pm.PM_ENODEV, pm.PM_ECUDA)


def test_batch_and_server_refuse_without_device():
    """The batched scan and the serving loop are device-only too."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present")
    except ImportError:
        pass
    with pytest.raises(pm.PmError) as e:
        pm.Server(budget_bytes=1 << 20)
    assert e.value.code in (pm.PM_ENODEV, pm.PM_ECUDA)
    h = pm.pm_ac_compile(["ACGTACGT"], HOST)
    try:  # a host-only set is never batched
        with pytest.raises(pm.PmError) as e:
            pm.pm_batch_prepare([h], [0], [16], [0, 4])
        assert e.value.code == pm.PM_EINVAL
    finally:
        pm.pm_set_free(h)


def test_worked_example_tables():
    h = pm.pm_ac_compile(["AAC", "AGT", "GTA"], HOST)
    try:
        info = pm.pm_set_get_info(h)
        # 9 trie states (Section 3.1 example); 3 terminal rows elided; + reset row
        assert info["n_states"] == 9 and info["n_rows"] == 7 and info["n_distinct"] == 3
        assert info["dna_mode"] == 1 and info["row_width"] == 4
        occ, cnt = pm.pm_selfcheck_host_walk(h, np.frombuffer(b"AGTAAC", np.uint8))
        assert [tuple(x) for x in zip(*pm.unpack(occ))] == [(0, 1), (1, 2), (3, 0)]
    finally:
        pm.pm_set_free(h)


def _random_case(rng, alphabet):
    n = int(rng.integers(0, 3000))
    m = int(rng.integers(1, 20))
    d = int(rng.integers(1, 40))
    A = np.frombuffer(alphabet, np.uint8)
    T = A[rng.integers(0, A.size, n)]
    P = A[rng.integers(0, A.size, (d, m))]
    for r in range(d):
        if n >= m and rng.random() < 0.5:
            s = int(rng.integers(0, n - m + 1))
            P[r] = T[s:s + m]
    if d > 2 and rng.random() < 0.5:
        P[-1] = P[0]
    return T, np.ascontiguousarray(P)


@pytest.mark.parametrize("alphabet", [b"ACGT", b"ACGTN\n", b"AC", b"acgt", b"AG", b"xyz", bytes(range(0, 256, 7))])
def test_ac_tables_match_oracle(alphabet):
    rng = np.random.default_rng(len(alphabet) * 31 + alphabet[0])
    for _ in range(40):
        T, P = _random_case(rng, alphabet)
        want_occ, want_cnt = oracle.brute(T, P)
        h = pm.pm_ac_compile(P, HOST)
        try:
            occ, cnt = pm.pm_selfcheck_host_walk(h, T)
        finally:
            pm.pm_set_free(h)
        assert np.array_equal(occ, want_occ) and np.array_equal(cnt, want_cnt)


@pytest.mark.parametrize("alphabet", [b"ACGT", b"ACGTN\n", b"AC", b"xyz", bytes(range(0, 256, 7))])
def test_pfac_tables_match_oracle(alphabet):
    """PFAC keeps only the goto edges of the merged table; a per-position
    walk over them finds exactly the definition's occurrences."""
    rng = np.random.default_rng(len(alphabet) * 53 + alphabet[0])
    for _ in range(40):
        T, P = _random_case(rng, alphabet)
        want_occ, want_cnt = oracle.brute(T, P)
        h = pm.pm_pfac_compile(P, HOST)
        try:
            assert pm.pm_set_get_info(h)["algo"] == pm.PM_ALGO_PFAC
            occ, cnt = pm.pm_selfcheck_host_walk(h, T)
        finally:
            pm.pm_set_free(h)
        assert np.array_equal(occ, want_occ) and np.array_equal(cnt, want_cnt)


@pytest.mark.parametrize("B", [1, 2, 3, 4])
def test_wm_tables_match_oracle(B):
    rng = np.random.default_rng(100 + B)
    for _ in range(40):
        T, P = _random_case(rng, b"ACGTN")
        if P.shape[1] < B:
            continue
        want_occ, want_cnt = oracle.brute(T, P)
        h = pm.pm_wm_compile(P, B, HOST)
        try:
            occ, cnt = pm.pm_selfcheck_host_walk(h, T)
        finally:
            pm.pm_set_free(h)
        assert np.array_equal(occ, want_occ) and np.array_equal(cnt, want_cnt)


@pytest.mark.parametrize("B", [1, 2, 3, 4])
def test_wm_packed_tables_match_oracle(B):
    """ACGT pattern sets (m <= 32) get exact-code WM tables; their host walk
    over texts with bytes outside the alphabet equals the definition."""
    rng = np.random.default_rng(200 + B)
    A = np.frombuffer(b"ACGT", np.uint8)
    checked = 0
    for trial in range(40):
        m = int(rng.integers(max(B, 1), 33))
        d = int(rng.integers(1, 80))
        n = int(rng.integers(0, 6000))
        T = np.frombuffer(b"ACGTN\n", np.uint8)[rng.choice(6, n, p=[.24, .24, .24, .24, .02, .02])]
        P = A[rng.integers(0, 4, (d, m))]
        for r in range(d):
            if n >= m and rng.random() < 0.6:
                s0 = int(rng.integers(0, n - m + 1))
                if all(x in b"ACGT" for x in T[s0:s0 + m].tobytes()):
                    P[r] = T[s0:s0 + m]
        if d > 2:
            P[-1] = P[0]
        P = np.ascontiguousarray(P)
        Bp = 2 if B <= 4 else 1
        h = pm.pm_wm_compile(P, B, {"host_only": 1, "wm_prefix_len": min(Bp, 6 - B)})
        try:
            info = pm.pm_set_get_info(h)
            assert info["dna_mode"] == 1
            occ, cnt = pm.pm_selfcheck_host_walk(h, T)
        finally:
            pm.pm_set_free(h)
        want_occ, want_cnt = oracle.brute(T, P) if n * d <= 200000 else oracle.dictionary(T, P)
        assert np.array_equal(occ, want_occ) and np.array_equal(cnt, want_cnt), (m, d, n)
        checked += 1
    assert checked == 40


def test_table_sizes_of_est_sets():
    """Row counts of the EST-shaped sets decide shared-memory placement."""
    T = synth.est_text(1 << 22, 1)
    P = synth.mixed_patterns(T, 8000, 8, synth.est_pattern_seed(8000, 8))
    h = pm.pm_ac_compile(P, HOST)
    try:
        info = pm.pm_set_get_info(h)
        assert info["entry_bytes"] == 2 and info["n_rows"] < 16384
        assert info["n_distinct"] <= 8000
    finally:
        pm.pm_set_free(h)


def _var_case(rng, alphabet, n_hi=3000, max_len=20):
    A = np.frombuffer(alphabet, np.uint8)
    n = int(rng.integers(0, n_hi))
    T = A[rng.integers(0, A.size, n)]
    if n and rng.random() < 0.5:
        T[rng.integers(0, n, max(1, n // 200))] = ord("\n")
    P = []
    for _ in range(int(rng.integers(1, 60))):
        L = int(rng.integers(1, max_len + 1))
        if n >= L and rng.random() < 0.6:
            s0 = int(rng.integers(0, n - L + 1))
            P.append(bytes(T[s0:s0 + L]))
        else:
            P.append(bytes(A[rng.integers(0, A.size, L)]))
    P.append(P[0][: max(1, len(P[0]) // 2)])   # a prefix of another pattern
    P.append(P[1 % len(P)][-max(1, len(P[1 % len(P)]) // 2):])  # a suffix
    P.append(P[0])                              # a duplicate
    return T, P


def _max_starts(P):
    return max(sum(1 for q in P if p[:len(q)] == q) for p in P)


@pytest.mark.parametrize("alphabet", [b"ACGT", b"ACGTN", b"xyz"])
def test_acv_host_walk_matches_oracle(alphabet):
    """Mixed-length sets: the host walk of the compiled DFA (output sets
    through supply links, every pattern at its own start) equals the
    oracle's definition; info reports the shortest length and the most
    patterns that can start at one position."""
    rng = np.random.default_rng(400 + len(alphabet))
    for case in range(30):
        T, P = _var_case(rng, alphabet)
        want_occ, want_cnt = oracle.dictionary_var(T, P, threads=4)
        h = pm.pm_acv_compile(P, HOST)
        try:
            info = pm.pm_set_get_info(h)
            assert info["algo"] == pm.PM_ALGO_ACV
            assert info["m"] == max(len(p) for p in P) and info["m_min"] == min(len(p) for p in P)
            assert info["max_starts"] == _max_starts(P)
            acgt = set(b"".join(P)) <= set(b"ACGT")
            assert info["dna_mode"] == (1 if acgt else 0)
            occ, cnt = pm.pm_selfcheck_host_walk(h, T)
        finally:
            pm.pm_set_free(h)
        assert np.array_equal(occ, want_occ), f"case {case}"
        assert np.array_equal(cnt, want_cnt), f"case {case}"


def test_acv_long_patterns_and_rejects():
    rng = np.random.default_rng(9)
    T = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 5000)]
    P = [bytes(T[100:165]), bytes(T[100:101]), bytes(T[200:233]), bytes(T[4000:4017])]
    h = pm.pm_acv_compile(P, HOST)
    try:
        occ, cnt = pm.pm_selfcheck_host_walk(h, T)
    finally:
        pm.pm_set_free(h)
    want = oracle.brute_var(T, P)
    assert np.array_equal(occ, want[0]) and np.array_equal(cnt, want[1])
    for bad, code in (([b"ACGT" * 17], pm.PM_ETOOBIG), ((np.zeros(4, np.uint8), np.array([0, 2, 2, 4])), pm.PM_EINVAL)):
        with pytest.raises(pm.PmError) as e:
            pm.pm_acv_compile(bad, HOST)
        assert e.value.code == code


@pytest.mark.parametrize("alphabet", [b"ACGT", b"ACGTN", b"xyz"])
def test_wmv_host_walk_matches_oracle(alphabet):
    """Wu-Manber over mixed lengths (m = the shortest length, every candidate
    verified over its own length): the host walk equals the oracle."""
    rng = np.random.default_rng(700 + len(alphabet))
    for case in range(30):
        T, P = _var_case(rng, alphabet)
        mmin = min(len(p) for p in P)
        want_occ, want_cnt = oracle.dictionary_var(T, P, threads=4)
        for B in sorted({1, min(2, mmin), min(3, mmin)}):
            h = pm.pm_wmv_compile(P, B, HOST)
            try:
                info = pm.pm_set_get_info(h)
                assert info["algo"] == pm.PM_ALGO_WMV and info["m_min"] == mmin
                assert info["m"] == max(len(p) for p in P) and info["max_starts"] == _max_starts(P)
                occ, cnt = pm.pm_selfcheck_host_walk(h, T)
            finally:
                pm.pm_set_free(h)
            assert np.array_equal(occ, want_occ), f"case {case} B={B}"
            assert np.array_equal(cnt, want_cnt), f"case {case} B={B}"
    with pytest.raises(pm.PmError) as e:  # B above the shortest length
        pm.pm_wmv_compile([b"ACGT", b"AC"], 3, HOST)
    assert e.value.code == pm.PM_EINVAL


def test_stride2_host_walk_matches_oracle():
    """Two characters per lookup (ACGT sets of at most 4096 rows, m <= 33):
    bytes outside the alphabet are walked under their class and the matches
    whose window holds one are dropped; the result is the definition's."""
    rng = np.random.default_rng(900)
    A = np.frombuffer(b"ACGT", np.uint8)
    checked = 0
    for case in range(60):
        m = int(rng.choice([1, 2, 3, 5, 8, 9, 16, 17, 24, 33]))
        d = int(rng.integers(1, 120))
        n = int(rng.integers(0, 5000))
        T = np.frombuffer(b"ACGTN\n", np.uint8)[rng.choice(6, n, p=[.235, .235, .235, .235, .04, .02])]
        P = A[rng.integers(0, 4, (d, m))]
        for r in range(d):
            if n >= m and rng.random() < 0.6:
                s0 = int(rng.integers(0, n - m + 1))
                if all(x in b"ACGT" for x in T[s0:s0 + m].tobytes()):
                    P[r] = T[s0:s0 + m]
        if d > 2:
            P[-1] = P[0]
        P = np.ascontiguousarray(P)
        want = oracle.brute(T, P)
        try:
            h = pm.pm_ac_compile(P, {"host_only": 1, "stride": 2})
        except pm.PmError as e:
            assert e.code == pm.PM_ETOOBIG  # more than 4096 rows
            continue
        try:
            occ, cnt = pm.pm_selfcheck_host_walk(h, T)
        finally:
            pm.pm_set_free(h)
        assert np.array_equal(occ, want[0]) and np.array_equal(cnt, want[1]), f"case {case} m={m} n={n}"
        checked += 1
    assert checked >= 40
    with pytest.raises(pm.PmError) as e:  # not an ACGT-like set
        pm.pm_ac_compile([b"ACGN"], {"host_only": 1, "stride": 2})
    assert e.value.code == pm.PM_ETOOBIG
