"""The oracle against facts fixed by the paper and by mathematics (no GPU)."""
import numpy as np
import pytest

import oracle
from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    pin(oracle._load())


def test_routes_agree_on_small_uniform_workload():
    """1 MiB uniform text, d=100, m=8 (50 sampled, 50 random): four routes agree,
    and the invariants that hold at any size hold."""
    from paper_1407_2889_gb300 import synth
    T, P = synth.small_uniform_case()
    T = T[: 1 << 17]  # brute force over 128 KiB keeps this test short
    P = synth.mixed_patterns(T, 100, 8, 0)
    occ_b, cnt_b = oracle.brute(T, P)
    occ_d, cnt_d = oracle.dictionary(T, P, threads=4)
    occ_a, cnt_a = oracle.ac_search(T, P)
    occ_w, cnt_w = oracle.wm_search(T, P, 2)
    for occ, cnt in [(occ_d, cnt_d), (occ_a, cnt_a), (occ_w, cnt_w)]:
        assert np.array_equal(occ, occ_b)
        assert np.array_equal(cnt, cnt_b)
    assert cnt_b.sum() == occ_b.size
    assert np.all(np.diff(occ_b.astype(np.uint64)) > 0)  # strictly sorted by (i, r)
    i, r = oracle.unpack(occ_b)
    win = T[i[:, None] + np.arange(8)[None, :]]
    assert np.array_equal(win, P[r])  # every reported pair is an occurrence
    assert np.all(cnt_b[:50] >= 1)  # each pattern copied from the text occurs


def test_duplicate_patterns_have_equal_counts():
    from paper_1407_2889_gb300 import synth
    T = synth.uniform_dna(1 << 14, 3)
    P = synth.mixed_patterns(T, 40, 5, 3)
    P = np.concatenate([P, P[:10]])
    occ, cnt = oracle.dictionary(T, P, threads=2)
    assert np.array_equal(cnt[:10], cnt[40:50])
    occ_a, cnt_a = oracle.ac_search(T, P)
    assert np.array_equal(occ_a, occ) and np.array_equal(cnt_a, cnt)


def test_concurrent_dictionary_calls_match_sequential_ones():
    """The dictionary routes sort their patterns with the comparison context
    passed as an argument, so calls running at the same time (ctypes drops
    the GIL) each sort by their own patterns."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_1407_2889_gb300 import synth
    T = synth.uniform_dna(1 << 16, 11)
    cases = [synth.mixed_patterns(T, 200 + 37 * k, 6 + (k % 3), 50 + k) for k in range(8)]
    var = [[bytes(p[: 4 + (j % 5)]) for j, p in enumerate(P)] for P in cases]
    want = [oracle.dictionary(T, P, threads=2) for P in cases]
    want_v = [oracle.dictionary_var(T, P, threads=2) for P in var]
    with ThreadPoolExecutor(max_workers=8) as ex:
        got = list(ex.map(lambda P: oracle.dictionary(T, P, threads=2), cases))
        got_v = list(ex.map(lambda P: oracle.dictionary_var(T, P, threads=2), var))
    for (wo, wc), (go, gc) in zip(want + want_v, got + got_v):
        assert np.array_equal(wo, go) and np.array_equal(wc, gc)


@pytest.mark.parametrize("threads", [1, 3, 7])
def test_cpu_dfa_baseline_equals_the_definition(threads):
    """The multithreaded CPU DFA scan (the timed baseline) reports exactly the
    definition's set, whatever the split: ranges cut mid-match, texts with
    bytes in no pattern, duplicate patterns, and runs of one letter."""
    from paper_1407_2889_gb300 import synth
    T = synth.est_text(1 << 16, 13)
    T = np.concatenate([T, np.full(500, ord("A"), np.uint8), T[:333]])
    P = synth.mixed_patterns(T, 150, 7, 13)
    P = np.concatenate([P, P[:5], np.full((1, 7), ord("A"), np.uint8)])
    want = oracle.brute(T, P)
    got = oracle.ac_dfa_scan(T, P, threads=threads)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    short = T[:5]
    assert oracle.ac_dfa_scan(short, P, threads=threads)[0].size == 0
