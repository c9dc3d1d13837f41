"""Pins for the CPU oracle: facts fixed by the paper and by mathematics.

Each ``pin_*`` takes a bound oracle library (the real one, or a copy with a
planted mistake) and raises ``AssertionError`` if the oracle disagrees with:

* the worked example of Section 3.1 (Figure 1: AAC, AGT, GTA) -- printed facts
  plus the states and supply links worked by hand from Algorithms 1-2;
* the Wu-Manber tables of Algorithm 4 worked by hand (Section 3.2 hash);
* closed forms: a single run of one letter, de Bruijn texts, m = 1, n < m;
* Python's ``re`` engine (overlapping lookahead search), a library routine
  that enumerates occurrences independently of every route here;
* for sets whose patterns have their own lengths: a hand-worked example,
  runs of one letter, a de Bruijn text, the regex engine, and agreement with
  the fixed-length routes when all lengths are equal.

``tests/test_oracle_pins.py`` runs them on the oracle; ``tests/test_oracle_mutants.py``
plants mistakes in a copy of the oracle and checks that some pin fails.
"""
from __future__ import annotations

import json
import os
import re

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _pairs(occ):
    i, r = oracle.unpack(occ)
    return list(zip(i.tolist(), r.tolist()))


def _all_routes(T, P, lib, B=None):
    """(name, occ, counts) from every oracle route on the same input."""
    P = oracle._as_patterns(P)
    m = P.shape[1]
    out = [("brute",) + oracle.brute(T, P, lib=lib),
           ("dict1",) + oracle.dictionary(T, P, threads=1, lib=lib),
           ("dict3",) + oracle.dictionary(T, P, threads=3, lib=lib),
           ("ac",) + oracle.ac_search(T, P, lib=lib),
           ("dfa1",) + oracle.ac_dfa_scan(T, P, threads=1, lib=lib),
           ("dfa3",) + oracle.ac_dfa_scan(T, P, threads=3, lib=lib)]
    for b in ([B] if B else sorted({1, min(2, m), min(3, m)})):
        out.append((f"wm{b}",) + oracle.wm_search(T, P, b, min(2, m), lib=lib))
    return out


def _regex_matches(T: bytes, P):
    """Occurrences enumerated by Python's regex engine (zero-width lookahead)."""
    res = []
    for r, p in enumerate(P):
        for mo in re.finditer(b"(?=" + re.escape(bytes(p)) + b")", T):
            res.append((mo.start(), r))
    return sorted(res)


def _check_against(expected_pairs, T, P, lib, B=None):
    d = len(P)
    exp_counts = np.zeros(d, dtype=np.int64)
    for _, r in expected_pairs:
        exp_counts[r] += 1
    for name, occ, counts in _all_routes(T, P, lib, B):
        got = _pairs(occ)
        assert got == expected_pairs, f"{name}: occurrences differ ({len(got)} vs {len(expected_pairs)})"
        assert np.array_equal(counts, exp_counts), f"{name}: per-pattern counts differ"


# ---------------------------------------------------------------------------
def pin_ac_worked_example(lib):
    g = _golden("ac_worked_example.json")
    ac = oracle.ACAutomaton(g["patterns"], lib=lib)
    for q, c, v in g["printed_facts"]["goto"]:
        assert ac.goto(q, c) == v, f"printed fact g({q},{c})={v}"
    for q, v in g["printed_facts"]["supply"]:
        assert ac.supply(q) == v, f"printed fact Supply({q})={v}"
    h = g["derived_by_hand"]
    assert ac.nstates == len(h["labels"])
    for q, c, v in h["trie_edges"]:
        assert ac.goto(q, c) == v, f"trie edge g({q},{c})={v}"
    for q, label in h["labels"].items():
        assert ac.depth(int(q)) == len(label)
    for q, v in h["supply"].items():
        assert ac.supply(int(q)) == v, f"Supply({q})={v}"
    for q in range(ac.nstates):
        assert ac.output(q) == h["output"].get(str(q), []), f"Output({q})"
    # after Algorithm 2 the root loops on every other byte; deeper misses stay fail
    assert ac.goto(0, "T") == 0 and ac.goto(0, "C") == 0 and ac.goto(0, "N") == 0
    assert ac.goto(1, "T") == -1 and ac.goto(3, "A") == -1
    occ, _ = ac.search(h["text"])
    assert _pairs(occ) == [tuple(x) for x in h["matches_i_r"]]
    _check_against([tuple(x) for x in h["matches_i_r"]], h["text"].encode(),
                   [p.encode() for p in g["patterns"]], lib)


def pin_wm_tables_example(lib):
    g = _golden("wm_tables_example.json")
    w = oracle.WMTables(g["patterns"], g["B"], g["Bp"], lib=lib)
    assert w.tsize == g["table_size"]
    for h in range(w.tsize):
        want = g["shift"].get(str(h), g["shift_default"])
        assert w.shift(h) == want, f"SHIFT[{h}] = {w.shift(h)}, hand value {want}"
        assert w.hash_list(h) == g["hash_lists"].get(str(h), []), f"HASH[{h}]"
    for r, v in enumerate(g["prefix"]):
        assert w.prefix(r) == v, f"PREFIX[{r}]"
    w3 = oracle.WMTables(["ACGT"], 3, 2, lib=lib)
    assert w3.shift(g["three_char_hash"]["ACG"]) == 1  # block ACG ends one before the end
    assert w3.shift(g["three_char_hash"]["ACG"] + 1) == 2  # never-seen value keeps m-B+1
    occ, _ = w.search(g["text"])
    assert _pairs(occ) == [tuple(x) for x in g["matches_i_r"]]
    _check_against([tuple(x) for x in g["matches_i_r"]], g["text"].encode(),
                   [p.encode() for p in g["patterns"]], lib)


def pin_single_letter_run(lib):
    # a^m occurs at every start of a^n: n - m + 1 times (two copies -> each r)
    for n, m in [(1, 1), (5, 5), (17, 3), (64, 8), (40, 12)]:
        T = b"A" * n
        P = [b"A" * m, b"C" * m, b"A" * m]
        exp = sorted([(i, 0) for i in range(n - m + 1)] + [(i, 2) for i in range(n - m + 1)])
        _check_against(exp, T, P, lib)


def _de_bruijn(k: int, m: int) -> list[int]:
    """Textbook de Bruijn sequence B(k, m) by concatenating Lyndon words (FKM)."""
    a = [0] * (k * m)
    seq: list[int] = []

    def db(t, p):
        if t > m:
            if m % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, k):
                a[t] = j
                db(t + 1, t)

    db(1, 1)
    return seq


def pin_de_bruijn(lib):
    # a linearised de Bruijn text holds every m-mer exactly once
    for m in (2, 3, 4):
        s = _de_bruijn(4, m)
        s = s + s[: m - 1]
        T = bytes(b"ACGT"[c] for c in s)
        assert len(T) == 4 ** m + m - 1
        P = [bytes(b"ACGT"[(x >> (2 * (m - 1 - j))) & 3] for j in range(m)) for x in range(4 ** m)]
        for name, occ, counts in _all_routes(T, P, lib):
            assert np.all(counts == 1), f"{name}: every m-mer exactly once"
            i, r = oracle.unpack(occ)
            assert sorted(i.tolist()) == list(range(4 ** m)), f"{name}: one m-mer per start"
            for ii, rr in zip(i.tolist(), r.tolist()):
                assert T[ii:ii + m] == P[rr], f"{name}: wrong pattern at {ii}"


def pin_degenerate_sizes(lib):
    _check_against([], b"ACG", [b"ACGT"], lib)          # n < m
    _check_against([(0, 0)], b"ACGT", [b"ACGT"], lib)   # n == m
    _check_against([], b"ACGTACGT", [b"TTTT"], lib)     # absent pattern
    T = b"GATTACA"                                      # m = 1
    exp = sorted([(i, 0) for i, c in enumerate(T) if c == ord("A")] +
                 [(i, 1) for i, c in enumerate(T) if c == ord("T")])
    _check_against(exp, T, [b"A", b"T"], lib)


def pin_regex_random(lib, cases: int = 60, seed: int = 7):
    rng = np.random.default_rng(seed)
    for case in range(cases):
        k = int(rng.integers(1, 5))
        alphabet = b"ACGTN\n"[: k + 1]
        n = int(rng.integers(0, 400))
        m = int(rng.integers(1, 9))
        d = int(rng.integers(1, 12))
        T = bytes(alphabet[j] for j in rng.integers(0, len(alphabet), n))
        P = []
        for _ in range(d):
            if n >= m and rng.random() < 0.5:
                s = int(rng.integers(0, n - m + 1))
                P.append(T[s:s + m])
            else:
                P.append(bytes(alphabet[j] for j in rng.integers(0, len(alphabet), m)))
        if rng.random() < 0.3:
            P.append(P[0])  # duplicate pattern
        exp = _regex_matches(T, P)
        _check_against(exp, T, P, lib)


def pin_periodic(lib):
    T = b"AC" * 50
    _check_against([(i, 0) for i in range(0, 97, 2)], T, [b"ACAC"], lib)
    T = b"AAC" * 20
    P = [b"AACA", b"ACAA", b"CAAC", b"AAAA"]
    _check_against(_regex_matches(T, P), T, P, lib)


# ---------------------------------------------------------------------------
# Sets whose patterns have their own lengths (the definition with len_r for m)
def _var_routes(T, P, lib):
    yield ("brute_var",) + tuple(oracle.brute_var(T, P, lib=lib))
    yield ("dictionary_var",) + tuple(oracle.dictionary_var(T, P, threads=3, lib=lib))


def _check_var(expected_pairs, T, P, lib):
    exp_counts = np.zeros(len(P), dtype=np.int64)
    for _, r in expected_pairs:
        exp_counts[r] += 1
    for name, occ, counts in _var_routes(T, P, lib):
        got = _pairs(occ)
        assert got == expected_pairs, f"{name}: occurrences differ ({len(got)} vs {len(expected_pairs)})"
        assert np.array_equal(counts, exp_counts), f"{name}: per-pattern counts differ"


def pin_var_hand_example(lib):
    # AAAAAC against A, AA, AAC, C, AC, worked by hand from the definition:
    # A at 0-4, AA at 0-3, AAC at 3, C at 5, AC at 4
    exp = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1), (3, 2),
           (4, 0), (4, 4), (5, 3)]
    _check_var(exp, b"AAAAAC", [b"A", b"AA", b"AAC", b"C", b"AC"], lib)


def pin_var_letter_runs(lib):
    # A^L occurs n-L+1 times in A^n (none when L > n); runs of C never
    for n in (1, 5, 17, 64):
        P = [b"A" * L for L in (1, 2, 3, 5, 8, 13)] + [b"CC", b"AAA"]
        exp = sorted((i, r) for r, p in enumerate(P) if p[:1] == b"A" for i in range(n - len(p) + 1))
        _check_var(exp, b"A" * n, P, lib)


def pin_var_de_bruijn(lib):
    # linearised de Bruijn text of order k (length 4^k + k - 1): every k-mer
    # once; every L-mer 4^(k-L) times cyclically, plus at most k-L of the
    # wrapped windows; the L-mers together fill all n - L + 1 windows
    k = 4
    s = _de_bruijn(4, k)
    T = bytes(b"ACGT"[c] for c in s + s[: k - 1])
    n = len(T)
    mers = {L: [bytes(b"ACGT"[(x >> (2 * (L - 1 - j))) & 3] for j in range(L)) for x in range(4 ** L)]
            for L in (1, 2, k)}
    P = mers[k] + mers[1] + mers[2]
    for name, occ, counts in _var_routes(T, P, lib):
        off = 0
        for L in (k, 1, 2):
            c = counts[off:off + 4 ** L]
            assert int(c.sum()) == n - L + 1, f"{name}: the {L}-mers fill every window"
            assert np.all(c >= 4 ** (k - L)) and np.all(c <= 4 ** (k - L) + (k - L)), f"{name}: {L}-mer counts"
            off += 4 ** L
        i, r = oracle.unpack(occ)
        for ii, rr in zip(i.tolist(), r.tolist()):
            assert T[ii:ii + len(P[rr])] == P[rr], f"{name}: wrong pattern at {ii}"


def pin_var_regex_random(lib, cases: int = 60, seed: int = 11):
    # mixed lengths, prefixes of one another, duplicates: Python's regex engine
    rng = np.random.default_rng(seed)
    for case in range(cases):
        alphabet = b"ACGTN"[: int(rng.integers(2, 6))]
        n = int(rng.integers(0, 300))
        T = bytes(alphabet[j] for j in rng.integers(0, len(alphabet), n))
        P = []
        for _ in range(int(rng.integers(1, 14))):
            L = int(rng.integers(1, 10))
            if n >= L and rng.random() < 0.5:
                s0 = int(rng.integers(0, n - L + 1))
                P.append(T[s0:s0 + L])
            else:
                P.append(bytes(alphabet[j] for j in rng.integers(0, len(alphabet), L)))
        if len(P) > 1 and rng.random() < 0.5:
            P.append(P[0][: max(1, len(P[0]) - 1)])  # a prefix of another pattern
        if rng.random() < 0.3:
            P.append(P[-1])  # a duplicate
        _check_var(_regex_matches(T, P), T, P, lib)


def pin_var_equal_lengths(lib):
    # with one length for all patterns the set is that of the fixed-length routes
    rng = np.random.default_rng(5)
    for case in range(20):
        m = int(rng.integers(1, 9))
        T = bytes(b"ACG"[j] for j in rng.integers(0, 3, int(rng.integers(0, 500))))
        P = [bytes(b"ACG"[j] for j in rng.integers(0, 3, m)) for _ in range(int(rng.integers(1, 10)))]
        want = oracle.brute(T, P, lib=lib)
        for name, occ, counts in _var_routes(T, P, lib):
            assert np.array_equal(occ, want[0]) and np.array_equal(counts, want[1]), name


ALL_PINS = [pin_ac_worked_example, pin_wm_tables_example, pin_single_letter_run,
            pin_de_bruijn, pin_degenerate_sizes, pin_regex_random, pin_periodic,
            pin_var_hand_example, pin_var_letter_runs, pin_var_de_bruijn, pin_var_regex_random,
            pin_var_equal_lengths]


def run_all(lib) -> list[str]:
    """Names of the pins that fail for ``lib`` (empty list: all hold)."""
    failed = []
    for pin in ALL_PINS:
        try:
            pin(lib)
        except AssertionError as e:
            failed.append(f"{pin.__name__}: {e}")
    return failed
