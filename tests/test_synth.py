"""The seeded input generators: deterministic, and shaped like the workloads."""
import numpy as np

from paper_1407_2889_gb300 import synth


def test_streams_are_deterministic_and_blockwise():
    a = synth.u64(5, 1, 1000)
    b = synth.u64(5, 1, 600, 400)
    assert np.array_equal(a[400:], b)
    assert not np.array_equal(synth.u64(5, 2, 100), a[:100])
    assert np.array_equal(synth.uniform_dna(12345, 9), synth.uniform_dna(12345, 9))


def test_uniform_dna_composition():
    T = synth.uniform_dna(1 << 20, 0)
    vals, cnt = np.unique(T, return_counts=True)
    assert bytes(vals.tolist()) == b"ACGT"
    assert np.all(np.abs(cnt / T.size - 0.25) < 0.005)


def test_est_text_shape():
    n = 1 << 22
    T = synth.est_text(n, 1)
    assert T.size == n
    assert set(np.unique(T).tolist()) <= set(b"ACGTN\n")
    frac_n = np.mean(T == ord("N"))
    assert 0.008 < frac_n < 0.012
    seps = np.flatnonzero(T == ord("\n"))
    lens = np.diff(np.concatenate([[-1], seps])) - 1
    assert lens.min() >= 100 and lens.max() <= 1200
    assert 400 < np.median(lens) < 500


def test_sampled_patterns_come_from_acgt_windows():
    T = synth.est_text(1 << 18, 1)
    P = synth.sampled_patterns(T, 200, 16, 7)
    assert P.shape == (200, 16)
    assert set(np.unique(P).tolist()) <= set(b"ACGT")
    Ts = T.tobytes()
    assert all(Ts.find(p.tobytes()) >= 0 for p in P)


def test_small_uniform_case_shape():
    T, P = synth.small_uniform_case()
    assert T.size == 1 << 20 and P.shape == (100, 8)


def test_mixed_length_patterns():
    T = synth.est_text(1 << 22, 1)
    P = synth.mixed_length_patterns(T, 500, 8, 16, 301)
    assert P == synth.mixed_length_patterns(T, 500, 8, 16, 301)  # seeded
    assert len(P) == 500 and {len(p) for p in P} <= set(range(8, 17)) and len({len(p) for p in P}) > 5
    assert all(set(p) <= set(b"ACGT") for p in P)
    text = T.tobytes()
    assert all(text.find(p) >= 0 for p in P[:250])  # the first half are windows of the text
