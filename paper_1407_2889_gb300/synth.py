"""Seeded synthetic inputs: nucleotide texts and pattern sets.

This module only draws bytes; it holds none of the matching arithmetic. Tests,
``bench.py``, ``__graft_entry__.smoke()`` and the oracle's tests all take their
inputs from here, so both sides of every parity check see identical bytes.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast Splittable
Pseudorandom Number Generators", OOPSLA 2014) evaluated at counters: output k
of stream (seed, sid) is ``mix(key + (k + 1) * 0x9E3779B97F4A7C15)``, computed
with wrapping numpy uint64 arithmetic, so any block of a stream can be made
independently and the same bytes come out on every little-endian host.

Workloads (stand-ins for the EST snapshot of the paper's Section 5, which is
not available here):

* :func:`uniform_dna` -- i.i.d. uniform bytes over ``ACGT``.
* :func:`est_text` -- EST-shaped text: sequences of lognormal length
  (median 450, sigma 0.6, clipped to [100, 1200]) separated by ``\\n``; each
  base is ``N`` with probability 164/16384 (about 1 %), else uniform ``ACGT``.
* :func:`sampled_patterns` -- patterns copied from random text windows that
  hold only ``ACGT`` (the paper builds its sets from subsequences of the text).
* :func:`random_patterns` -- i.i.d. uniform ``ACGT`` patterns.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1
ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)

# stream ids: one per purpose, so changing one draw never shifts another
SID_TEXT = 1
SID_LENGTHS = 2
SID_SAMPLE = 3
SID_RANDOM_PAT = 4
SID_MISC = 5

EST_N_THRESHOLD = 164  # out of 2**14: P(N) = 164/16384 = 1.001 %


def _mix_scalar(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(0xBF58476D1CE4E5B9)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, sid: int) -> int:
    return _mix_scalar(_mix_scalar(int(seed) * GOLDEN + 0x632BE59BD9B4E019) ^ (int(sid) * GOLDEN))


def u64(seed: int, sid: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of stream (seed, sid) as uint64."""
    key = np.uint64(stream_key(seed, sid))
    k = np.arange(offset + 1, offset + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + k * np.uint64(GOLDEN))


def uniform01(seed: int, sid: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in (0, 1) from the top 53 bits (never exactly 0)."""
    v = u64(seed, sid, count, offset) >> np.uint64(11)
    return (v.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def uniform_int(seed: int, sid: int, count: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """Integers in [lo, hi] (inclusive) by 64-bit modulo (bias < 2**-30 here)."""
    span = np.uint64(hi - lo + 1)
    return (u64(seed, sid, count, offset) % span).astype(np.int64) + lo


_BLOCK_WORDS = 1 << 20


def uniform_dna(n: int, seed: int, sid: int = SID_TEXT) -> np.ndarray:
    """n i.i.d. uniform bytes over ACGT; 32 bases per 64-bit draw."""
    out = np.empty(n, dtype=np.uint8)
    words_needed = (n + 31) // 32
    pos = 0
    for w0 in range(0, words_needed, _BLOCK_WORDS):
        nw = min(_BLOCK_WORDS, words_needed - w0)
        b = u64(seed, sid, nw, w0).astype("<u8").view(np.uint8)  # 8 bytes per word
        codes = np.empty((b.size, 4), dtype=np.uint8)
        for k in range(4):
            codes[:, k] = (b >> np.uint8(2 * k)) & np.uint8(3)
        chunk = ACGT[codes.reshape(-1)]
        take = min(chunk.size, n - pos)
        out[pos:pos + take] = chunk[:take]
        pos += take
    return out


def est_lengths(total: int, seed: int) -> np.ndarray:
    """Sequence lengths until their sum plus one separator each reaches ``total``.

    Lognormal with median 450 and sigma 0.6 (Box-Muller normal deviates),
    rounded and clipped to [100, 1200].
    """
    lengths = []
    have = 0
    offset = 0
    while have < total:
        batch = max(1024, int((total - have) / 480) + 1024)
        u = uniform01(seed, SID_LENGTHS, 2 * batch, offset)
        offset += 2 * batch
        z = np.sqrt(-2.0 * np.log(u[0::2])) * np.cos(2.0 * math.pi * u[1::2])
        L = np.clip(np.rint(450.0 * np.exp(0.6 * z)), 100, 1200).astype(np.int64)
        cs = np.cumsum(L + 1)
        k = int(np.searchsorted(cs, total - have, side="left"))
        take = min(k + 1, L.size)
        lengths.append(L[:take])
        have += int(cs[take - 1])
    return np.concatenate(lengths)


def est_text(n: int, seed: int) -> np.ndarray:
    """EST-shaped text of exactly n bytes (the last sequence is truncated)."""
    out = np.empty(n, dtype=np.uint8)
    # bases: 16 bits per base -> 2 bits choose ACGT, 14 bits decide N
    words_needed = (n + 3) // 4
    pos = 0
    for w0 in range(0, words_needed, _BLOCK_WORDS):
        nw = min(_BLOCK_WORDS, words_needed - w0)
        v = u64(seed, SID_TEXT, nw, w0).astype("<u8").view("<u2")
        chunk = ACGT[(v & np.uint16(3)).astype(np.uint8)]
        chunk[(v >> np.uint16(2)) < EST_N_THRESHOLD] = ord("N")
        take = min(chunk.size, n - pos)
        out[pos:pos + take] = chunk[:take]
        pos += take
    # separators after each sequence
    L = est_lengths(n, seed)
    sep = np.cumsum(L + 1) - 1
    out[sep[sep < n]] = ord("\n")
    return out


def sampled_patterns(text: np.ndarray, count: int, m: int, seed: int) -> np.ndarray:
    """``count`` windows of length m copied from random starts in [0, n-m] whose
    bytes are all in ACGT (rejection sampling in stream order)."""
    n = text.size
    if count == 0:
        return np.empty((0, m), dtype=np.uint8)
    if n < m:
        raise ValueError("text shorter than m")
    ok_byte = np.zeros(256, dtype=bool)
    ok_byte[ACGT] = True
    rows = []
    got = 0
    offset = 0
    span = np.arange(m, dtype=np.int64)
    while got < count:
        batch = 2 * (count - got) + 64
        starts = uniform_int(seed, SID_SAMPLE, batch, 0, n - m, offset)
        offset += batch
        win = text[starts[:, None] + span[None, :]]
        good = ok_byte[win].all(axis=1)
        acc = win[good][: count - got]
        rows.append(acc)
        got += acc.shape[0]
        if offset > 1000 * count + 100000:
            raise RuntimeError("text has too few ACGT-only windows")
    return np.ascontiguousarray(np.concatenate(rows), dtype=np.uint8)


def random_patterns(count: int, m: int, seed: int) -> np.ndarray:
    """``count`` i.i.d. uniform ACGT patterns of length m."""
    flat = uniform_dna(count * m, seed, SID_RANDOM_PAT)
    return flat.reshape(count, m)


def mixed_patterns(text: np.ndarray, d: int, m: int, seed: int) -> np.ndarray:
    """First d//2 sampled from the text, the remaining d - d//2 random."""
    a = sampled_patterns(text, d // 2, m, seed)
    b = random_patterns(d - d // 2, m, seed)
    return np.ascontiguousarray(np.concatenate([a, b]), dtype=np.uint8)


def mixed_length_patterns(text: np.ndarray, d: int, lmin: int, lmax: int, seed: int) -> list[bytes]:
    """d patterns whose lengths are uniform in [lmin, lmax]; patterns
    0..d//2-1 are ACGT-only windows copied from the text, the rest i.i.d.
    ACGT (each length drawn from its own streams, seed * 1000 + length)."""
    lens = uniform_int(seed, SID_MISC, d, lmin, lmax)
    out: list[bytes] = [b""] * d
    for L in range(lmin, lmax + 1):
        idx = np.nonzero(lens == L)[0]
        k = int((idx < d // 2).sum())
        a = sampled_patterns(text, k, L, seed * 1000 + L)
        b = random_patterns(idx.size - k, L, seed * 1000 + L)
        for j, r in enumerate(idx):
            out[int(r)] = bytes(a[j] if j < k else b[j - k])
    return out


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
SMALL_N = 1 << 20
EST_N = 1 << 30
EST_D = (1000, 8000, 20000)
EST_M = (8, 16, 32)


def small_uniform_case():
    """1 MiB uniform ACGT text (seed 0); d=100, m=8: 50 sampled + 50 random."""
    T = uniform_dna(SMALL_N, 0)
    P = mixed_patterns(T, 100, 8, 0)
    return T, P


def est_pattern_seed(d: int, m: int) -> int:
    return 100 + 10 * EST_D.index(d) + EST_M.index(m)


def est_case(d: int, m: int, n: int = EST_N, text: np.ndarray | None = None):
    """EST-shaped text (seed 1) and a mixed pattern set of d patterns of length m."""
    T = est_text(n, 1) if text is None else text
    P = mixed_patterns(T, d, m, est_pattern_seed(d, m))
    return T, P


def large_set(d: int, text: np.ndarray, m: int = 32):
    """Large pattern set (d = 1e5 -> seed 200, 5e5 -> seed 201) over an EST text."""
    seed = {100000: 200, 500000: 201}.get(d, 202)
    return mixed_patterns(text, d, m, seed)


# ---------------------------------------------------------------------------
# Batched workload: many independent (text, pattern set) instances
# ---------------------------------------------------------------------------
BATCH_K = 4096
BATCH_SEED = 4000
BATCH_N = (1 << 10, 1 << 22)     # text length, log-uniform
BATCH_D = (10, 10000)            # patterns per set, log-uniform
BATCH_M = (8, 64)                # pattern length, uniform integer
BATCH_SAMPLE_SPAN = 1 << 16      # sampled patterns come from this much text


def _log_uniform(u: float, lo: int, hi: int) -> int:
    return int(min(hi, max(lo, round(lo * (hi / lo) ** u))))


def batch_plan(k: int, base_n: int, seed: int = BATCH_SEED, n_range=BATCH_N,
               d_range=BATCH_D, m_range=BATCH_M):
    """Shapes of k instances over one EST-shaped base text of base_n bytes.

    Instance j draws from its own seed (seed + j): a text length log-uniform
    in n_range, a start uniform in [0, base_n - length] rounded down to a
    multiple of 16, d log-uniform in d_range and m uniform in m_range. Texts
    are slices of the base text, so they keep its EST shape and may overlap.
    Returns int64 arrays (off, length, d, m).
    """
    off = np.empty(k, np.int64)
    ln = np.empty(k, np.int64)
    d = np.empty(k, np.int64)
    m = np.empty(k, np.int64)
    for j in range(k):
        u = uniform01(seed + j, SID_MISC, 4)
        ln[j] = min(_log_uniform(float(u[0]), *n_range), base_n)
        off[j] = (int(u[1] * (base_n - ln[j] + 1)) // 16) * 16
        d[j] = _log_uniform(float(u[2]), *d_range)
        m[j] = m_range[0] + min(int(u[3] * (m_range[1] - m_range[0] + 1)), m_range[1] - m_range[0])
    return off, ln, d, m


def batch_patterns(base: np.ndarray, off: int, length: int, d: int, m: int, seed: int) -> np.ndarray:
    """Pattern set of one instance: d//2 windows sampled from the base text
    starting at the instance's slice (at least BATCH_SAMPLE_SPAN bytes of it,
    so that short slices still offer ACGT-only windows), the rest random."""
    span = max(length, BATCH_SAMPLE_SPAN)
    lo = max(0, min(off, base.size - span))
    return mixed_patterns(base[lo:lo + span], d, m, seed)
