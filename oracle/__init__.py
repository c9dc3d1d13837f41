"""CPU oracle for multiple pattern matching -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package. The product
library never loads it, and it shares no code with the CUDA path.

It answers the question of Section 1 (Definition) of Kouzinopoulos et al.:
every (i, r) with 0 <= i <= n-m and T[i+j] == P[r][j] for all j < m, plus the
per-pattern counts. Four independent routes are offered (see ``pm_oracle.c``):

* :func:`brute` -- the definition as nested loops (tiny inputs);
* :func:`dictionary` -- membership of each window in a sorted dictionary,
  multithreaded (large inputs);
* :func:`ac_search` -- sequential Aho-Corasick, Algorithms 1-3;
* :func:`wm_search` -- sequential Wu-Manber, Algorithms 4-5, paper's hash;
* :func:`brute_var` / :func:`dictionary_var` -- the definition for sets whose
  patterns have their own lengths (each pattern's length in place of m).

Occurrences come back as ``uint64`` keys ``(i << 32) | r`` sorted ascending.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libpmoracle.so")
_lock = threading.Lock()
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (plain C, -O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
           "-pthread", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    vp = ctypes.c_void_p
    lib.orc_brute.restype = i64
    lib.orc_brute.argtypes = [_u8p, i64, _u8p, i64, i32, _u64p, i64, _i64p]
    lib.orc_dict.restype = i64
    lib.orc_dict.argtypes = [_u8p, i64, _u8p, i64, i32, i32, _u64p, i64, _i64p]
    lib.orc_ac_build.restype = vp
    lib.orc_ac_build.argtypes = [_u8p, i64, i32]
    lib.orc_ac_free.argtypes = [vp]
    lib.orc_ac_nstates.restype = i64
    lib.orc_ac_nstates.argtypes = [vp]
    lib.orc_ac_goto.restype = i32
    lib.orc_ac_goto.argtypes = [vp, i64, i32]
    lib.orc_ac_supply.restype = i32
    lib.orc_ac_supply.argtypes = [vp, i64]
    lib.orc_ac_depth.restype = i32
    lib.orc_ac_depth.argtypes = [vp, i64]
    lib.orc_ac_output_first.restype = i64
    lib.orc_ac_output_first.argtypes = [vp, i64]
    lib.orc_ac_output_next.restype = i64
    lib.orc_ac_output_next.argtypes = [vp, i64]
    lib.orc_ac_search.restype = i64
    lib.orc_ac_search.argtypes = [vp, _u8p, i64, _u64p, i64, _i64p]
    lib.orc_wm_build.restype = vp
    lib.orc_wm_build.argtypes = [_u8p, i64, i32, i32, i32]
    lib.orc_wm_free.argtypes = [vp]
    lib.orc_wm_tsize.restype = i64
    lib.orc_wm_tsize.argtypes = [vp]
    lib.orc_wm_shift.restype = i32
    lib.orc_wm_shift.argtypes = [vp, i64]
    lib.orc_wm_prefix.restype = i64
    lib.orc_wm_prefix.argtypes = [vp, i64]
    lib.orc_wm_hash_first.restype = i64
    lib.orc_wm_hash_first.argtypes = [vp, i64]
    lib.orc_wm_hash_next.restype = i64
    lib.orc_wm_hash_next.argtypes = [vp, i64]
    lib.orc_wm_search.restype = i64
    lib.orc_wm_search.argtypes = [vp, _u8p, i64, _u64p, i64, _i64p]
    lib.orc_ac_dfa_scan.restype = i64
    lib.orc_ac_dfa_scan.argtypes = [vp, _u8p, i64, i32, _u64p, i64, _i64p]
    if hasattr(lib, "orc_brute_var"):
        lib.orc_brute_var.restype = i64
        lib.orc_brute_var.argtypes = [_u8p, i64, _u8p, _i64p, i64, _u64p, i64, _i64p]
        lib.orc_dict_var.restype = i64
        lib.orc_dict_var.argtypes = [_u8p, i64, _u8p, _i64p, i64, i32, _u64p, i64, _i64p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def compile_variant(src_text: str, out_dir: str, name: str = "variant"):
    """Compile C source text (e.g. the oracle with a planted mistake) and bind it.

    Used only by the oracle's own mutation tests, which check that the pins
    catch a planted mistake. Returns the bound ``ctypes`` library.
    """
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, "lib" + name + ".so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
                    "-pthread", "-o", so, src], check=True)
    return _bind(ctypes.CDLL(so))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _as_text(T) -> np.ndarray:
    if isinstance(T, (bytes, bytearray, str)):
        T = np.frombuffer(T.encode() if isinstance(T, str) else bytes(T), dtype=np.uint8)
    return np.ascontiguousarray(T, dtype=np.uint8)


def _as_patterns(P) -> np.ndarray:
    """Patterns as a (d, m) uint8 array; accepts a list of equal-length strings."""
    if isinstance(P, (list, tuple)):
        rows = [np.frombuffer(p.encode() if isinstance(p, str) else bytes(p), dtype=np.uint8)
                for p in P]
        if not rows:
            raise ValueError("empty pattern set")
        m = len(rows[0])
        if any(len(r) != m for r in rows):
            raise ValueError("all patterns must have the same length m")
        P = np.stack(rows)
    P = np.ascontiguousarray(P, dtype=np.uint8)
    if P.ndim != 2:
        raise ValueError("patterns must be a (d, m) array")
    return P


def _ptr(a, typ):
    return a.ctypes.data_as(typ)


def _run_two_pass(fn, n_hint: int, d: int):
    """Call ``fn(occ, cap, counts)``; grow ``occ`` once if the guess was short."""
    cap = max(int(n_hint), 16)
    occ = np.empty(cap, dtype=np.uint64)
    counts = np.zeros(d, dtype=np.int64)
    total = fn(occ, cap, counts)
    if total < 0:
        raise MemoryError("oracle ran out of memory")
    if total > cap:
        occ = np.empty(total, dtype=np.uint64)
        total = fn(occ, total, counts)
    return occ[:total].copy(), counts


def brute(T, P, lib=None):
    """Definition of Section 1 as three nested loops. Returns (occ, counts)."""
    lib = lib or _load()
    T, P = _as_text(T), _as_patterns(P)
    d, m = P.shape

    def fn(occ, cap, counts):
        return lib.orc_brute(_ptr(T, _u8p), T.size, _ptr(P, _u8p), d, m,
                             _ptr(occ, _u64p), cap, _ptr(counts, _i64p))

    return _run_two_pass(fn, max(1024, T.size // 8), d)


def dictionary(T, P, threads: int | None = None, lib=None):
    """Same set as :func:`brute`, by sorted-dictionary membership; multithreaded."""
    lib = lib or _load()
    T, P = _as_text(T), _as_patterns(P)
    d, m = P.shape
    if threads is None:
        threads = os.cpu_count() or 1

    def fn(occ, cap, counts):
        return lib.orc_dict(_ptr(T, _u8p), T.size, _ptr(P, _u8p), d, m, int(threads),
                            _ptr(occ, _u64p), cap, _ptr(counts, _i64p))

    return _run_two_pass(fn, max(1024, T.size // 4), d)


def _as_var_patterns(P):
    """A variable-length set as (concatenated bytes, offsets int64[d+1]) from
    a list of byte strings / str / uint8 arrays."""
    rows = [np.frombuffer(p.encode() if isinstance(p, str) else bytes(p), dtype=np.uint8)
            if not isinstance(p, np.ndarray) else np.ascontiguousarray(p, dtype=np.uint8) for p in P]
    if not rows:
        raise ValueError("empty pattern set")
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    off[1:] = np.cumsum([r.size for r in rows])
    cat = np.ascontiguousarray(np.concatenate(rows)) if off[-1] else np.zeros(1, np.uint8)
    return cat, off


def brute_var(T, P, lib=None):
    """The definition for patterns of their own lengths, as loops. Returns (occ, counts)."""
    lib = lib or _load()
    T = _as_text(T)
    cat, off = _as_var_patterns(P)
    d = off.size - 1

    def fn(occ, cap, counts):
        return lib.orc_brute_var(_ptr(T, _u8p), T.size, _ptr(cat, _u8p), _ptr(off, _i64p), d,
                                 _ptr(occ, _u64p), cap, _ptr(counts, _i64p))

    return _run_two_pass(fn, max(1024, T.size // 8), d)


def dictionary_var(T, P, threads: int | None = None, lib=None):
    """Same set as :func:`brute_var`, by dictionary membership per length; multithreaded."""
    lib = lib or _load()
    T = _as_text(T)
    cat, off = _as_var_patterns(P)
    d = off.size - 1
    if threads is None:
        threads = os.cpu_count() or 1

    def fn(occ, cap, counts):
        return lib.orc_dict_var(_ptr(T, _u8p), T.size, _ptr(cat, _u8p), _ptr(off, _i64p), d, int(threads),
                                _ptr(occ, _u64p), cap, _ptr(counts, _i64p))

    return _run_two_pass(fn, max(1024, T.size // 4), d)


class ACAutomaton:
    """Algorithms 1 and 2: goto trie in insertion order plus supply links."""

    def __init__(self, P, lib=None):
        self._lib = lib or _load()
        self.P = _as_patterns(P)
        self.d, self.m = self.P.shape
        self._h = self._lib.orc_ac_build(_ptr(self.P, _u8p), self.d, self.m)
        if not self._h:
            raise ValueError("orc_ac_build failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_ac_free(h)
            self._h = None

    @property
    def nstates(self) -> int:
        return int(self._lib.orc_ac_nstates(self._h))

    def goto(self, q: int, c) -> int:
        """g(q, c) after Algorithm 2; -1 stands for ``fail``."""
        if isinstance(c, str):
            c = ord(c)
        return int(self._lib.orc_ac_goto(self._h, q, c))

    def supply(self, q: int) -> int:
        return int(self._lib.orc_ac_supply(self._h, q))

    def depth(self, q: int) -> int:
        return int(self._lib.orc_ac_depth(self._h, q))

    def output(self, q: int) -> list[int]:
        out, r = [], int(self._lib.orc_ac_output_first(self._h, q))
        while r >= 0:
            out.append(r)
            r = int(self._lib.orc_ac_output_next(self._h, r))
        return out

    def search(self, T):
        """Algorithm 3. Returns (occ, counts)."""
        T = _as_text(T)

        def fn(occ, cap, counts):
            return self._lib.orc_ac_search(self._h, _ptr(T, _u8p), T.size,
                                           _ptr(occ, _u64p), cap, _ptr(counts, _i64p))

        return _run_two_pass(fn, max(1024, T.size // 8), self.d)


class WMTables:
    """Algorithm 4 with the paper's shift-and-add hash (bitshift 2)."""

    def __init__(self, P, B: int, Bp: int = 2, lib=None):
        self._lib = lib or _load()
        self.P = _as_patterns(P)
        self.d, self.m = self.P.shape
        self.B, self.Bp = int(B), int(Bp)
        self._h = self._lib.orc_wm_build(_ptr(self.P, _u8p), self.d, self.m, self.B, self.Bp)
        if not self._h:
            raise ValueError("orc_wm_build failed (need 1 <= B, B' <= m)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_wm_free(h)
            self._h = None

    @property
    def tsize(self) -> int:
        return int(self._lib.orc_wm_tsize(self._h))

    def shift(self, h: int) -> int:
        return int(self._lib.orc_wm_shift(self._h, h))

    def prefix(self, r: int) -> int:
        return int(self._lib.orc_wm_prefix(self._h, r))

    def hash_list(self, h: int) -> list[int]:
        out, r = [], int(self._lib.orc_wm_hash_first(self._h, h))
        while r >= 0:
            out.append(r)
            r = int(self._lib.orc_wm_hash_next(self._h, r))
        return out

    def search(self, T):
        """Algorithm 5. Returns (occ, counts)."""
        T = _as_text(T)

        def fn(occ, cap, counts):
            return self._lib.orc_wm_search(self._h, _ptr(T, _u8p), T.size,
                                           _ptr(occ, _u64p), cap, _ptr(counts, _i64p))

        return _run_two_pass(fn, max(1024, T.size // 8), self.d)


def ac_search(T, P, lib=None):
    """Sequential Aho-Corasick (Algorithms 1-3). Returns (occ, counts)."""
    return ACAutomaton(P, lib=lib).search(T)


def ac_dfa_scan(T, P, threads: int | None = None, automaton=None, lib=None, n_hint: int | None = None):
    """The CPU baseline: Algorithms 1-2's automaton as a full DFA over byte
    classes, walked by ``threads`` host threads over contiguous ranges with
    the m-1 overlap. Returns (occ, counts). Pass ``automaton`` (an
    ACAutomaton of P) to time the scan without the build."""
    T = _as_text(T)
    A = automaton or ACAutomaton(P, lib=lib)
    nt = int(threads or os.cpu_count() or 1)

    def fn(occ, cap, counts):
        return A._lib.orc_ac_dfa_scan(A._h, _ptr(T, _u8p), T.size, nt, _ptr(occ, _u64p), cap,
                                      _ptr(counts, _i64p))

    return _run_two_pass(fn, n_hint if n_hint is not None else max(1024, T.size // 8), A.d)


def wm_search(T, P, B: int, Bp: int = 2, lib=None):
    """Sequential Wu-Manber (Algorithms 4-5). Returns (occ, counts)."""
    P = _as_patterns(P)
    Bp = min(Bp, P.shape[1])
    return WMTables(P, B, Bp, lib=lib).search(T)


def unpack(occ: np.ndarray):
    """Split ``(i << 32) | r`` keys into (i, r) int64 arrays."""
    occ = np.asarray(occ, dtype=np.uint64)
    return (occ >> np.uint64(32)).astype(np.int64), (occ & np.uint64(0xFFFFFFFF)).astype(np.int64)
