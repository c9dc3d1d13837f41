"""Thin ctypes binding over ``libpmscan.so`` (C ABI in ``include/pmscan.h``).

Argument marshalling only: every step of a scan runs in the library's CUDA
kernels. The functions keep the C names (``pm_ac_compile``, ``pm_scan`` ...);
:class:`PatternSet` wraps a handle for convenience. Loading raises
``ImportError`` when the library has not been built -- there is no CPU
fallback.

Device buffers for :func:`pm_scan_device` are plain device pointers; torch
CUDA tensors are accepted wherever a device pointer is expected.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpmscan.so")

PM_OK, PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_ETOOBIG, PM_ETIMEOUT, PM_ECAPACITY, PM_ENODEV = range(8)
PM_HOST_TEXT, PM_DEVICE_TEXT, PM_COUNTS_ONLY = 0, 1, 2
PM_PLACE_AUTO, PM_PLACE_SMEM, PM_PLACE_HYBRID, PM_PLACE_GLOBAL = range(4)
PM_ALGO_AC, PM_ALGO_WM, PM_ALGO_PFAC, PM_ALGO_ACV, PM_ALGO_WMV = 1, 2, 3, 4, 5

EXPORTED = [
    "pm_ac_compile", "pm_pfac_compile", "pm_acv_compile", "pm_wm_compile", "pm_wmv_compile", "pm_set_free", "pm_set_get_info",
    "pm_plan_for_device", "pm_scan",
    "pm_scan_to_host", "pm_result_free", "pm_scan_workspace_bytes", "pm_scan_device",
    "pm_scan_device_noalloc", "pm_noalloc_scratch_bytes", "pm_noalloc_scan_status", "pm_scan_status",
    "pm_scan_batch", "pm_batch_prepare", "pm_batch_free", "pm_batch_counts_total",
    "pm_batch_workspace_bytes", "pm_batch_warps", "pm_batch_scan_device", "pm_batch_tune",
    "pm_batch_set_warps", "pm_batch_set_placement", "pm_batch_placement", "pm_batch_capture", "pm_batch_replay",
    "pm_tune", "pm_server_create", "pm_server_submit", "pm_server_wait", "pm_server_get_stats",
    "pm_server_reset_stats", "pm_server_destroy",
    "pm_selfcheck_host_walk", "pm_strerror", "pm_last_cuda_error", "pm_version",
]


class pm_params(ctypes.Structure):
    _fields_ = [("placement", ctypes.c_int32), ("smem_table_bytes", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("wm_prefix_len", ctypes.c_int32), ("host_only", ctypes.c_int32),
                ("counters", ctypes.c_int32), ("ids_place", ctypes.c_int32),
                ("stride", ctypes.c_int32)]


class pm_plan_info(ctypes.Structure):
    _fields_ = [("placement", ctypes.c_int32), ("warps", ctypes.c_int32), ("warps_list", ctypes.c_int32),
                ("ids_place", ctypes.c_int32), ("counters", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("smem_rows", ctypes.c_int64), ("smem_bytes", ctypes.c_int64), ("smem_bytes_list", ctypes.c_int64)]


class pm_set_info(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("m", ctypes.c_int32), ("d", ctypes.c_int64),
                ("n_distinct", ctypes.c_int64), ("n_states", ctypes.c_int64),
                ("n_rows", ctypes.c_int64), ("n_classes", ctypes.c_int32),
                ("row_width", ctypes.c_int32), ("entry_bytes", ctypes.c_int32),
                ("dna_mode", ctypes.c_int32), ("placement", ctypes.c_int32),
                ("smem_rows", ctypes.c_int64), ("table_bytes", ctypes.c_int64),
                ("B", ctypes.c_int32), ("Bp", ctypes.c_int32),
                ("shift_entries", ctypes.c_int64), ("n_zero_shift", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("m_min", ctypes.c_int32),
                ("max_starts", ctypes.c_int32), ("stride", ctypes.c_int32)]


class pm_result(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int64), ("n_occ", ctypes.c_int64),
                ("counts", ctypes.POINTER(ctypes.c_int64)),
                ("occ", ctypes.POINTER(ctypes.c_uint64))]


class pm_server_params(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("counter_words", ctypes.c_int64),
                ("host_pool_bytes", ctypes.c_int64)]


class pm_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("bytes", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("reruns", ctypes.c_int64), ("peak_inflight", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("arena_used", ctypes.c_int64), ("mean_batch", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("gbs", ctypes.c_double),
                ("dispatch_busy_s", ctypes.c_double), ("complete_busy_s", ctypes.c_double)]


class PmError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib_or_none().pm_strerror(code).decode() if _lib_or_none() else str(code)
        if code == PM_ECUDA and _lib_or_none():
            msg += f" (cudaError {_lib_or_none().pm_last_cuda_error()})"
        super().__init__(f"{what}: {msg}" if what else msg)


_lock = threading.Lock()
_lib = None


def _lib_or_none():
    return _lib


def lib():
    """Load ``libpmscan.so``; ImportError if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        pp = ctypes.POINTER(vp)
        L.pm_ac_compile.restype = ctypes.c_int
        L.pm_ac_compile.argtypes = [vp, i64, i32, ctypes.POINTER(pm_params), pp]
        L.pm_pfac_compile.restype = ctypes.c_int
        L.pm_pfac_compile.argtypes = [vp, i64, i32, ctypes.POINTER(pm_params), pp]
        L.pm_acv_compile.restype = ctypes.c_int
        L.pm_acv_compile.argtypes = [vp, vp, i64, ctypes.POINTER(pm_params), pp]
        L.pm_wmv_compile.restype = ctypes.c_int
        L.pm_wmv_compile.argtypes = [vp, vp, i64, i32, ctypes.POINTER(pm_params), pp]
        L.pm_wm_compile.restype = ctypes.c_int
        L.pm_wm_compile.argtypes = [vp, i64, i32, i32, ctypes.POINTER(pm_params), pp]
        L.pm_set_free.restype = None
        L.pm_set_free.argtypes = [vp]
        L.pm_set_get_info.restype = ctypes.c_int
        L.pm_set_get_info.argtypes = [vp, ctypes.POINTER(pm_set_info)]
        L.pm_plan_for_device.restype = ctypes.c_int
        L.pm_plan_for_device.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(pm_plan_info)]
        L.pm_scan.restype = ctypes.c_int
        L.pm_scan.argtypes = [vp, vp, i64, u32, vp, ctypes.POINTER(ctypes.POINTER(pm_result))]
        L.pm_scan_to_host.restype = ctypes.c_int
        L.pm_scan_to_host.argtypes = [vp, vp, i64, u32, vp, vp, i64, ctypes.POINTER(i64), vp]
        L.pm_result_free.restype = None
        L.pm_result_free.argtypes = [ctypes.POINTER(pm_result)]
        L.pm_scan_workspace_bytes.restype = i64
        L.pm_scan_workspace_bytes.argtypes = [vp, i64, u32]
        L.pm_scan_device.restype = ctypes.c_int
        L.pm_scan_device.argtypes = [vp, vp, i64, u32, vp, vp, i64, vp, vp, i64, vp]
        L.pm_scan_device_noalloc.restype = ctypes.c_int
        L.pm_scan_device_noalloc.argtypes = [vp, vp, i64, u32, vp, vp, i64, vp, vp]
        L.pm_noalloc_scratch_bytes.restype = i64
        L.pm_noalloc_scratch_bytes.argtypes = []
        L.pm_noalloc_scan_status.restype = ctypes.c_int
        L.pm_noalloc_scan_status.argtypes = [vp]
        L.pm_scan_status.restype = ctypes.c_int
        L.pm_scan_status.argtypes = [vp, vp]
        L.pm_scan_batch.restype = ctypes.c_int
        L.pm_scan_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(i64), i32, u32, vp,
                                    ctypes.POINTER(ctypes.POINTER(pm_result))]
        L.pm_batch_prepare.restype = ctypes.c_int
        L.pm_batch_prepare.argtypes = [ctypes.POINTER(vp), i32, vp, vp, vp, u32, pp]
        L.pm_batch_free.restype = None
        L.pm_batch_free.argtypes = [vp]
        L.pm_batch_counts_total.restype = i64
        L.pm_batch_counts_total.argtypes = [vp]
        L.pm_batch_workspace_bytes.restype = i64
        L.pm_batch_workspace_bytes.argtypes = [vp]
        L.pm_batch_warps.restype = i32
        L.pm_batch_warps.argtypes = [vp]
        L.pm_batch_scan_device.restype = ctypes.c_int
        L.pm_batch_scan_device.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
        L.pm_batch_tune.restype = ctypes.c_int
        L.pm_batch_tune.argtypes = [vp, vp, vp, vp, vp, vp, i64, i32, vp, ctypes.POINTER(ctypes.c_float)]
        L.pm_batch_set_warps.restype = ctypes.c_int
        L.pm_batch_set_warps.argtypes = [vp, i32]
        L.pm_batch_set_placement.restype = ctypes.c_int
        L.pm_batch_set_placement.argtypes = [vp, i32]
        L.pm_batch_placement.restype = i32
        L.pm_batch_placement.argtypes = [vp]
        L.pm_batch_capture.restype = ctypes.c_int
        L.pm_batch_capture.argtypes = [vp, vp, vp, vp, vp, vp, i64]
        L.pm_batch_replay.restype = ctypes.c_int
        L.pm_batch_replay.argtypes = [vp, vp]
        L.pm_tune.restype = ctypes.c_int
        L.pm_tune.argtypes = [vp, vp, i64, u32, i32, vp, ctypes.POINTER(pm_params),
                              ctypes.POINTER(ctypes.c_float)]
        L.pm_server_create.restype = ctypes.c_int
        L.pm_server_create.argtypes = [ctypes.POINTER(pm_server_params), pp]
        L.pm_server_submit.restype = ctypes.c_int
        L.pm_server_submit.argtypes = [vp, vp, vp, i64, u32, ctypes.POINTER(i64)]
        L.pm_server_wait.restype = ctypes.c_int
        L.pm_server_wait.argtypes = [vp, i64, ctypes.POINTER(ctypes.POINTER(pm_result))]
        L.pm_server_get_stats.restype = ctypes.c_int
        L.pm_server_get_stats.argtypes = [vp, ctypes.POINTER(pm_server_stats)]
        L.pm_server_reset_stats.restype = ctypes.c_int
        L.pm_server_reset_stats.argtypes = [vp]
        L.pm_server_destroy.restype = None
        L.pm_server_destroy.argtypes = [vp]
        L.pm_selfcheck_host_walk.restype = ctypes.c_int
        L.pm_selfcheck_host_walk.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.POINTER(pm_result))]
        L.pm_strerror.restype = ctypes.c_char_p
        L.pm_strerror.argtypes = [ctypes.c_int]
        L.pm_last_cuda_error.restype = ctypes.c_int
        L.pm_last_cuda_error.argtypes = []
        L.pm_version.restype = ctypes.c_char_p
        L.pm_version.argtypes = []
        _lib = L
        return L


def _check(rc: int, what: str):
    if rc != PM_OK:
        raise PmError(rc, what)


def _dev_ptr(x) -> int:
    """Device pointer of a torch CUDA tensor, or an int address."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError(f"expected a device tensor or address, got {type(x)}")


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


def _patterns(P) -> np.ndarray:
    if isinstance(P, (list, tuple)):
        rows = [np.frombuffer(p.encode() if isinstance(p, str) else bytes(p), dtype=np.uint8) for p in P]
        P = np.stack(rows)
    P = np.ascontiguousarray(P, dtype=np.uint8)
    if P.ndim != 2:
        raise ValueError("patterns must be a (d, m) uint8 array")
    return P


def _make_params(params) -> pm_params | None:
    if params is None:
        return None
    if isinstance(params, pm_params):
        return params
    p = pm_params()
    for k, v in dict(params).items():
        setattr(p, k, int(v))
    return p


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------
def pm_ac_compile(P, params=None) -> int:
    P = _patterns(P)
    h = ctypes.c_void_p()
    prm = _make_params(params)
    _check(lib().pm_ac_compile(P.ctypes.data, P.shape[0], P.shape[1],
                               ctypes.byref(prm) if prm is not None else None, ctypes.byref(h)),
           "pm_ac_compile")
    return h.value


def pm_pfac_compile(P, params=None) -> int:
    P = _patterns(P)
    h = ctypes.c_void_p()
    p = _make_params(params)
    _check(lib().pm_pfac_compile(P.ctypes.data, P.shape[0], P.shape[1],
                                 ctypes.byref(p) if p is not None else None, ctypes.byref(h)),
           "pm_pfac_compile")
    return int(h.value)


def var_patterns(P):
    """A mixed-length set as (concatenated uint8 bytes, int64 offsets[d+1])
    from a list of byte strings, str or uint8 arrays, or such a pair."""
    if isinstance(P, tuple) and len(P) == 2 and isinstance(P[1], np.ndarray):
        cat = np.ascontiguousarray(P[0], dtype=np.uint8)
        off = np.ascontiguousarray(P[1], dtype=np.int64)
        return cat, off
    rows = [np.frombuffer(p.encode() if isinstance(p, str) else bytes(p), dtype=np.uint8)
            if not isinstance(p, np.ndarray) else np.ascontiguousarray(p, dtype=np.uint8).ravel() for p in P]
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    off[1:] = np.cumsum([r.size for r in rows])
    cat = np.ascontiguousarray(np.concatenate(rows)) if rows and off[-1] else np.zeros(1, np.uint8)
    return cat, off


def pm_acv_compile(P, params=None) -> int:
    """Compile a set of patterns of mixed lengths (a list, or (bytes, offsets))."""
    cat, off = var_patterns(P)
    h = ctypes.c_void_p()
    p = _make_params(params)
    _check(lib().pm_acv_compile(cat.ctypes.data, off.ctypes.data, off.size - 1,
                                ctypes.byref(p) if p is not None else None, ctypes.byref(h)),
           "pm_acv_compile")
    return int(h.value)


def pm_wmv_compile(P, B: int, params=None) -> int:
    """Wu-Manber tables for patterns of mixed lengths (a list, or (bytes, offsets))."""
    cat, off = var_patterns(P)
    h = ctypes.c_void_p()
    p = _make_params(params)
    _check(lib().pm_wmv_compile(cat.ctypes.data, off.ctypes.data, off.size - 1, int(B),
                                ctypes.byref(p) if p is not None else None, ctypes.byref(h)),
           "pm_wmv_compile")
    return int(h.value)


def pm_wm_compile(P, B: int, params=None) -> int:
    P = _patterns(P)
    h = ctypes.c_void_p()
    prm = _make_params(params)
    _check(lib().pm_wm_compile(P.ctypes.data, P.shape[0], P.shape[1], int(B),
                               ctypes.byref(prm) if prm is not None else None, ctypes.byref(h)),
           "pm_wm_compile")
    return h.value


def pm_set_free(h: int) -> None:
    if h:
        lib().pm_set_free(h)


def pm_set_get_info(h: int) -> dict:
    info = pm_set_info()
    _check(lib().pm_set_get_info(h, ctypes.byref(info)), "pm_set_get_info")
    return {name: getattr(info, name) for name, _ in info._fields_}


def pm_plan_for_device(h: int, sm_count: int, smem_optin: int, smem_per_sm: int) -> dict:
    out = pm_plan_info()
    _check(lib().pm_plan_for_device(h, sm_count, smem_optin, smem_per_sm, ctypes.byref(out)),
           "pm_plan_for_device")
    return {name: getattr(out, name) for name, _ in out._fields_}


class _ResultOwner:
    """Frees a pm_result once the last array viewing its buffers is gone."""

    __slots__ = ("rp",)

    def __init__(self, rp):
        self.rp = rp

    def __del__(self):
        try:
            lib().pm_result_free(self.rp)
        except Exception:  # interpreter shutdown
            pass


def _view(ptr, n: int, ctype, dtype, owner) -> np.ndarray:
    buf = (ctype * n).from_address(ctypes.addressof(ptr.contents))
    buf._owner = owner
    return np.frombuffer(buf, dtype=dtype)


def _take_result(rp) -> tuple[np.ndarray, np.ndarray]:
    """(occ, counts) arrays viewing the result's buffers, no copy: the
    result is freed when both arrays (and every view of them) are gone."""
    r = rp.contents
    d, n_occ = r.d, r.n_occ
    owner = _ResultOwner(rp)
    counts = _view(r.counts, d, ctypes.c_int64, np.int64, owner) if d > 0 else np.zeros(0, np.int64)
    if r.occ and n_occ > 0:
        occ = _view(r.occ, n_occ, ctypes.c_uint64, np.uint64, owner)
    else:
        occ = np.zeros(0, dtype=np.uint64)
    return occ, counts


def pm_scan(h: int, T, flags: int = PM_HOST_TEXT, stream=None):
    """Scan T (numpy uint8 host array, or a torch CUDA uint8 tensor with
    PM_DEVICE_TEXT). Returns (occ uint64 keys (i<<32)|r, counts int64)."""
    rp = ctypes.POINTER(pm_result)()
    if flags & PM_DEVICE_TEXT:
        ptr, n = _dev_ptr(T), int(T.numel())
    else:
        T = np.ascontiguousarray(T, dtype=np.uint8)
        ptr, n = T.ctypes.data, T.size
    _check(lib().pm_scan(h, ptr, n, flags, _stream_ptr(stream), ctypes.byref(rp)), "pm_scan")
    return _take_result(rp)


def pm_scan_to_host(h: int, T, counts_out, occ_out, flags: int = PM_HOST_TEXT, stream=None) -> int:
    """Scan into caller-owned host arrays (numpy, or pinned torch CPU tensors).
    Returns the total number of occurrences; raises PmError(PM_ECAPACITY) if
    occ_out was too small (its first len(occ_out) keys are still written)."""
    if flags & PM_DEVICE_TEXT:
        ptr, n = _dev_ptr(T), int(T.numel())
    elif hasattr(T, "data_ptr"):
        ptr, n = int(T.data_ptr()), int(T.numel())
    else:
        T = np.ascontiguousarray(T, dtype=np.uint8)
        ptr, n = T.ctypes.data, T.size

    def host_ptr(x):
        if x is None:
            return 0, 0
        if hasattr(x, "data_ptr"):
            return int(x.data_ptr()), int(x.numel())
        return x.ctypes.data, x.size

    cp, _ = host_ptr(counts_out)
    op, cap = host_ptr(occ_out)
    total = ctypes.c_int64(0)
    rc = lib().pm_scan_to_host(h, ptr, n, flags, cp, op, cap, ctypes.byref(total), _stream_ptr(stream))
    _check(rc, "pm_scan_to_host")
    return int(total.value)


def pm_scan_workspace_bytes(h: int, n: int, flags: int = PM_HOST_TEXT) -> int:
    v = lib().pm_scan_workspace_bytes(h, int(n), flags)
    if v < 0:
        raise PmError(PM_EINVAL, "pm_scan_workspace_bytes")
    return int(v)


def pm_scan_device(h: int, d_text, n: int, flags: int, d_counts, d_occ, occ_capacity: int,
                   d_n_occ, d_workspace, workspace_bytes: int, stream=None) -> None:
    _check(lib().pm_scan_device(h, _dev_ptr(d_text), int(n), flags, _dev_ptr(d_counts),
                                _dev_ptr(d_occ), int(occ_capacity), _dev_ptr(d_n_occ),
                                _dev_ptr(d_workspace), int(workspace_bytes), _stream_ptr(stream)),
           "pm_scan_device")


def pm_scan_device_noalloc(h: int, d_text, n: int, flags: int, d_counts, d_occ,
                           occ_capacity: int, d_n_occ, stream=None) -> None:
    """pm_scan_device without a workspace: for callers that cannot allocate
    device memory while scanning (the library's fixed scratch array is used;
    calls that overlap on the GPU race on it)."""
    _check(lib().pm_scan_device_noalloc(h, _dev_ptr(d_text), int(n), flags, _dev_ptr(d_counts),
                                        _dev_ptr(d_occ), int(occ_capacity), _dev_ptr(d_n_occ),
                                        _stream_ptr(stream)),
           "pm_scan_device_noalloc")


def pm_noalloc_scratch_bytes() -> int:
    return int(lib().pm_noalloc_scratch_bytes())


def pm_noalloc_scan_status(stream=None) -> int:
    return int(lib().pm_noalloc_scan_status(_stream_ptr(stream)))


def pm_scan_status(d_workspace, stream=None) -> int:
    return int(lib().pm_scan_status(_dev_ptr(d_workspace), _stream_ptr(stream)))


def pm_scan_batch(handles, texts, flags: int = PM_HOST_TEXT, stream=None):
    k = len(handles)
    hs = (ctypes.c_void_p * k)(*handles)
    keep, ptrs, ns = [], [], []
    for T in texts:
        if flags & PM_DEVICE_TEXT:
            ptrs.append(_dev_ptr(T)); ns.append(int(T.numel()))
        else:
            T = np.ascontiguousarray(T, dtype=np.uint8)
            keep.append(T); ptrs.append(T.ctypes.data); ns.append(T.size)
    tp = (ctypes.c_void_p * k)(*ptrs)
    npv = (ctypes.c_int64 * k)(*ns)
    outs = (ctypes.POINTER(pm_result) * k)()
    _check(lib().pm_scan_batch(hs, tp, npv, k, flags, _stream_ptr(stream), outs), "pm_scan_batch")
    return [_take_result(outs[j]) for j in range(k)]


def pm_tune(h: int, d_text, n: int, flags: int = 0, reps: int = 3, stream=None):
    """Autotune the set's launch plan on a device text; returns (params dict, ms)."""
    p = pm_params()
    ms = ctypes.c_float(0.0)
    _check(lib().pm_tune(h, _dev_ptr(d_text), int(n), flags, int(reps), _stream_ptr(stream),
                         ctypes.byref(p), ctypes.byref(ms)), "pm_tune")
    return {f: getattr(p, f) for f, _ in pm_params._fields_}, float(ms.value)


def pm_batch_prepare(handles, text_off, text_len, occ_off, flags: int = 0) -> int:
    """Prepared batch: instance j scans text_len[j] bytes at text_off[j] of one
    device buffer with set handles[j]; its keys go to occ[occ_off[j]:occ_off[j+1]]."""
    k = len(handles)
    hs = (ctypes.c_void_p * max(k, 1))(*handles)
    to = np.ascontiguousarray(text_off, dtype=np.int64)
    tl = np.ascontiguousarray(text_len, dtype=np.int64)
    oo = np.ascontiguousarray(occ_off, dtype=np.int64)
    if to.size != k or tl.size != k or oo.size != k + 1:
        raise ValueError("text_off and text_len need k entries, occ_off k+1")
    b = ctypes.c_void_p()
    _check(lib().pm_batch_prepare(hs, k, to.ctypes.data, tl.ctypes.data, oo.ctypes.data, flags,
                                  ctypes.byref(b)),
           "pm_batch_prepare")
    return int(b.value)


def pm_batch_free(b: int) -> None:
    if b:
        lib().pm_batch_free(b)


def pm_batch_counts_total(b: int) -> int:
    return int(lib().pm_batch_counts_total(b))


def pm_batch_workspace_bytes(b: int) -> int:
    return int(lib().pm_batch_workspace_bytes(b))


def pm_batch_warps(b: int) -> int:
    return int(lib().pm_batch_warps(b))


def pm_batch_scan_device(b: int, d_text, d_counts, d_occ, d_n_occ, d_workspace,
                         workspace_bytes: int, stream=None) -> None:
    _check(lib().pm_batch_scan_device(b, _dev_ptr(d_text), _dev_ptr(d_counts), _dev_ptr(d_occ),
                                      _dev_ptr(d_n_occ), _dev_ptr(d_workspace), int(workspace_bytes),
                                      _stream_ptr(stream)),
           "pm_batch_scan_device")


def pm_batch_tune(b: int, d_text, d_counts, d_occ, d_n_occ, d_workspace, workspace_bytes: int,
                  reps: int = 3, stream=None) -> float:
    ms = ctypes.c_float(0.0)
    _check(lib().pm_batch_tune(b, _dev_ptr(d_text), _dev_ptr(d_counts), _dev_ptr(d_occ),
                               _dev_ptr(d_n_occ), _dev_ptr(d_workspace), int(workspace_bytes),
                               int(reps), _stream_ptr(stream), ctypes.byref(ms)),
           "pm_batch_tune")
    return float(ms.value)


def pm_batch_set_warps(b: int, warps: int) -> None:
    _check(lib().pm_batch_set_warps(b, int(warps)), "pm_batch_set_warps")


def pm_batch_set_placement(b: int, placement: int) -> None:
    _check(lib().pm_batch_set_placement(b, int(placement)), "pm_batch_set_placement")


def pm_batch_placement(b: int) -> int:
    return int(lib().pm_batch_placement(b))


def pm_batch_capture(b: int, d_text, d_counts, d_occ, d_n_occ, d_workspace,
                     workspace_bytes: int) -> None:
    _check(lib().pm_batch_capture(b, _dev_ptr(d_text), _dev_ptr(d_counts), _dev_ptr(d_occ),
                                  _dev_ptr(d_n_occ), _dev_ptr(d_workspace), int(workspace_bytes)),
           "pm_batch_capture")


def pm_batch_replay(b: int, stream=None) -> None:
    _check(lib().pm_batch_replay(b, _stream_ptr(stream)), "pm_batch_replay")


def pm_selfcheck_host_walk(h: int, T):
    T = np.ascontiguousarray(T, dtype=np.uint8)
    rp = ctypes.POINTER(pm_result)()
    _check(lib().pm_selfcheck_host_walk(h, T.ctypes.data, T.size, ctypes.byref(rp)),
           "pm_selfcheck_host_walk")
    return _take_result(rp)


def pm_version() -> str:
    return lib().pm_version().decode()


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------
class PatternSet:
    """A compiled pattern set (AC DFA or WM tables) owning its device tables."""

    def __init__(self, handle: int, algo: int):
        self.h = handle
        self.algo = algo

    @classmethod
    def ac(cls, P, params=None) -> "PatternSet":
        return cls(pm_ac_compile(P, params), PM_ALGO_AC)

    @classmethod
    def pfac(cls, P, params=None) -> "PatternSet":
        return cls(pm_pfac_compile(P, params), PM_ALGO_PFAC)

    @classmethod
    def wm(cls, P, B: int, params=None) -> "PatternSet":
        return cls(pm_wm_compile(P, B, params), PM_ALGO_WM)

    @classmethod
    def acv(cls, P, params=None) -> "PatternSet":
        """Aho-Corasick over patterns of mixed lengths (list of byte strings)."""
        return cls(pm_acv_compile(P, params), PM_ALGO_ACV)

    @classmethod
    def wmv(cls, P, B: int, params=None) -> "PatternSet":
        """Wu-Manber over patterns of mixed lengths (m = the shortest)."""
        return cls(pm_wmv_compile(P, B, params), PM_ALGO_WMV)

    def info(self) -> dict:
        return pm_set_get_info(self.h)

    def plan_for(self, sm_count: int, smem_optin: int, smem_per_sm: int) -> dict:
        """The planner's launch plan for this AC or PFAC set on a device of the
        given shape (no device needed; works for host-only sets)."""
        return pm_plan_for_device(self.h, sm_count, smem_optin, smem_per_sm)

    def scan(self, T, counts_only: bool = False, stream=None):
        flags = PM_COUNTS_ONLY if counts_only else 0
        if hasattr(T, "is_cuda") and T.is_cuda:
            flags |= PM_DEVICE_TEXT
        return pm_scan(self.h, T, flags, stream)

    def tune(self, d_text, counts_only: bool = False, reps: int = 3, stream=None):
        """Autotune the launch plan on a device text (AC and WM sets); (params, ms)."""
        return pm_tune(self.h, d_text, int(d_text.numel()), PM_COUNTS_ONLY if counts_only else 0,
                       reps, stream)

    def workspace_bytes(self, n: int, counts_only: bool = False) -> int:
        return pm_scan_workspace_bytes(self.h, n, PM_COUNTS_ONLY if counts_only else 0)

    def selfcheck_host_walk(self, T):
        return pm_selfcheck_host_walk(self.h, T)

    def close(self):
        if self.h:
            pm_set_free(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """k Aho-Corasick instances over one device text, scanned in one launch.

    Owns its device result buffers (torch tensors: device memory only).
    ``occ_caps`` gives each instance's key capacity; ``None`` means counts
    only. :meth:`exact` sizes the capacities with a counts-only pass first.
    """

    def __init__(self, sets, d_text, text_off, text_len, occ_caps=None):
        import torch

        self.sets = list(sets)
        self.k = len(self.sets)
        self.d_text = d_text
        self.text_off = np.asarray(text_off, dtype=np.int64)
        self.text_len = np.asarray(text_len, dtype=np.int64)
        self.counts_only = occ_caps is None
        caps = np.zeros(self.k, np.int64) if occ_caps is None else np.asarray(occ_caps, np.int64)
        self.occ_off = np.zeros(self.k + 1, np.int64)
        np.cumsum(caps, out=self.occ_off[1:])
        flags = PM_COUNTS_ONLY if self.counts_only else 0
        self.b = pm_batch_prepare([s.h for s in self.sets], self.text_off, self.text_len,
                                  self.occ_off, flags)
        dev = d_text.device
        self.count_off = np.zeros(self.k + 1, np.int64)
        np.cumsum([s.info()["d"] for s in self.sets], out=self.count_off[1:])
        self.counts = torch.empty(max(1, pm_batch_counts_total(self.b)), dtype=torch.int64, device=dev)
        self.n_occ = torch.empty(max(1, self.k), dtype=torch.int64, device=dev)
        self.occ = torch.empty(max(1, int(self.occ_off[-1])), dtype=torch.int64, device=dev)
        self.ws_bytes = pm_batch_workspace_bytes(self.b)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)

    @classmethod
    def exact(cls, sets, d_text, text_off, text_len, stream=None) -> "Batch":
        """List-mode batch whose capacities are the exact totals (one
        counts-only batched scan, synchronised, sizes them)."""
        import torch

        probe = cls(sets, d_text, text_off, text_len, None)
        probe.scan(stream)
        torch.cuda.synchronize()
        caps = probe.n_occ[: probe.k].cpu().numpy().copy()
        probe.close()
        return cls(sets, d_text, text_off, text_len, caps)

    def _bufs(self):
        return (self.d_text, self.counts, None if self.counts_only else self.occ, self.n_occ, self.ws,
                self.ws_bytes)

    def scan(self, stream=None) -> None:
        pm_batch_scan_device(self.b, *self._bufs(), stream=stream)

    def tune(self, reps: int = 3, stream=None) -> float:
        return pm_batch_tune(self.b, *self._bufs(), reps=reps, stream=stream)

    def set_warps(self, warps: int) -> None:
        pm_batch_set_warps(self.b, warps)

    @property
    def warps(self) -> int:
        return pm_batch_warps(self.b)

    def set_placement(self, placement: int) -> None:
        pm_batch_set_placement(self.b, placement)

    @property
    def placement(self) -> int:
        return pm_batch_placement(self.b)

    def capture(self) -> None:
        pm_batch_capture(self.b, *self._bufs())

    def replay(self, stream=None) -> None:
        pm_batch_replay(self.b, stream)

    def status(self, stream=None) -> int:
        return pm_scan_status(self.ws, stream)

    def results(self):
        """[(occ uint64 array, counts int64 array)] per instance (synchronises)."""
        n_occ = self.n_occ[: self.k].cpu().numpy()
        counts = self.counts.cpu().numpy()
        occ = None if self.counts_only else self.occ.cpu().numpy().view(np.uint64)
        out = []
        for j in range(self.k):
            c = counts[self.count_off[j]:self.count_off[j + 1]].copy()
            if occ is None:
                o = np.empty(0, np.uint64)
            else:
                cap = int(self.occ_off[j + 1] - self.occ_off[j])
                o = occ[self.occ_off[j]:self.occ_off[j] + min(cap, int(n_occ[j]))].copy()
            out.append((o, c, int(n_occ[j])))
        return out

    def close(self):
        if getattr(self, "b", 0):
            pm_batch_free(self.b)
            self.b = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The library's serving loop (pm_server_*): submit host texts against
    device-resident sets, wait for results; continuous batching inside."""

    def __init__(self, budget_bytes: int = 4 << 30, max_batch: int = 512, max_inflight: int = 3,
                 warps: int = 12, counter_words: int = 0, host_pool_bytes: int = 0):
        p = pm_server_params(int(budget_bytes), int(max_batch), int(max_inflight), int(warps), 0,
                             int(counter_words), int(host_pool_bytes))
        h = ctypes.c_void_p()
        _check(lib().pm_server_create(ctypes.byref(p), ctypes.byref(h)), "pm_server_create")
        self.h = int(h.value)
        self._keep = {}
        self._klock = threading.Lock()

    def submit(self, pset, T, counts_only: bool = False) -> int:
        """Queue a scan of host text T (numpy uint8 or CPU tensor, kept alive
        until its wait) against a PatternSet; returns the ticket."""
        if hasattr(T, "data_ptr"):
            ptr, n = int(T.data_ptr()), int(T.numel())
        else:
            T = np.ascontiguousarray(T, dtype=np.uint8)
            ptr, n = T.ctypes.data, T.size
        t = ctypes.c_int64(0)
        _check(lib().pm_server_submit(self.h, pset.h, ptr, n, PM_COUNTS_ONLY if counts_only else 0,
                                      ctypes.byref(t)),
               "pm_server_submit")
        with self._klock:
            self._keep[t.value] = (T, pset)
        return int(t.value)

    def wait(self, ticket: int):
        """(occ uint64 array, counts int64 array) of the request."""
        rp = ctypes.POINTER(pm_result)()
        rc = lib().pm_server_wait(self.h, int(ticket), ctypes.byref(rp))
        with self._klock:
            self._keep.pop(int(ticket), None)
        if rc != PM_OK:
            if rp:
                lib().pm_result_free(rp)
            raise PmError(rc, "pm_server_wait")
        return _take_result(rp)

    def stats(self) -> dict:
        st = pm_server_stats()
        _check(lib().pm_server_get_stats(self.h, ctypes.byref(st)), "pm_server_get_stats")
        return {f: getattr(st, f) for f, _ in pm_server_stats._fields_}

    def reset_stats(self) -> None:
        _check(lib().pm_server_reset_stats(self.h), "pm_server_reset_stats")

    def close(self):
        if getattr(self, "h", 0):
            lib().pm_server_destroy(self.h)
            self.h = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unpack(occ: np.ndarray):
    occ = np.asarray(occ, dtype=np.uint64)
    return (occ >> np.uint64(32)).astype(np.int64), (occ & np.uint64(0xFFFFFFFF)).astype(np.int64)
