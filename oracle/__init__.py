"""QuickMergesort oracle: ctypes binding of the single-threaded C++ reference.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares nothing
with the CUDA library (no headers, helpers or constants) and never imports it.

Paper: Edelkamp & Weiss, "QuickMergesort: Practically Efficient Constant-Factor
Optimal Sorting" (arXiv 1804.10062).  ``qms_ref.cpp`` cites the sections each
function follows (QuickXsort skeleton Sec. 2, Fig. 3 listing Sec. 3, MoM and
hybrid variants Sec. 4, comparison counter Sec. 5).

Parity status: every exported function is pinned by the ``-m "not gpu"``
tests (exhaustive permutations against the exact-average recurrence derived
from the proof of Thm. 1, duplicates, Mergesort closed forms, the Cor. 1 band,
the worst-case bound of Sec. 4, the Fig. 1 worked example and a library sort;
for the median-of-medians machinery of Sec. 4: the median of five on every
permutation and tied word, the selection against the order statistic and the
BFPRT discard bound (tight on a constructed input), the 2 floor(n/6) pivot
rank of every MoM round, the 2n/3 partition, the hybrid's switching rule;
for the move counter, closed forms of Fig. 3's moves on reverse input; for
the four-way swap-merge Mergesort of Sec. 6's future work: every small
permutation, buffer preservation, comparisons equal to an independent
two-level merge sort, an exact move recurrence and the lg(n!) average
bound).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libqms_oracle.so")
_SRC = os.path.join(_HERE, "qms_ref.cpp")
_lock = threading.Lock()
_lib = None

DTYPES = {"u32": 0, "u64": 1, "i64": 2, "f32": 3}
NP_DTYPES = {"u32": np.uint32, "u64": np.uint64, "i64": np.int64, "f32": np.float32}
VARIANTS = {"m3": 0, "sqrtn": 1, "mom": 2, "hybrid": 3}
MODES = {"analysis": 0, "paper": 1}


def build(force: bool = False) -> str:
    """Compiles qms_ref.cpp into a shared library (plain g++, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                           _SRC, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.qms_ref_sort.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       u64p, u64p]
            L.qms_ref_sort.restype = ctypes.c_int
            L.qms_ref_out_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                          ctypes.c_size_t, ctypes.c_int, u64p]
            L.qms_ref_out_u32.restype = ctypes.c_int
            L.qms_ref_dp.argtypes = [ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]
            L.qms_ref_dp.restype = ctypes.c_int
            L.qms_ref_adversary_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                                ctypes.c_int, u64p]
            L.qms_ref_adversary_u32.restype = ctypes.c_int
            L.qms_ref_sort2.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, u64p, u64p]
            L.qms_ref_sort2.restype = ctypes.c_int
            L.qms_ref_moves_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, u64p]
            L.qms_ref_moves_u32.restype = ctypes.c_int
            L.qms_ref_out_moves_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                                ctypes.c_size_t, ctypes.c_int, u64p, u64p]
            L.qms_ref_out_moves_u32.restype = ctypes.c_int
            L.qms_ref_median5_u32.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), u64p]
            L.qms_ref_median5_u32.restype = ctypes.c_int
            szp = ctypes.POINTER(ctypes.c_size_t)
            L.qms_ref_select_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                             ctypes.c_int, szp, u64p, ctypes.c_void_p,
                                             ctypes.c_size_t, szp]
            L.qms_ref_select_u32.restype = ctypes.c_int
            L.qms_ref_rounds_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_size_t, szp, u64p]
            L.qms_ref_rounds_u32.restype = ctypes.c_int
            L.qms_ref_qmqs_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_size_t, u64p]
            L.qms_ref_qmqs_u32.restype = ctypes.c_int
            L.qms_ref_dp_qmqs.argtypes = [ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p,
                                          ctypes.c_void_p]
            L.qms_ref_dp_qmqs.restype = ctypes.c_int
            L.qms_ref_out_x_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                            ctypes.c_size_t, ctypes.c_int, ctypes.c_size_t, u64p]
            L.qms_ref_out_x_u32.restype = ctypes.c_int
            L.qms_ref_sort4_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                            ctypes.c_int, u64p, u64p, u64p]
            L.qms_ref_sort4_u32.restype = ctypes.c_int
            L.qms_ref_msort4_u32.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                             ctypes.c_size_t, ctypes.c_int, ctypes.c_int, u64p, u64p]
            L.qms_ref_msort4_u32.restype = ctypes.c_int
            _lib = L
    return _lib


def _dtype_name(a: np.ndarray) -> str:
    for k, v in NP_DTYPES.items():
        if a.dtype == v:
            return k
    raise TypeError("unsupported key dtype %s" % a.dtype)


MOM_RULES = {"basic": 0, "faithful": 1}


def sort(keys: np.ndarray, vals: np.ndarray | None = None, variant: str = "m3",
         mode: str = "analysis", side: int = 0, mom: str = "basic"):
    """Sorts ``keys`` in place (and ``vals`` with them).

    ``mom="faithful"`` adds the Sec. 4 details to median-of-medians rounds
    (adaptive selection, partition of the 2n/3 non-medians only).
    Returns ``(comparisons, rounds)``.
    """
    assert keys.flags.c_contiguous
    d = _dtype_name(keys)
    vp = None
    if vals is not None:
        assert vals.dtype == np.uint32 and vals.flags.c_contiguous and len(vals) == len(keys)
        vp = vals.ctypes.data
    c = ctypes.c_uint64(0)
    r = ctypes.c_uint64(0)
    rc = lib().qms_ref_sort2(keys.ctypes.data, vp, len(keys), DTYPES[d], VARIANTS[variant],
                             MODES[mode], side, MOM_RULES[mom], ctypes.byref(c), ctypes.byref(r))
    if rc != 0:
        raise RuntimeError("qms_ref_sort failed: %d" % rc)
    return c.value, r.value


def sort_moves_u32(keys: np.ndarray, variant: str = "m3", mode: str = "analysis", side: int = 0,
                   mom: str = "basic"):
    """Sorts uint32 ``keys`` in place counting element moves (Sec. 5: an
    assignment of an input element is one move, a swap three).

    Returns ``(comparisons, moves)``.
    """
    assert keys.dtype == np.uint32 and keys.flags.c_contiguous
    c = ctypes.c_uint64(0)
    m = ctypes.c_uint64(0)
    rc = lib().qms_ref_moves_u32(keys.ctypes.data, len(keys), VARIANTS[variant], MODES[mode],
                                 side, MOM_RULES[mom], ctypes.byref(c), ctypes.byref(m))
    if rc != 0:
        raise RuntimeError("qms_ref_moves_u32 failed: %d" % rc)
    return c.value, m.value


def out_moves_u32(a: np.ndarray, b: int, e: int, temp: int, mode: str = "analysis"):
    """Fig. 3 ``out`` with moves counted; returns ``(comparisons, moves)``."""
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    c = ctypes.c_uint64(0)
    m = ctypes.c_uint64(0)
    rc = lib().qms_ref_out_moves_u32(a.ctypes.data, b, e, temp, MODES[mode], ctypes.byref(c),
                                     ctypes.byref(m))
    if rc != 0:
        raise RuntimeError("qms_ref_out_moves_u32 failed: %d" % rc)
    return c.value, m.value


def sort4_u32(keys: np.ndarray, variant: str = "m3", mode: str = "analysis"):
    """QuickMergesort whose Mergesort step is the four-way swap-merge (the
    multi-way merging of Sec. 6) on uint32 ``keys``, in place.

    Returns ``(comparisons, rounds, moves)``.
    """
    assert keys.dtype == np.uint32 and keys.flags.c_contiguous
    c, r, m = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = lib().qms_ref_sort4_u32(keys.ctypes.data, len(keys), VARIANTS[variant], MODES[mode],
                                 ctypes.byref(c), ctypes.byref(r), ctypes.byref(m))
    if rc != 0:
        raise RuntimeError("qms_ref_sort4_u32 failed: %d" % rc)
    return c.value, r.value, m.value


def msort4_u32(a: np.ndarray, b: int, n: int, t: int, to_target: bool = False,
               mode: str = "analysis"):
    """The four-way swap-merge Mergesort alone on ``a`` (changed in place):
    ``a[b:b+n]`` sorted in place with the buffer ``a[t:t+n]``, or into
    ``a[t:t+n]`` with ``to_target``.  Returns ``(comparisons, moves)``."""
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    c, m = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = lib().qms_ref_msort4_u32(a.ctypes.data, b, n, t, 1 if to_target else 0, MODES[mode],
                                  ctypes.byref(c), ctypes.byref(m))
    if rc != 0:
        raise RuntimeError("qms_ref_msort4_u32 failed: %d" % rc)
    return c.value, m.value


def median5_u32(v) -> tuple:
    """The selection's median of five: ``(index of the median in v, comparisons)``."""
    a = np.ascontiguousarray(np.asarray(v, dtype=np.uint32))
    assert a.size == 5
    pos = ctypes.c_int(-1)
    c = ctypes.c_uint64(0)
    rc = lib().qms_ref_median5_u32(a.ctypes.data, ctypes.byref(pos), ctypes.byref(c))
    if rc != 0:
        raise RuntimeError("qms_ref_median5_u32 failed")
    return pos.value, c.value


def select_u32(a: np.ndarray, i: int, adaptive: bool = False, trace_cap: int = 4096):
    """Groups-of-five selection of rank ``i`` in ``a`` (rearranged in place).

    Returns ``(position, comparisons, trace)`` with ``trace`` an array of
    (range size, size continued on) pairs, one per iteration.
    """
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    pos = ctypes.c_size_t(0)
    c = ctypes.c_uint64(0)
    ln = ctypes.c_size_t(0)
    tr = np.zeros(2 * trace_cap, dtype=np.uint64)
    rc = lib().qms_ref_select_u32(a.ctypes.data, len(a), i, 1 if adaptive else 0,
                                  ctypes.byref(pos), ctypes.byref(c), tr.ctypes.data, trace_cap,
                                  ctypes.byref(ln))
    if rc != 0:
        raise RuntimeError("qms_ref_select_u32 failed")
    k = min(ln.value, trace_cap)
    return pos.value, c.value, tr[: 2 * k].reshape(k, 2)


def qmqs_u32(keys: np.ndarray, x_thresh: int, variant: str = "m3", mode: str = "analysis") -> int:
    """QuickMergeXsort (Sec. 3): Mergesort stops below ``x_thresh`` elements
    and X = CleverQuicksort sorts the block.  Sorts in place; returns the
    comparisons."""
    assert keys.dtype == np.uint32 and keys.flags.c_contiguous
    c = ctypes.c_uint64(0)
    rc = lib().qms_ref_qmqs_u32(keys.ctypes.data, len(keys), VARIANTS[variant], MODES[mode],
                                x_thresh, ctypes.byref(c))
    if rc != 0:
        raise RuntimeError("qms_ref_qmqs_u32 failed")
    return c.value


def out_x_u32(a: np.ndarray, b: int, e: int, temp: int, x_thresh: int, mode: str = "analysis") -> int:
    """Fig. 3 ``out`` with X = CleverQuicksort for msort calls below x_thresh."""
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    c = ctypes.c_uint64(0)
    rc = lib().qms_ref_out_x_u32(a.ctypes.data, b, e, temp, MODES[mode], x_thresh, ctypes.byref(c))
    if rc != 0:
        raise RuntimeError("qms_ref_out_x_u32 failed")
    return c.value


def dp_qmqs(nmax: int, x_thresh: int):
    """Exact-average tables (T, Q) of QuickMergeXsort with X = CleverQuicksort
    below x_thresh (T) and of CleverQuicksort alone (Q), n = 0..nmax."""
    T = np.zeros(nmax + 1, dtype=np.float64)
    Q = np.zeros(nmax + 1, dtype=np.float64)
    rc = lib().qms_ref_dp_qmqs(nmax, x_thresh, T.ctypes.data, Q.ctypes.data)
    if rc != 0:
        raise RuntimeError("qms_ref_dp_qmqs failed")
    return T, Q


ROUND_FIELDS = ("b", "e", "lt", "gt", "mom", "cmp_pivot", "cmp_part", "left")


def rounds_u32(keys: np.ndarray, variant: str = "m3", mode: str = "analysis", side: int = 0,
               mom: str = "basic", cap: int = 1 << 16):
    """Sorts uint32 ``keys`` in place and returns ``(rounds, comparisons)``,
    ``rounds`` an array of records with the fields ``ROUND_FIELDS``."""
    assert keys.dtype == np.uint32 and keys.flags.c_contiguous
    rec = np.zeros(8 * cap, dtype=np.uint64)
    ln = ctypes.c_size_t(0)
    c = ctypes.c_uint64(0)
    rc = lib().qms_ref_rounds_u32(keys.ctypes.data, len(keys), VARIANTS[variant], MODES[mode],
                                  side, MOM_RULES[mom], rec.ctypes.data, cap, ctypes.byref(ln),
                                  ctypes.byref(c))
    if rc != 0:
        raise RuntimeError("qms_ref_rounds_u32 failed")
    k = min(ln.value, cap)
    return rec[: 8 * k].reshape(k, 8), c.value


def out_u32(a: np.ndarray, b: int, e: int, temp: int, mode: str = "analysis") -> int:
    """Fig. 3 ``out``: Mergesorts a[b:e] with the buffer at a[temp:]."""
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    c = ctypes.c_uint64(0)
    rc = lib().qms_ref_out_u32(a.ctypes.data, b, e, temp, MODES[mode], ctypes.byref(c))
    if rc != 0:
        raise RuntimeError("qms_ref_out_u32 failed: %d" % rc)
    return c.value


def dp(nmax: int):
    """Exact-average tables (T, M) for n = 0..nmax (analysis-mode median-of-3)."""
    T = np.zeros(nmax + 1, dtype=np.float64)
    M = np.zeros(nmax + 1, dtype=np.float64)
    rc = lib().qms_ref_dp(nmax, T.ctypes.data, M.ctypes.data)
    if rc != 0:
        raise RuntimeError("qms_ref_dp failed")
    return T, M


def adversary_u32(n: int, variant: str = "m3", mode: str = "analysis"):
    """McIlroy-adversary input (a permutation of 0..n-1) against this oracle.

    Returns ``(keys, comparisons the oracle made on it)``.
    """
    a = np.empty(n, dtype=np.uint32)
    c = ctypes.c_uint64(0)
    rc = lib().qms_ref_adversary_u32(a.ctypes.data, n, VARIANTS[variant], MODES[mode],
                                     ctypes.byref(c))
    if rc != 0:
        raise RuntimeError("qms_ref_adversary_u32 failed")
    return a, c.value


def reference_sorted(keys: np.ndarray) -> np.ndarray:
    """The plain definition of the result (Sec. 1: the ascending order of the
    input; floats in IEEE order with -0 before +0).  The ascending order is
    unique, so any correct sort equals it byte for byte."""
    if keys.dtype == np.float32:
        order = np.lexsort((~np.signbit(keys), keys))
        return keys[order]
    return np.sort(keys, kind="stable")


def canonical_pairs(keys: np.ndarray, vals: np.ndarray):
    """(key, payload) pairs sorted by key order, then payload: the canonical
    form used to compare key-value results whose order among equal keys is
    not fixed (QuickMergesort is not stable)."""
    if keys.dtype == np.float32:
        order = np.lexsort((vals, ~np.signbit(keys), keys))
    else:
        order = np.lexsort((vals, keys))
    return keys[order], vals[order]
