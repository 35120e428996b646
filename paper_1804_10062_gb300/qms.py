"""ctypes binding of libqms.so (include/qms.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Key tensors are
CUDA tensors (uint32, uint64, int64 or float32; any 4/8-byte dtype with an
explicit ``dtype=`` names raw bit patterns); payload tensors are uint32 (or
int32 bit views).  The stream is the current torch stream unless given.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

QMS_OK, QMS_EINVAL, QMS_ENOMEM, QMS_EBUDGET, QMS_ECUDA, QMS_ETIMEOUT, QMS_EAGAIN, QMS_EINTERNAL = \
    0, -1, -2, -3, -4, -5, -6, -7
DTYPE_CODES = {"u32": 0, "u64": 1, "i64": 2, "f32": 3}
PIVOTS = {"m3": 0, "sqrtn": 1, "mom": 2, "hybrid": 3}

_lock = threading.Lock()
_lib = None


class QmsError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed: %s (%d)" % (what, error_string(code), code))
        self.code = code


NKINDS = 8
KIND_NAMES = ["leaf", "merge_split", "merge", "part_local", "part_scan", "part_exchange", "pivot",
              "batch"]


class qms_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * NKINDS), ("bytes", ctypes.c_uint64 * NKINDS),
                ("launches", ctypes.c_uint64 * NKINDS)]

    def as_dict(self):
        return {KIND_NAMES[i]: {"ms": self.ms[i], "bytes": self.bytes[i],
                                "launches": self.launches[i]} for i in range(NKINDS)}


class qms_options(ctypes.Structure):
    _fields_ = [("pivot", ctypes.c_int), ("count_cmps", ctypes.c_int),
                ("flags", ctypes.c_int), ("spin_limit", ctypes.c_int),
                ("profile", ctypes.POINTER(qms_profile))]


class qms_stats(ctypes.Structure):
    _fields_ = [("comparisons", ctypes.c_uint64), ("aux_bytes", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("mom_rounds", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class qms_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("batch_size", ctypes.c_int), ("n", ctypes.c_uint64),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class qms_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "completed", "keys", "batches", "batched_requests", "pending", "in_flight",
        "peak_in_flight", "used_bytes", "peak_used_bytes", "budget_bytes")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libqms.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
            vp, sz, i, u64p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)
            sig = {
                "qms_version": ([], i),
                "qms_error_string": ([i], ctypes.c_char_p),
                "qms_release_cached": ([], i),
                "qms_sort": ([vp, sz, i, ctypes.POINTER(qms_options), vp, ctypes.POINTER(qms_stats)], i),
                "qms_sort_pairs": ([vp, vp, sz, i, ctypes.POINTER(qms_options), vp,
                                    ctypes.POINTER(qms_stats)], i),
                "qms_tile_sort": ([vp, vp, sz, i, vp], i),
                "qms_sort_batched": ([vp, vp, vp, sz, i, ctypes.POINTER(qms_options), vp,
                                      ctypes.POINTER(qms_stats)], i),
                "qms_partition": ([vp, vp, sz, i, i, vp, u64p, u64p], i),
                "qms_mergesort": ([vp, vp, sz, sz, i, vp], i),
                "qms_mergesort_half": ([vp, vp, sz, sz, i, vp], i),
                "qms_sort_noalloc": ([vp, sz, i, ctypes.POINTER(qms_options), vp,
                                      ctypes.POINTER(qms_stats)], i),
                "qms_batched_autotune": ([i, i, vp, ctypes.c_char_p, sz], i),
                "qms_batched_get_plan": ([i, i, ctypes.POINTER(i), i, ctypes.POINTER(i)], i),
                "qms_batched_set_plan": ([i, i, ctypes.POINTER(i), i], i),
                "qms_batched_plan_read": ([ctypes.c_char_p, i, i, i, ctypes.POINTER(i), i], i),
                "qms_batched_plan_write": ([ctypes.c_char_p, i, i, i, ctypes.POINTER(i),
                                            ctypes.POINTER(ctypes.c_double), i], i),
                "qms_batched_config_name": ([i], ctypes.c_char_p),
                "qms_server_create": ([sz, i, i, i, ctypes.POINTER(vp)], i),
                "qms_server_submit": ([vp, vp, vp, sz, i, i, u64p], i),
                "qms_server_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(i),
                                     ctypes.POINTER(qms_request_info)], i),
                "qms_server_wait": ([vp, ctypes.c_uint64, ctypes.c_double,
                                     ctypes.POINTER(qms_request_info)], i),
                "qms_server_get_stats": ([vp, ctypes.POINTER(qms_server_stats)], i),
                "qms_server_destroy": ([vp], i),
                "qms_server_pause": ([vp, i], i),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def error_string(code: int) -> str:
    return lib().qms_error_string(code).decode()


def qms_release_cached():
    """Frees the device-driven sort's cached graph instances and workspaces
    on the current device (later calls rebuild them)."""
    _raise(lib().qms_release_cached(), "qms_release_cached")


def _dtype_code(t, dtype):
    import torch
    if dtype is not None:
        return DTYPE_CODES[dtype]
    m = {torch.uint32: "u32", torch.uint64: "u64", torch.int64: "i64", torch.float32: "f32"}
    if t.dtype not in m:
        raise TypeError("key dtype %s needs an explicit dtype=" % t.dtype)
    return DTYPE_CODES[m[t.dtype]]


def _check_keys(t, dtype):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("keys must be a contiguous CUDA tensor")
    code = _dtype_code(t, dtype)
    want = 4 if code in (0, 3) else 8
    if t.element_size() != want:
        raise ValueError("element size %d does not match dtype" % t.element_size())
    return code


def _check_vals(v, n):
    if v is None:
        return None
    if not v.is_cuda or not v.is_contiguous() or v.element_size() != 4 or v.numel() != n:
        raise ValueError("payload must be a contiguous CUDA tensor of n 4-byte words")
    return ctypes.c_void_p(v.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _raise(rc, what):
    if rc != QMS_OK:
        raise QmsError(rc, what)


QMS_FLAG_ASYNC = 1
QMS_FLAG_HOST_DRIVEN = 2
QMS_FLAG_LARGER_SIDE = 4
QMS_FLAG_TEST_WITHHOLD = 8
QMS_FLAG_DEVICE_DRIVEN = 16
SIDES = {"fig3": 0, "larger": QMS_FLAG_LARGER_SIDE}


def _options(pivot, count_cmps, profile, flags=0, spin_limit=0):
    opt = qms_options(PIVOTS[pivot], 1 if count_cmps else 0, flags, int(spin_limit), None)
    if profile is not None:
        opt.profile = ctypes.pointer(profile)
    return opt


def _driver_flags(host_driven):
    if host_driven is None:
        return 0
    return QMS_FLAG_HOST_DRIVEN if host_driven else QMS_FLAG_DEVICE_DRIVEN


def qms_sort(keys, pivot: str = "m3", count_cmps: bool = False, stream=None, dtype=None,
             profile: qms_profile | None = None, host_driven: bool | None = None,
             wait: bool = True, side: str = "fig3", spin_limit: int = 0,
             test_withhold: bool = False):
    """Sorts ``keys`` in place; returns the qms_stats fields as a dict (or
    None with ``wait=False``: the sort is only enqueued on the stream).

    ``profile`` (a qms_profile) accumulates per-kernel device times (this
    runs the rounds from the host); ``host_driven`` True selects that driver
    without profiling, False the device-driven graph, None the library's
    choice (host-driven for waiting calls of 2^16 keys or more).  ``side``: "fig3" (Fig. 3's rule, full-size buffer) or
    "larger" (Mergesort the larger side with a half-size buffer when it
    fits).  ``spin_limit`` bounds the device waits of the overlapped merge
    (polls of one flag; 0 = default); ``test_withhold`` is the failure-test
    hook QMS_FLAG_TEST_WITHHOLD."""
    code = _check_keys(keys, dtype)
    flags = (_driver_flags(host_driven) | (0 if wait else QMS_FLAG_ASYNC)
             | SIDES[side] | (QMS_FLAG_TEST_WITHHOLD if test_withhold else 0))
    opt = _options(pivot, count_cmps, profile, flags, spin_limit)
    st = qms_stats()
    rc = lib().qms_sort(ctypes.c_void_p(keys.data_ptr()), keys.numel(), code, ctypes.byref(opt),
                        _stream(stream), ctypes.byref(st) if wait else None)
    _raise(rc, "qms_sort")
    return st.as_dict() if wait else None


def qms_sort_pairs(keys, vals, pivot: str = "m3", count_cmps: bool = False, stream=None, dtype=None,
                   profile: qms_profile | None = None, host_driven: bool | None = None,
                   side: str = "fig3", wait: bool = True):
    """Sorts ``keys`` in place, moving ``vals`` with them; returns stats (or
    None with ``wait=False``: the sort is only enqueued on the stream).
    ``host_driven`` as for qms_sort."""
    code = _check_keys(keys, dtype)
    vp = _check_vals(vals, keys.numel())
    opt = _options(pivot, count_cmps, profile,
                   _driver_flags(host_driven) | SIDES[side]
                   | (0 if wait else QMS_FLAG_ASYNC))
    st = qms_stats()
    rc = lib().qms_sort_pairs(ctypes.c_void_p(keys.data_ptr()), vp, keys.numel(), code,
                              ctypes.byref(opt), _stream(stream), ctypes.byref(st) if wait else None)
    _raise(rc, "qms_sort_pairs")
    return st.as_dict() if wait else None


def qms_sort_batched(keys, offsets, vals=None, pivot: str = "m3", count_cmps: bool = False,
                     stream=None, dtype=None, profile: qms_profile | None = None):
    """Sorts every segment keys[offsets[i]:offsets[i+1]] (offsets: CUDA int64/uint64
    tensor of nseg + 1 entries); returns stats."""
    code = _check_keys(keys, dtype)
    if not offsets.is_cuda or not offsets.is_contiguous() or offsets.element_size() != 8:
        raise ValueError("offsets must be a contiguous CUDA tensor of 8-byte integers")
    opt = _options(pivot, count_cmps, profile)
    st = qms_stats()
    rc = lib().qms_sort_batched(ctypes.c_void_p(keys.data_ptr()), _check_vals(vals, keys.numel()),
                                ctypes.c_void_p(offsets.data_ptr()), offsets.numel() - 1, code,
                                ctypes.byref(opt), _stream(stream), ctypes.byref(st))
    _raise(rc, "qms_sort_batched")
    return st.as_dict()


def qms_tile_sort(keys, vals=None, stream=None, dtype=None):
    code = _check_keys(keys, dtype)
    rc = lib().qms_tile_sort(ctypes.c_void_p(keys.data_ptr()), _check_vals(vals, keys.numel()),
                             keys.numel(), code, _stream(stream))
    _raise(rc, "qms_tile_sort")


def qms_partition(keys, vals=None, pivot: str = "m3", stream=None, dtype=None):
    """One partition step; returns (pivot index k, further equal keys eq)."""
    code = _check_keys(keys, dtype)
    k = ctypes.c_uint64(0)
    eq = ctypes.c_uint64(0)
    rc = lib().qms_partition(ctypes.c_void_p(keys.data_ptr()), _check_vals(vals, keys.numel()),
                             keys.numel(), code, PIVOTS[pivot], _stream(stream), ctypes.byref(k),
                             ctypes.byref(eq))
    _raise(rc, "qms_partition")
    return k.value, eq.value


def qms_mergesort(keys, m: int, buf: int, vals=None, stream=None, dtype=None):
    """Sorts keys[0:m] using keys[buf:buf+m] as swap buffer (buf >= m)."""
    code = _check_keys(keys, dtype)
    if buf + m > keys.numel():
        raise ValueError("buffer out of range")
    rc = lib().qms_mergesort(ctypes.c_void_p(keys.data_ptr()), _check_vals(vals, keys.numel()), m,
                             buf, code, _stream(stream))
    _raise(rc, "qms_mergesort")


def qms_mergesort_half(keys, m: int, buf: int, vals=None, stream=None, dtype=None):
    """Sorts keys[0:m] using the ceil(m/2) slots keys[buf:...] as swap buffer
    (buf >= m): Fig. 3 "out" with its overlapped final merge."""
    code = _check_keys(keys, dtype)
    if buf < m or buf + (m - m // 2) > keys.numel():
        raise ValueError("buffer out of range")
    rc = lib().qms_mergesort_half(ctypes.c_void_p(keys.data_ptr()), _check_vals(vals, keys.numel()),
                                  m, buf, code, _stream(stream))
    _raise(rc, "qms_mergesort_half")


QMS_BATCH_BINS = 17
BATCH_CONFIGS = ["group32x16", "group64x16", "group128x16", "group256x16", "group512x16",
                 "group256x32", "group512x32", "block_qms", "group1024x32", "pair1024x32"]
BCFG = {name: i for i, name in enumerate(BATCH_CONFIGS)}


def qms_batched_autotune(dtype: str = "u32", payload: bool = False, stream=None) -> str:
    """Times every batched-form configuration per length bin on this GPU,
    installs and stores the fastest plan; returns the timing report."""
    buf = ctypes.create_string_buffer(1 << 16)
    rc = lib().qms_batched_autotune(DTYPE_CODES[dtype], 1 if payload else 0, _stream(stream), buf,
                                    len(buf))
    _raise(rc, "qms_batched_autotune")
    return buf.value.decode()


def qms_batched_get_plan(dtype: str = "u32", payload: bool = False):
    """(list of configuration names per length bin, tuned flag) on this device."""
    cfg = (ctypes.c_int * QMS_BATCH_BINS)()
    tuned = ctypes.c_int(0)
    rc = lib().qms_batched_get_plan(DTYPE_CODES[dtype], 1 if payload else 0, cfg, QMS_BATCH_BINS,
                                    ctypes.byref(tuned))
    _raise(rc, "qms_batched_get_plan")
    return [BATCH_CONFIGS[c] for c in cfg], bool(tuned.value)


def qms_batched_set_plan(names, dtype: str = "u32", payload: bool = False):
    cfg = (ctypes.c_int * QMS_BATCH_BINS)(*[BCFG[n] for n in names])
    rc = lib().qms_batched_set_plan(DTYPE_CODES[dtype], 1 if payload else 0, cfg, QMS_BATCH_BINS)
    _raise(rc, "qms_batched_set_plan")


def qms_batched_plan_read(path: str, dtype: str = "u32", payload: bool = False, sm_count: int = 152):
    """(names per bin, found) from a plan file; the default plan when not found."""
    cfg = (ctypes.c_int * QMS_BATCH_BINS)()
    rc = lib().qms_batched_plan_read(path.encode(), DTYPE_CODES[dtype], 1 if payload else 0, sm_count,
                                     cfg, QMS_BATCH_BINS)
    if rc not in (QMS_OK, QMS_EAGAIN):
        _raise(rc, "qms_batched_plan_read")
    return [BATCH_CONFIGS[c] for c in cfg], rc == QMS_OK


def qms_batched_plan_write(path: str, names, dtype: str = "u32", payload: bool = False,
                           sm_count: int = 152, ns_per_key=None):
    cfg = (ctypes.c_int * QMS_BATCH_BINS)(*[BCFG[n] for n in names])
    ns = None
    if ns_per_key is not None:
        ns = (ctypes.c_double * QMS_BATCH_BINS)(*ns_per_key)
    rc = lib().qms_batched_plan_write(path.encode(), DTYPE_CODES[dtype], 1 if payload else 0,
                                      sm_count, cfg, ns, QMS_BATCH_BINS)
    _raise(rc, "qms_batched_plan_write")


QMS_NOALLOC_MAX_N = 1 << 24


def qms_sort_noalloc(keys, pivot: str = "m3", count_cmps: bool = False, stream=None, dtype=None):
    """qms_sort without device allocation (n <= 2^24; scratch is a fixed
    device array shared by all calls: do not overlap calls on the GPU)."""
    code = _check_keys(keys, dtype)
    opt = _options(pivot, count_cmps, None)
    st = qms_stats()
    rc = lib().qms_sort_noalloc(ctypes.c_void_p(keys.data_ptr()), keys.numel(), code,
                                ctypes.byref(opt), _stream(stream), ctypes.byref(st))
    _raise(rc, "qms_sort_noalloc")
    return st.as_dict()


class QmsServer:
    """The qms_server_* calls.  ``submit`` takes raw addresses (host or
    device) so that callers keep full control of where the data lives."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 256, workers: int = 4,
                 max_batch: int = 4096):
        self._h = ctypes.c_void_p()
        rc = lib().qms_server_create(hbm_budget_bytes, max_slots, workers, max_batch,
                                     ctypes.byref(self._h))
        _raise(rc, "qms_server_create")

    def qms_server_submit(self, in_ptr: int, out_ptr: int, n: int, dtype: str,
                          pivot: str = "m3") -> int:
        t = ctypes.c_uint64(0)
        rc = lib().qms_server_submit(self._h, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), n,
                                     DTYPE_CODES[dtype], PIVOTS[pivot], ctypes.byref(t))
        _raise(rc, "qms_server_submit")
        return t.value

    def qms_server_poll(self, ticket: int):
        """Returns the request info dict when done, else None."""
        d = ctypes.c_int(0)
        info = qms_request_info()
        rc = lib().qms_server_poll(self._h, ticket, ctypes.byref(d), ctypes.byref(info))
        if rc == QMS_EAGAIN:
            return None
        _raise(rc, "qms_server_poll")
        return info.as_dict()

    def qms_server_wait(self, ticket: int, timeout_ms: float = 60000.0):
        info = qms_request_info()
        rc = lib().qms_server_wait(self._h, ticket, timeout_ms, ctypes.byref(info))
        _raise(rc, "qms_server_wait")
        return info.as_dict()

    def qms_server_get_stats(self):
        st = qms_server_stats()
        _raise(lib().qms_server_get_stats(self._h, ctypes.byref(st)), "qms_server_get_stats")
        return st.as_dict()

    def qms_server_pause(self, paused: bool = True):
        _raise(lib().qms_server_pause(self._h, 1 if paused else 0), "qms_server_pause")

    def qms_server_destroy(self):
        if self._h:
            rc = lib().qms_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            _raise(rc, "qms_server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.qms_server_destroy()
