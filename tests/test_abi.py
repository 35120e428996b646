"""The C-ABI library builds, loads without a GPU and exports every function
that include/qms.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "qms.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qms_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = _declared()
    for want in ("qms_sort", "qms_sort_pairs", "qms_tile_sort", "qms_partition", "qms_mergesort",
                 "qms_mergesort_half", "qms_sort_batched", "qms_server_create",
                 "qms_server_submit", "qms_server_poll", "qms_server_destroy",
                 "qms_sort_noalloc", "qms_release_cached"):
        assert want in names, want


def _define(name):
    txt = open(os.path.join(ROOT, "include", "qms.h")).read()
    m = re.search(r"#define\s+%s\s+\(?(-?[0-9a-fx]+)(ull)?" % name, txt)
    assert m, name
    return int(m.group(1), 0)


def test_header_constants_match_the_binding():
    import paper_1804_10062_gb300 as q
    txt = open(os.path.join(ROOT, "include", "qms.h")).read()
    m = re.search(r"#define\s+QMS_NOALLOC_MAX_N\s+\(1ull\s*<<\s*(\d+)\)", txt)
    assert m and (1 << int(m.group(1))) == q.QMS_NOALLOC_MAX_N
    for name in ("QMS_OK", "QMS_EINVAL", "QMS_ENOMEM", "QMS_EBUDGET", "QMS_ECUDA",
                 "QMS_ETIMEOUT", "QMS_EAGAIN", "QMS_EINTERNAL", "QMS_FLAG_ASYNC",
                 "QMS_FLAG_HOST_DRIVEN", "QMS_FLAG_LARGER_SIDE", "QMS_FLAG_TEST_WITHHOLD",
                 "QMS_FLAG_DEVICE_DRIVEN"):
        assert _define(name) == getattr(q, name), name
    # qms_options field order: pivot, count_cmps, flags, spin_limit, profile
    body = re.search(r"typedef struct \{([^{}]*)\} qms_options;", txt).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)\s*;", body)
    assert fields == [f for f, _ in q.qms_options._fields_], fields


def test_library_exports_every_declared_symbol():
    from paper_1804_10062_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_error_strings_and_argument_checks_without_gpu():
    import paper_1804_10062_gb300 as q
    lib = q.lib()
    assert lib.qms_version() >= 10000
    assert q.error_string(q.QMS_EINVAL) == "invalid argument"
    # argument validation happens before any CUDA call
    assert lib.qms_sort(None, 10, 0, None, None, None) == q.QMS_EINVAL
    assert lib.qms_sort(None, 1, 0, None, None, None) == q.QMS_OK
    assert lib.qms_tile_sort(None, None, 9000, 0, None) == q.QMS_EINVAL
    # the no-allocation entry point checks its size cap before any CUDA call
    assert lib.qms_sort_noalloc(None, q.QMS_NOALLOC_MAX_N + 1, 0, None, None, None) == q.QMS_EINVAL


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1804_10062_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "qms_ref" not in src, fn
