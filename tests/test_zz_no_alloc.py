"""GPU test of qms_sort_noalloc, the allocation-free sort.

Some callers cannot allocate device memory: an application that owns all GPU
memory through its own pool allocator and forbids any other cudaMalloc, or a
latency-critical loop where an allocation could synchronise the device or fail
under memory pressure.  qms_sort_noalloc keeps its scratch in a fixed device
array instead.  This test calls it through the C ABI and checks its output
byte for byte against the plain definition of the result (the ascending order
of the input, which is unique), on two calls in a row that share that array:
every pivot rule, one call with comparison counting, and the largest sizes
the fixed array admits.  The file is collected last so that a first-failure
run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import qms_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NP = {"u32": np.uint32, "u64": np.uint64, "i64": np.int64, "f32": np.float32}
CODES = {"u32": 0, "u64": 1, "i64": 2, "f32": 3}
PIVOTS = {"m3": 0, "sqrtn": 1, "mom": 2, "hybrid": 3}


def _dev(a):
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32).copy()).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64).copy()).cuda()
    return torch.from_numpy(a.copy()).cuda()


def _call(lib, q, t, n, dtype, pivot="m3", count=False):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    opt = q.qms_options(PIVOTS[pivot], 1 if count else 0, 0, 0, None)
    st = q.qms_stats()
    rc = lib.qms_sort_noalloc(ctypes.c_void_p(t.data_ptr()), n, CODES[dtype], ctypes.byref(opt),
                              stream, ctypes.byref(st))
    return rc, st


def test_noalloc_matches_the_definition_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_10062_gb300 as q
    lib = q.lib()
    cap = q.QMS_NOALLOC_MAX_N
    cases = [("u32", "uniform", (1 << 20) + 17, "m3", False),
             ("f32", "normal", 300001, "sqrtn", False),
             ("i64", "uniform", (1 << 18) + 5, "mom", False),
             ("u64", "mod16", 100003, "hybrid", False),
             ("u32", "uniform", 250007, "m3", True),
             ("u32", "uniform", cap, "m3", False),
             ("u64", "uniform", cap - 1, "hybrid", False)]
    for call in range(2):
        for dtype, dist, n, pivot, count in cases:
            k = gen.keys(dist, dtype, n, 40 + call)
            ref = oracle.reference_sorted(k)
            b = _dev(k)
            rc, st = _call(lib, q, b, n, dtype, pivot, count)
            assert rc == q.QMS_OK, (call, dtype, n, pivot, rc)
            torch.cuda.synchronize()
            rb = b.cpu().numpy().view(NP[dtype])
            assert rb.tobytes() == ref.tobytes(), (call, dtype, n, pivot)
            if count:
                # between the information-theoretic bound and a few times it
                lg = float(np.sum(np.log2(np.arange(2, n + 1, dtype=np.float64))))
                assert lg < st.comparisons < 3 * lg, (st.comparisons, lg)
            del b


def test_noalloc_rejects_sizes_beyond_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_10062_gb300 as q
    lib = q.lib()
    t = torch.zeros(8, dtype=torch.int32, device="cuda")
    # the size check comes before any access to the keys
    rc, _ = _call(lib, q, t, q.QMS_NOALLOC_MAX_N + 1, "u32")
    assert rc == q.QMS_EINVAL
