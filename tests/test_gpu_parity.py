"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Key-only results must be byte-identical to the oracle (the ascending order is
unique).  Key-value results must have byte-identical keys and the same
(key, payload) multiset (payload = original index, so every pair is
identified); the order among equal keys is not fixed."""
import math

import numpy as np
import pytest

import oracle
import qms_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE = 8192
NP = {"u32": np.uint32, "u64": np.uint64, "i64": np.int64, "f32": np.float32}


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_10062_gb300 as q
    q.lib()
    return q


def _dev(a):
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32).copy()).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64).copy()).cuda()
    return torch.from_numpy(a.copy()).cuda()


def _host(t, dtype):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(NP[dtype])


def _dist_keys(dist, dtype, n, seed):
    if dist == "normal" and dtype != "f32":
        dist = "uniform"
    return gen.keys(dist, dtype, n, seed)


# ---------------------------------------------------------------------------
# Base case X


@pytest.mark.parametrize("dtype", ["u32", "u64", "i64", "f32"])
@pytest.mark.parametrize("n", [2, 3, 31, 32, 33, 511, 512, 513, 4095, 8191, 8192])
def test_tile_sort(q, dtype, n):
    k = _dist_keys("normal" if dtype == "f32" else "uniform", dtype, n, n)
    d = _dev(k)
    q.qms_tile_sort(d, dtype=dtype)
    assert _host(d, dtype).tobytes() == oracle.reference_sorted(k).tobytes()
    v = gen.payload_index(n)
    d, dv = _dev(k), _dev(v)
    q.qms_tile_sort(d, dv, dtype=dtype)
    ko, vo = _host(d, dtype), _host(dv, "u32")
    assert ko.tobytes() == oracle.reference_sorted(k).tobytes()
    assert k[vo].tobytes() == ko.tobytes()
    assert np.array_equal(np.sort(vo), v)


def test_tile_sort_max_keys_with_payload(q):
    # Real keys equal to the largest key must not be confused with padding.
    n = 5000
    k = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    k[::7] = 3
    v = gen.payload_index(n)
    d, dv = _dev(k), _dev(v)
    q.qms_tile_sort(d, dv, dtype="u32")
    ko, vo = _host(d, "u32"), _host(dv, "u32")
    assert ko.tobytes() == np.sort(k).tobytes()
    assert np.array_equal(np.sort(vo), v)
    assert np.array_equal(k[vo], ko)


# ---------------------------------------------------------------------------
# Partition step


@pytest.mark.parametrize("pivot", ["m3", "sqrtn", "mom"])
@pytest.mark.parametrize("dtype,dist", [("u32", "uniform"), ("u64", "mod16"), ("f32", "normal"),
                                        ("i64", "organ"), ("u32", "sorted")])
@pytest.mark.parametrize("n", [3, 100, TILE + 1, 5 * TILE + 777, 200003])
def test_partition_step(q, pivot, dtype, dist, n):
    k = _dist_keys(dist, dtype, n, 5 + n)
    v = gen.payload_index(n)
    d, dv = _dev(k), _dev(v)
    kk, eq = q.qms_partition(d, dv, pivot=pivot, dtype=dtype)
    ko, vo = _host(d, dtype), _host(dv, "u32")
    assert 0 <= kk < n and kk + 1 + eq <= n
    # same multiset of pairs
    assert np.array_equal(np.sort(vo), v)
    assert k[vo].tobytes() == ko.tobytes()
    p = ko[kk]
    if dtype == "f32":
        def lt(x, y):
            return (x < y) | ((x == y) & np.signbit(x) & ~np.signbit(y))

        def same(x, y):
            return (x == y) & (np.signbit(x) == np.signbit(y))
    else:
        def lt(x, y):
            return x < y

        def same(x, y):
            return x == y
    assert np.all(lt(ko[:kk], p))
    assert np.all(same(ko[kk:kk + 1 + eq], p))
    if eq:
        assert np.all(lt(p, ko[kk + 1 + eq:]))
    else:
        assert not np.any(lt(ko[kk + 1:], p))


# ---------------------------------------------------------------------------
# Mergesort with swap buffer (Fig. 3 "out")


@pytest.mark.parametrize("dtype", ["u32", "u64", "f32", "i64"])
@pytest.mark.parametrize("m", [2, 100, TILE, TILE + 1, 3 * TILE - 5, 8 * TILE, 9 * TILE + 17,
                               100000])
def test_mergesort_swap_buffer(q, dtype, m):
    k = _dist_keys("normal" if dtype == "f32" else "uniform", dtype, 2 * m + 3, m)
    v = gen.payload_index(2 * m + 3)
    d, dv = _dev(k), _dev(v)
    q.qms_mergesort(d, m, m + 3, dv, dtype=dtype)
    ko, vo = _host(d, dtype), _host(dv, "u32")
    assert ko[:m].tobytes() == oracle.reference_sorted(k[:m]).tobytes()
    # the three untouched slots between part and buffer
    assert ko[m:m + 3].tobytes() == k[m:m + 3].tobytes()
    # buffer multiset preserved (with its payloads)
    assert np.array_equal(np.sort(vo[m + 3:]), v[m + 3:])
    assert k[vo].tobytes() == ko.tobytes()


@pytest.mark.parametrize("dtype", ["u32", "u64", "f32", "i64"])
@pytest.mark.parametrize("m", [2, 3, 100, TILE, TILE + 1, 2 * TILE + 3, 3 * TILE - 5, 8 * TILE,
                               9 * TILE + 17, 100001, (1 << 20) + 7])
def test_mergesort_half_buffer(q, dtype, m):
    """Fig. 3 "out" with its ceil(m/2) buffer (overlapped final merge)."""
    r = m - m // 2
    k = _dist_keys("normal" if dtype == "f32" else "uniform", dtype, m + 5 + r, m + 1)
    v = gen.payload_index(m + 5 + r)
    d, dv = _dev(k), _dev(v)
    q.qms_mergesort_half(d, m, m + 5, dv, dtype=dtype)
    ko, vo = _host(d, dtype), _host(dv, "u32")
    assert ko[:m].tobytes() == oracle.reference_sorted(k[:m]).tobytes()
    # every part key travels with its payload
    assert np.array_equal(np.sort(vo[:m]), np.arange(m, dtype=np.uint32))
    assert np.array_equal(ko[:m], k[vo[:m]])
    assert ko[m:m + 5].tobytes() == k[m:m + 5].tobytes()
    # the buffer keeps its (key, payload) multiset
    assert np.array_equal(np.sort(vo[m + 5:]), v[m + 5:])
    assert np.array_equal(ko[m + 5:], k[vo[m + 5:]])


@pytest.mark.parametrize("dist", ["sorted", "reverse", "mod16", "organ"])
@pytest.mark.parametrize("m", [4 * TILE + 1, 300001])
def test_mergesort_half_vs_oracle_out(q, dist, m):
    """The same step on inputs whose halves do not interleave (every window
    of the overlapped merge waits on early tiles, or none does) and with
    many ties, against the oracle's Fig. 3 "out" on the same array."""
    r = m - m // 2
    k = gen.keys(dist, "u32", m + r, 9)
    ref = k.copy()
    oracle.out_u32(ref, 0, m, m)
    d = _dev(k)
    q.qms_mergesort_half(d, m, m, dtype="u32")
    ko = _host(d, "u32")
    assert ko[:m].tobytes() == ref[:m].tobytes()
    assert np.array_equal(np.sort(ko[m:]), np.sort(ref[m:]))


@pytest.mark.parametrize("side", ["larger", "fig3"])
@pytest.mark.parametrize("host_driven", [False, True])
@pytest.mark.parametrize("dist", ["uniform", "sorted", "mod16", "killer"])
def test_sort_side_policies(q, side, host_driven, dist):
    n = 3 * (1 << 17) + 4321
    if dist == "killer":
        k, _ = oracle.adversary_u32(n, "hybrid", "paper")
    else:
        k = gen.keys(dist, "u32", n, 21)
    ref = oracle.reference_sorted(k)
    d = _dev(k)
    q.qms_sort(d, pivot="hybrid", dtype="u32", side=side, host_driven=host_driven)
    assert _host(d, "u32").tobytes() == ref.tobytes()


# ---------------------------------------------------------------------------
# Whole sort against the oracle


def test_config1_permutation_m3(q):
    n = 1 << 20
    k = gen.permutation_u32(n, 1)
    ref = k.copy()
    c_ref, _ = oracle.sort(ref, variant="m3", mode="analysis")
    d = _dev(k)
    st = q.qms_sort(d, pivot="m3", count_cmps=True, dtype="u32")
    out = _host(d, "u32")
    assert out.tobytes() == ref.tobytes()
    # No comparison sort decides a permutation of n keys with fewer than
    # lg(n!) comparisons.  The GPU's merges add merge-path searches and its
    # leaves run sorting networks, so it compares more than the oracle's
    # Fig. 3 Mergesort, but by a bounded factor (1.38 measured at 2^20).
    lg_fact = math.lgamma(n + 1) / math.log(2)
    assert st["comparisons"] >= lg_fact
    assert c_ref <= st["comparisons"] <= 1.7 * c_ref


# host_driven: None is the library's choice for a waiting call of this size
# (the host loop), False the device-driven graph.
@pytest.mark.parametrize("host_driven", [None, False])
@pytest.mark.parametrize("pivot", ["m3", "sqrtn", "mom", "hybrid"])
@pytest.mark.parametrize("dtype,dist", [("u32", "uniform"), ("i64", "uniform"), ("f32", "normal"),
                                        ("u64", "uniform")])
def test_sort_vs_oracle(q, pivot, dtype, dist, host_driven):
    n = (1 << 18) + 12345
    k = _dist_keys(dist, dtype, n, 2)
    ref = k.copy()
    oracle.sort(ref, variant=pivot, mode="paper")
    d = _dev(k)
    q.qms_sort(d, pivot=pivot, dtype=dtype, host_driven=host_driven)
    assert _host(d, dtype).tobytes() == ref.tobytes()


@pytest.mark.parametrize("host_driven", [None, False])
@pytest.mark.parametrize("dist", ["uniform", "mod16", "sorted", "reverse", "organ", "killer"])
@pytest.mark.parametrize("pivot", ["hybrid", "m3"])
def test_pairs_vs_oracle(q, dist, pivot, host_driven):
    n = (1 << 17) + 3
    if dist == "killer":
        if pivot == "m3":
            pytest.skip("median-of-3 alone is quadratic on its adversary by design")
        k32, _ = oracle.adversary_u32(n, "hybrid", "paper")
        k = k32.astype(np.uint64)
    else:
        k = gen.keys(dist, "u64", n, 9)
    v = gen.payload_index(n)
    rk, rv = k.copy(), v.copy()
    oracle.sort(rk, rv, variant=pivot, mode="paper")
    d, dv = _dev(k), _dev(v)
    q.qms_sort_pairs(d, dv, pivot=pivot, dtype="u64", host_driven=host_driven)
    ko, vo = _host(d, "u64"), _host(dv, "u32")
    assert ko.tobytes() == rk.tobytes()
    ck, cv = oracle.canonical_pairs(ko, vo)
    rck, rcv = oracle.canonical_pairs(rk, rv)
    assert ck.tobytes() == rck.tobytes() and cv.tobytes() == rcv.tobytes()


@pytest.mark.parametrize("n", [0, 1, 2, 3, TILE - 1, TILE, TILE + 1, 2 * TILE + 1, 3 * TILE])
def test_edge_sizes(q, n):
    for dist in ("uniform", "mod16", "sorted", "reverse"):
        k = gen.keys(dist, "u64", n, 17)
        ref = oracle.reference_sorted(k)
        if n == 0:
            continue
        d = _dev(k)
        q.qms_sort(d, pivot="hybrid", dtype="u64")
        assert _host(d, "u64").tobytes() == ref.tobytes()


def test_all_equal_keys(q):
    n = 300000
    k = np.full(n, 42, dtype=np.uint32)
    v = gen.payload_index(n)
    d, dv = _dev(k), _dev(v)
    st = q.qms_sort_pairs(d, dv, pivot="m3", dtype="u32")
    assert np.all(_host(d, "u32") == 42)
    assert np.array_equal(np.sort(_host(dv, "u32")), v)
    assert st["rounds"] <= 2  # the equal block is final after one round


def test_invalid_arguments(q):
    d = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(q.QmsError):
        q.qms_tile_sort(torch.zeros(TILE + 1, dtype=torch.int32, device="cuda"), dtype="u32")
    lib = q.lib()
    assert lib.qms_sort(None, 10, 0, None, None, None) == q.QMS_EINVAL
    assert lib.qms_sort(d.data_ptr(), 10, 7, None, None, None) == q.QMS_EINVAL
    assert lib.qms_sort(None, 0, 0, None, None, None) == q.QMS_OK
    assert lib.qms_sort(None, 1, 0, None, None, None) == q.QMS_OK


def test_full_size_2_24_sampled(q):
    # BASELINE sizes: 2^24 uint32 / int64 / float32 (median-of-3 and the
    # worst-case-guaranteed variant), checked against the plain definition.
    n = 1 << 24
    for dtype, dist, pivot in (("u32", "uniform", "m3"), ("i64", "uniform", "hybrid"),
                               ("f32", "normal", "sqrtn"), ("u32", "uniform", "mom")):
        k = _dist_keys(dist, dtype, n, 3)
        d = _dev(k)
        q.qms_sort(d, pivot=pivot, dtype=dtype)
        assert _host(d, dtype).tobytes() == oracle.reference_sorted(k).tobytes(), (dtype, pivot)


@pytest.mark.parametrize("pivot", ["m3", "sqrtn", "mom", "hybrid"])
@pytest.mark.parametrize("dtype", ["u32", "i64"])
def test_host_driven_driver_matches_oracle(q, pivot, dtype):
    # The rounds can also run from the host (one launch per step; the
    # profiling path): same kernels, same result.
    n = (1 << 17) + 999
    k = _dist_keys("uniform", dtype, n, 44)
    ref = oracle.reference_sorted(k)
    d = _dev(k)
    st = q.qms_sort(d, pivot=pivot, dtype=dtype, host_driven=True)
    assert _host(d, dtype).tobytes() == ref.tobytes()
    d2 = _dev(k)
    st2 = q.qms_sort(d2, pivot=pivot, dtype=dtype, host_driven=False)
    assert _host(d2, dtype).tobytes() == ref.tobytes()
    assert st2["rounds"] >= 1 and st2["launches"] > 0


def test_release_cached_then_sort_again(q):
    # The device-driven sort's cached instances can be freed between calls;
    # the next call builds a new one.
    for rep in range(2):
        k = gen.keys("uniform", "u32", (1 << 18) + rep, 31 + rep)
        d = _dev(k)
        q.qms_sort(d, dtype="u32", wait=False)
        q.qms_release_cached()  # waits for that sort's launch, then frees
        assert _host(d, "u32").tobytes() == oracle.reference_sorted(k).tobytes()
    q.qms_release_cached()  # nothing cached: still fine


def test_async_sorts_growing_and_two_streams(q):
    # Back-to-back sorts whose sizes grow (the reused instance's workspace is
    # replaced while its previous sort may still run) on two streams at once.
    sizes = [(1 << 18) + 7, (1 << 21) + 3, (1 << 22) + 11, (1 << 19) + 5]
    arrays = [gen.keys("uniform", "u32", n, 80 + i) for i, n in enumerate(sizes)]
    ds = [_dev(a) for a in arrays]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    for i, d in enumerate(ds):
        s = streams[i % 2]
        with torch.cuda.stream(s):
            assert q.qms_sort(d, dtype="u32", wait=False, stream=s) is None
    for a, d in zip(arrays, ds):
        assert _host(d, "u32").tobytes() == np.sort(a).tobytes()


def test_async_sorts_back_to_back(q):
    # Several device-driven sorts enqueued without host waits on one stream.
    arrays = [gen.keys("uniform", "u32", (1 << 19) + i * 1001, 60 + i) for i in range(4)]
    ds = [_dev(a) for a in arrays]
    for d in ds:
        assert q.qms_sort(d, dtype="u32", wait=False) is None
    for a, d in zip(arrays, ds):
        assert _host(d, "u32").tobytes() == np.sort(a).tobytes()
