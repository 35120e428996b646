"""GPU parity of the batched form: every segment equals the oracle's sort of
that segment (byte-identical keys; identical canonical pairs), and equals the
single-array sort of the same segment alone."""
import numpy as np
import pytest

import oracle
import qms_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def _lengths(seed, nseg, extra=()):
    L = gen.batch_lengths(nseg, seed, 16, 65536).tolist()
    L += [0, 1, 2, 3, 8191, 8192, 8193, 16385] + list(extra)
    rng = np.random.default_rng(seed)
    rng.shuffle(L)
    return np.array(L, dtype=np.int64)


@pytest.mark.parametrize("dtype,dist", [("u32", "uniform"), ("f32", "uniform"), ("u64", "mod16"),
                                        ("i64", "uniform")])
@pytest.mark.parametrize("pivot", ["m3", "hybrid", "sqrtn", "mom"])
def test_batched_keys_vs_oracle(q, dtype, dist, pivot):
    L = _lengths(3, 120)
    off = gen.offsets_of(L)
    k = gen.keys(dist, dtype, int(off[-1]), 7)
    d = _dev(k)
    doff = torch.from_numpy(off.view(np.int64)).cuda()
    st = q.qms_sort_batched(d, doff, pivot=pivot, dtype=dtype)
    out = _host(d, dtype)
    for i in range(len(L)):
        a, b = int(off[i]), int(off[i + 1])
        ref = k[a:b].copy()
        oracle.sort(ref, variant=pivot, mode="paper")
        assert out[a:b].tobytes() == ref.tobytes(), (i, b - a)
    assert st["launches"] >= 1


@pytest.mark.parametrize("dist", ["uniform", "mod16", "sorted", "organ"])
def test_batched_pairs_vs_oracle(q, dist):
    L = _lengths(5, 80)
    off = gen.offsets_of(L)
    n = int(off[-1])
    k = gen.keys(dist, "u64", n, 11)
    v = gen.payload_index(n)
    d, dv = _dev(k), _dev(v)
    doff = torch.from_numpy(off.view(np.int64)).cuda()
    q.qms_sort_batched(d, doff, vals=dv, pivot="hybrid", dtype="u64")
    ko, vo = _host(d, "u64"), _host(dv, "u32")
    for i in range(len(L)):
        a, b = int(off[i]), int(off[i + 1])
        rk, rv = k[a:b].copy(), v[a:b].copy()
        oracle.sort(rk, rv, variant="hybrid", mode="paper")
        assert ko[a:b].tobytes() == rk.tobytes()
        ck, cv = oracle.canonical_pairs(ko[a:b], vo[a:b])
        rck, rcv = oracle.canonical_pairs(rk, rv)
        assert cv.tobytes() == rcv.tobytes()


def test_batched_large_segments_use_grid_path(q):
    # segments beyond one block's limit (64 tiles) run through the grid driver
    L = np.array([700000, 5, 600001, 70000, 0, 9000], dtype=np.int64)
    off = gen.offsets_of(L)
    k = gen.keys("uniform", "u32", int(off[-1]), 13)
    d = _dev(k)
    st = q.qms_sort_batched(d, torch.from_numpy(off.view(np.int64)).cuda(), dtype="u32")
    out = _host(d, "u32")
    for i in range(len(L)):
        a, b = int(off[i]), int(off[i + 1])
        assert out[a:b].tobytes() == np.sort(k[a:b]).tobytes()
    assert st["rounds"] > 0


def test_each_result_alone_equals_in_the_mix(q):
    L = _lengths(9, 60)
    off = gen.offsets_of(L)
    k = gen.keys("uniform", "f32", int(off[-1]), 21)
    d = _dev(k)
    q.qms_sort_batched(d, torch.from_numpy(off.view(np.int64)).cuda(), dtype="f32")
    mix = _host(d, "f32")
    for i in range(0, len(L), 7):
        a, b = int(off[i]), int(off[i + 1])
        if b - a < 2:
            continue
        alone = _dev(k[a:b])
        q.qms_sort(alone, dtype="f32")
        assert _host(alone, "f32").tobytes() == mix[a:b].tobytes()


def test_batched_rejects_decreasing_offsets(q):
    off = np.array([0, 10, 5, 20], dtype=np.uint64)
    d = torch.zeros(20, dtype=torch.int32, device="cuda")
    with pytest.raises(q.QmsError):
        q.qms_sort_batched(d, torch.from_numpy(off.view(np.int64)).cuda(), dtype="u32")


def test_batched_full_size_sampled(q):
    # 65,536 segments, lengths log-uniform in [16, 65536] (about 2^29 keys):
    # every segment checked sorted on the device, 64 sampled segments against
    # the oracle, and the key multiset checked by a sum.
    nseg = 65536
    L = gen.batch_lengths(nseg, 1, 16, 65536)
    off = gen.offsets_of(L)
    n = int(off[-1])
    k = gen.keys("uniform", "u32", n, 1)
    d = _dev(k)
    before = int(torch.sum(d.to(torch.int64) & 0xFFFFFFFF).item())
    q.qms_sort_batched(d, torch.from_numpy(off.view(np.int64)).cuda(), dtype="u32")
    du = d.to(torch.int64) & 0xFFFFFFFF
    assert int(torch.sum(du).item()) == before
    seg_id = torch.repeat_interleave(torch.arange(nseg, device="cuda"),
                                     torch.from_numpy(L).cuda())
    same = seg_id[1:] == seg_id[:-1]
    assert bool(torch.all((du[1:] >= du[:-1]) | ~same).item())
    rng = np.random.default_rng(0)
    out = None
    for i in rng.choice(nseg, 64, replace=False):
        a, b = int(off[i]), int(off[i + 1])
        ref = k[a:b].copy()
        oracle.sort(ref, variant="m3", mode="paper")
        got = d[a:b].cpu().numpy().view(np.uint32)
        assert got.tobytes() == ref.tobytes()
