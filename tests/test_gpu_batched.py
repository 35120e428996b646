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


CAPACITY = {"group32x16": 512, "group64x16": 1024, "group128x16": 2048, "group256x16": 4096,
            "group512x16": 8192, "group256x32": 8192, "group512x32": 16384,
            "group1024x32": 32768, "pair1024x32": 65536}


def _forced_plan(q, cfg, dtype, payload):
    """Every bin that cfg's tile holds takes cfg; the others the rounds."""
    names = [cfg if CAPACITY[cfg] >= (1 << b) else "block_qms" for b in range(q.QMS_BATCH_BINS)]
    q.qms_batched_set_plan(names, dtype=dtype, payload=payload)
    return names


@pytest.mark.parametrize("cfg", list(CAPACITY))
def test_every_group_configuration_vs_oracle(q, cfg):
    # Lengths across every bin up to the tile and a little beyond.
    L = [0, 1, 2, 3, 5, 16, 17, 31, 32, 33, 100, 511, 512, 513, 1000, 1024, 1025, 2047, 2048,
         2049, 4095, 4096, 4097, 8191, 8192, 8193, 12000, 16384, 16385, 20000, 32767, 32768,
         32769, 40000, 65535, 65536, 65537]
    L = np.array(L * 3, dtype=np.int64)
    np.random.default_rng(2).shuffle(L)
    off = gen.offsets_of(L)
    cases = [("u32", None), ("f32", None)] if cfg.endswith("x32") else \
        [("u32", None), ("f32", None), ("i64", None), ("u64", "pairs")]
    try:
        for dtype, extra in cases:
            payload = extra == "pairs"
            _forced_plan(q, cfg, dtype, payload)
            n = int(off[-1])
            k = gen.keys("mod16" if payload else ("normal" if dtype == "f32" else "uniform"), dtype, n, 5)
            d = _dev(k)
            doff = torch.from_numpy(off.view(np.int64)).cuda()
            if payload:
                v = gen.payload_index(n)
                dv = _dev(v)
                q.qms_sort_batched(d, doff, vals=dv, dtype=dtype)
                vo = _host(dv, "u32")
            else:
                q.qms_sort_batched(d, doff, dtype=dtype)
            out = _host(d, dtype)
            for i in range(len(L)):
                a, b = int(off[i]), int(off[i + 1])
                ref = oracle.reference_sorted(k[a:b])
                assert out[a:b].tobytes() == ref.tobytes(), (cfg, dtype, b - a)
                if payload:
                    assert np.array_equal(k[vo[a:b]], out[a:b]), (cfg, b - a)
                    assert np.array_equal(np.sort(vo[a:b]), np.arange(a, b, dtype=np.uint32))
    finally:
        for dtype, payload in (("u32", False), ("f32", False), ("i64", False), ("u64", True)):
            default = [min((c for c in CAPACITY if CAPACITY[c] >= (1 << b) and
                            (not c.endswith("x32") or (dtype in ("u32", "f32") and not payload))),
                           key=lambda c: CAPACITY[c], default="block_qms")
                       for b in range(q.QMS_BATCH_BINS)]
            q.qms_batched_set_plan(default, dtype=dtype, payload=payload)


def test_group_configuration_comparison_count(q):
    # The counting kernels of the group path report comparisons: at least
    # lg(n!) per segment (every comparison sort needs that many).
    L = np.array([300, 3000, 12000, 40] * 4, dtype=np.int64)
    off = gen.offsets_of(L)
    k = gen.keys("uniform", "u32", int(off[-1]), 8)
    d = _dev(k)
    st = q.qms_sort_batched(d, torch.from_numpy(off.view(np.int64)).cuda(), dtype="u32",
                            count_cmps=True)
    lg = sum(float(np.sum(np.log2(np.arange(2, m + 1)))) for m in L)
    assert lg < st["comparisons"] < 3 * lg


def test_autotuner_installs_and_stores_a_plan(q, tmp_path, monkeypatch):
    monkeypatch.setenv("QMS_AUTOTUNE_DIR", str(tmp_path))
    rep = q.qms_batched_autotune("u32")
    assert "ns/key" in rep and "plan written" in rep
    names, tuned = q.qms_batched_get_plan("u32")
    assert tuned
    for b, c in enumerate(names):
        assert c == "block_qms" or CAPACITY[c] >= (1 << b)
    files = list(tmp_path.glob("batched_k4_v0_sm*.json"))
    assert len(files) == 1
    sms = int(files[0].name.split("_sm")[1].split(".")[0])
    got, found = q.qms_batched_plan_read(str(files[0]), "u32", sm_count=sms)
    assert found and got[1:] == names[1:]
    # the tuned plan sorts correctly
    L = _lengths(4, 200)
    off = gen.offsets_of(L)
    k = gen.keys("uniform", "u32", int(off[-1]), 3)
    d = _dev(k)
    q.qms_sort_batched(d, torch.from_numpy(off.view(np.int64)).cuda(), dtype="u32")
    out = _host(d, "u32")
    for i in range(len(L)):
        a, b = int(off[i]), int(off[i + 1])
        assert out[a:b].tobytes() == np.sort(k[a:b]).tobytes()
