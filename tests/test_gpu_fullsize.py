"""GPU parity at the full sizes of the benchmark configurations.

The oracle cannot sort 2^27..2^28 keys within test time, so these cases are
checked through properties that hold at any size, each against the input:

* ascending order of the output;
* the multiset of keys: order-free signatures of the key bit patterns (sum,
  sum of squares and xor, all mod 2^64);
* sampled ranks computed one by one from the input: for y = out[i],
  count(input < y) <= i < count(input <= y);
* for key-value pairs: the payloads (original indices) form a permutation
  and every output key equals the input key at its payload.

The plain sort runs through the same entry point that bench.py times (a
waiting qms_sort call, host-driven rounds at these sizes); one case runs the
device-driven graph at full size as well."""
import numpy as np
import pytest

import oracle
import qms_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NP = {"u32": np.uint32, "u64": np.uint64, "i64": np.int64, "f32": np.float32}
BITS = {"u32": np.uint32, "u64": np.uint64, "i64": np.uint64, "f32": np.uint32}


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_10062_gb300 as q
    q.lib()
    return q


def _dev(a):
    view = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}.get(a.dtype)
    return torch.from_numpy(a.view(view) if view is not None else a).cuda()


def _host(t, dtype):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(NP[dtype])


def _signature(a, dtype):
    b = a.view(BITS[dtype]).astype(np.uint64)
    return (int(np.add.reduce(b, dtype=np.uint64)),
            int(np.add.reduce(b * b, dtype=np.uint64)),
            int(np.bitwise_xor.reduce(b)))


def _check_keys(inp, out, dtype, samples=24, seed=0):
    assert out.shape == inp.shape
    assert np.all(out[1:] >= out[:-1]), "output not ascending"
    assert _signature(out, dtype) == _signature(inp, dtype), "key multiset changed"
    rng = np.random.default_rng(seed)
    n = inp.size
    idx = np.concatenate([[0, n - 1, n // 2], rng.integers(0, n, samples - 3)])
    for i in idx:
        y = out[i]
        lo = int(np.count_nonzero(inp < y))
        hi = int(np.count_nonzero(inp <= y))
        assert lo <= i < hi, (int(i), lo, hi)


@pytest.mark.parametrize("dtype,dist,pivot,seed", [
    ("u32", "uniform", "m3", 2),      # the benchmark workload itself
    ("i64", "uniform", "hybrid", 3),
    ("f32", "normal", "sqrtn", 4),
    ("u32", "uniform", "mom", 5),     # the worst-case-guaranteed variant (Sec. 4)
])
def test_full_size_2_28(q, dtype, dist, pivot, seed):
    n = 1 << 28
    k = gen.keys(dist, dtype, n, seed)
    d = _dev(k)
    q.qms_sort(d, pivot=pivot, dtype=dtype)  # a waiting call: host-driven rounds at this size
    out = _host(d, dtype)
    del d
    _check_keys(k, out, dtype, seed=seed)


def test_full_size_2_28_device_driven(q):
    # The same workload as the benchmark through the device-driven graph (an
    # asynchronous call, which always takes the graph).
    n = 1 << 28
    k = gen.keys("uniform", "u32", n, 2)
    d = _dev(k)
    q.qms_sort(d, pivot="m3", dtype="u32", wait=False)
    out = _host(d, "u32")
    del d
    _check_keys(k, out, "u32", seed=2)


@pytest.mark.parametrize("dist", ["uniform", "mod16", "sorted", "reverse", "organ", "killer"])
def test_full_size_pairs_2_27(q, dist):
    # 2^27 uint64 keys with uint32 payload = original index, hybrid pivot.
    n = 1 << 27
    if dist == "killer":
        k32, _ = oracle.adversary_u32(n, "hybrid", "paper")
        k = k32.astype(np.uint64)
    else:
        k = gen.keys(dist, "u64", n, 9)
    dk = _dev(k)
    dv = torch.arange(n, dtype=torch.int32, device="cuda")
    q.qms_sort_pairs(dk, dv, pivot="hybrid", dtype="u64")
    torch.cuda.synchronize()
    # payload permutation and key/payload consistency on the device
    p = dv.to(torch.int64)
    assert int(p.min()) == 0 and int(p.max()) == n - 1
    mark = torch.zeros(n, dtype=torch.int32, device="cuda")
    mark[p] = 1
    assert int(mark.sum()) == n, "payloads are not a permutation"
    dk_in = _dev(k)
    assert bool(torch.equal(dk, dk_in[p])), "a key does not match its payload's input key"
    del mark, dk_in, p
    out = _host(dk, "u64")
    _check_keys(k, out, "u64", seed=7)
