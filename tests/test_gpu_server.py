"""GPU tests of the served form: continuous batching under an HBM budget.
Each result must equal that request's sort alone (and the oracle's plain
definition of the result), whatever else was in flight."""
import numpy as np
import pytest

import oracle
import qms_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"u32": torch.int32, "f32": torch.float32, "u64": torch.int64, "i64": torch.int64}
NP = {"u32": np.uint32, "u64": np.uint64, "i64": np.int64, "f32": np.float32}


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_10062_gb300 as q
    q.lib()
    return q


def _t(a, device, pin=False):
    v = a.view({4: np.int32, 8: np.int64}[a.itemsize]) if a.dtype != np.float32 else a
    t = torch.from_numpy(v.copy())
    if device == "cuda":
        return t.cuda()
    return t.pin_memory() if pin else t


def test_mixed_requests_equal_alone(q):
    rng = np.random.default_rng(1)
    reqs = []
    sizes = [10, 300, 5000, 8192, 20000, 65536, 100003, 600001, 7, 2, 1, 0]
    for i in range(60):
        n = int(sizes[i % len(sizes)] if i < len(sizes) else int(2 ** rng.uniform(4, 17)))
        dtype = ["u32", "u64", "f32", "i64"][i % 4]
        dist = "normal" if dtype == "f32" else ("mod16" if i % 5 == 0 and dtype == "u64" else "uniform")
        k = gen.keys(dist, dtype, n, 100 + i)
        mode = ["host_pinned", "host_pageable", "dev_inplace", "dev_copy"][i % 4]
        reqs.append((n, dtype, k, mode))
    with q.QmsServer(1 << 30, max_slots=64, workers=3, max_batch=32) as srv:
        live = []
        for n, dtype, k, mode in reqs:
            if mode.startswith("host"):
                src = _t(k, "cpu", pin=(mode == "host_pinned"))
                dst = torch.empty_like(src)
                if mode == "host_pinned":
                    dst = dst.pin_memory()
                ip, op = src.data_ptr(), dst.data_ptr()
            elif mode == "dev_inplace":
                src = _t(k, "cuda")
                dst = src
                ip = op = src.data_ptr()
            else:
                src = _t(k, "cuda")
                dst = torch.empty_like(src)
                ip, op = src.data_ptr(), dst.data_ptr()
            torch.cuda.synchronize()
            t = srv.qms_server_submit(ip, op, n, dtype)
            live.append((t, n, dtype, k, src, dst))
        for t, n, dtype, k, src, dst in live:
            info = srv.qms_server_wait(t, 120000.0)
            assert info["status"] == 0
            got = dst.cpu().numpy().view(NP[dtype]) if n else np.empty(0, NP[dtype])
            assert got.tobytes() == oracle.reference_sorted(k).tobytes(), (n, dtype)
            if n > 1:
                alone = _t(k, "cuda")
                q.qms_sort(alone, dtype=dtype)
                assert alone.cpu().numpy().view(NP[dtype]).tobytes() == got.tobytes()
        st = srv.qms_server_get_stats()
        assert st["completed"] == len(reqs)
        assert st["used_bytes"] == 0 and st["in_flight"] == 0


def test_budget_admission(q):
    # Tight budget: 6 MiB for requests of ~1 MiB each -> never more than the
    # budget held at once, all finish.
    budget = 6 << 20
    with q.QmsServer(budget, max_slots=1000, workers=4, max_batch=8) as srv:
        ks, ts = [], []
        for i in range(40):
            n = 250000
            k = gen.keys("uniform", "u32", n, i)
            src = _t(k, "cpu", pin=True)
            dst = torch.empty_like(src).pin_memory()
            ts.append(srv.qms_server_submit(src.data_ptr(), dst.data_ptr(), n, "u32"))
            ks.append((k, src, dst))
        for t, (k, src, dst) in zip(ts, ks):
            assert srv.qms_server_wait(t)["status"] == 0
            assert dst.numpy().view(np.uint32).tobytes() == np.sort(k).tobytes()
        st = srv.qms_server_get_stats()
        assert 0 < st["peak_used_bytes"] <= budget
        with pytest.raises(q.QmsError) as e:
            big = torch.empty(4 << 20, dtype=torch.int32).pin_memory()
            srv.qms_server_submit(big.data_ptr(), big.data_ptr(), big.numel(), "u32")
        assert e.value.code == q.QMS_EBUDGET


def test_poll_releases_ticket(q):
    with q.QmsServer(1 << 28, workers=1) as srv:
        k = gen.keys("uniform", "u32", 1000, 3)
        d = _t(k, "cuda")
        t = srv.qms_server_submit(d.data_ptr(), d.data_ptr(), 1000, "u32")
        info = None
        for _ in range(200000):
            info = srv.qms_server_poll(t)
            if info is not None:
                break
        assert info is not None and info["status"] == 0
        with pytest.raises(q.QmsError):
            srv.qms_server_poll(t)


def test_bounded_wait_times_out_while_paused(q):
    # Failure made on the host: the server is paused, so a queued request
    # cannot finish; the bounded wait returns QMS_ETIMEOUT and the request
    # completes normally once the server resumes.
    with q.QmsServer(1 << 28, workers=2) as srv:
        srv.qms_server_pause(True)
        k = gen.keys("uniform", "u32", 50000, 5)
        d = _t(k, "cuda")
        t = srv.qms_server_submit(d.data_ptr(), d.data_ptr(), len(k), "u32")
        with pytest.raises(q.QmsError) as e:
            srv.qms_server_wait(t, 50.0)
        assert e.value.code == q.QMS_ETIMEOUT
        assert srv.qms_server_poll(t) is None
        srv.qms_server_pause(False)
        assert srv.qms_server_wait(t, 60000.0)["status"] == 0
        assert d.cpu().numpy().view(np.uint32).tobytes() == np.sort(k).tobytes()
