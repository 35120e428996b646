"""Sharding of independent units over ranks (CPU, gloo, world size 2): every
unit is assigned exactly once, the LPT loads are balanced, and the ranks'
results (the oracle on each rank's share) cover the whole batch."""
import os

import numpy as np
import pytest

import qms_inputs as gen
from paper_1804_10062_gb300 import shard


def test_lpt_covers_and_balances():
    L = gen.batch_lengths(65536, 1, 16, 65536)
    for world in (1, 2, 4, 8):
        a = shard.lpt_assign(L, world)
        allidx = np.sort(np.concatenate(a))
        assert np.array_equal(allidx, np.arange(len(L)))
        loads = shard.rank_loads(L, a)
        assert max(loads) <= min(loads) * 1.01 + shard.unit_cost(65536)


def test_local_segments_pack():
    L = np.array([5, 0, 7, 3], dtype=np.int64)
    off = gen.offsets_of(L)
    loc, b, e = shard.local_segments(off, np.array([0, 2]))
    assert loc.tolist() == [0, 5, 12]
    assert b.tolist() == [0, 5] and e.tolist() == [5, 12]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L = gen.batch_lengths(200, 4, 16, 4096)
    off = gen.offsets_of(L)
    keys = gen.keys("uniform", "u32", int(off[-1]), 8)
    mine = shard.lpt_assign(L, world)[rank]
    done = {}
    for i in mine:
        seg = keys[int(off[i]):int(off[i + 1])].copy()
        oracle.sort(seg, variant="hybrid", mode="paper")
        done[int(i)] = int(np.bitwise_xor.reduce(seg.astype(np.uint64) * np.arange(1, len(seg) + 1,
                                                                                  dtype=np.uint64)))
    gathered = [None] * world
    dist.all_gather_object(gathered, done)
    if rank == 0:
        merged = {}
        for d in gathered:
            assert not (set(d) & set(merged))
            merged.update(d)
        ok = sorted(merged) == list(range(len(L)))
        for i in range(len(L)):
            ref = np.sort(keys[int(off[i]):int(off[i + 1])]).astype(np.uint64)
            h = int(np.bitwise_xor.reduce(ref * np.arange(1, len(ref) + 1, dtype=np.uint64)))
            ok = ok and merged[i] == h
        q.put(ok)
    dist.destroy_process_group()


def test_two_rank_gloo_shard():
    torch = pytest.importorskip("torch")
    import socket
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = mp.Queue()
    ps = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    assert q.get(timeout=10) is True
