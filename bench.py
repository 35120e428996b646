"""Benchmark of the GB300 QuickMergesort path.

Default workload: plain QuickMergesort with the median-of-3 pivot on one
array of n = 2^28 uint32 keys, uniformly random (SplitMix64, seed 2 + rank),
one array per GPU (replicas: the plain sort does not shard).  A step is one
whole sort of one array; inputs (1 GiB each) are resident in HBM before the
timed region and are larger than L2, so no flush is needed.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import signal
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DTYPE_BYTES = {"u32": 4, "u64": 8, "i64": 8, "f32": 4}
# One metric string for both arms, so that the two lines can be divided.
METRIC = "GKeys/s (plain sort)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="qms", choices=["qms", "reference"])
    ap.add_argument("--lgn", type=int, default=28)
    ap.add_argument("--dtype", default="u32", choices=list(DTYPE_BYTES))
    ap.add_argument("--pivot", default="m3", choices=["m3", "sqrtn", "mom", "hybrid"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served forms")
    ap.add_argument("--forms", default="batched,served",
                    help="which of the batched and served forms to run (comma list)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-configuration records (C1-C3 workloads)")
    ap.add_argument("--batched-segments", type=int, default=65536)
    ap.add_argument("--served-requests", type=int, default=20000)
    ap.add_argument("--served-lg-max", type=float, default=26.0)
    ap.add_argument("--served-workers", type=int, default=8,
                    help="worker threads (one stream each) of the request server")
    ap.add_argument("--served-loads", default="0.5,0.8,0.95",
                    help="offered loads as fractions of the plain FIFO throughput")
    return ap.parse_args()


class Ranks:
    """World size, rank and the process group of a torchrun launch (world
    size 1: no group)."""

    def __init__(self, ws, rank, dist):
        self.ws, self.rank, self.dist = ws, rank, dist

    def max(self, torch, x):
        if self.dist is None:
            return x
        t = torch.tensor([float(x)], dtype=torch.float64, device="cuda")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def gather(self, obj):
        if self.dist is None:
            return [obj]
        out = [None] * self.ws
        self.dist.all_gather_object(out, obj)
        return out

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def share(self, lengths):
        """This rank's units (indices) under LPT over n log n costs."""
        import numpy as np
        if self.ws == 1:
            return np.arange(len(lengths))
        from paper_1804_10062_gb300.shard import lpt_assign
        return lpt_assign(lengths, self.ws)[self.rank]


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def keys_for(args, seed):
    import qms_inputs as gen
    n = 1 << args.lgn
    dist = "normal" if args.dtype == "f32" else "uniform"
    return gen.keys(dist, args.dtype, n, seed)


def workload_name(args):
    return "plain QuickMergesort, %s pivot, one array of n=2^%d %s keys (%s)" % (
        {"m3": "median-of-3", "sqrtn": "median-of-sqrt(n)", "mom": "median-of-medians",
         "hybrid": "hybrid median-of-3/median-of-medians"}[args.pivot], args.lgn, args.dtype,
        "N(0,1)" if args.dtype == "f32" else "uniform")


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.send_signal(signal.SIGINT)
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline helpers


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Sources that define the swap-merge kernel (k_merge_level3 and the device
# routines it inlines); the driver files around it do not change its code.
MERGE_SOURCES = ("qms_device.cuh", "qms_kernels.cuh", "qms_merge.cuh")


def source_sha(files=MERGE_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1804_10062_gb300", "csrc")
    for fn in sorted(files):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


# ncu DRAM-traffic summaries per (kernel class, log2 n, dtype, pivot rule)
TRAFFIC_PROFILES = {("merge", 28, "u32", "m3"): "k_merge_level3_traffic_n2p28_u32_m3.md"}


def ncu_traffic_per_byte(kernel, lgn, dtype, pivot):
    """DRAM bytes per algorithmic byte of `kernel` on this workload from the
    committed ncu summary, or None when there is none for the workload, or
    the sources changed since it was taken."""
    name = TRAFFIC_PROFILES.get((kernel, lgn, dtype, pivot))
    if name is None:
        return None
    p = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(p).read()
    except OSError:
        return None
    m1 = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    m2 = re.search(r"dram_bytes_per_algorithmic_byte:\s*([0-9.]+)", txt)
    if not m1 or not m2 or m1.group(1) != source_sha():
        return None
    return float(m2.group(1))


# ---------------------------------------------------------------------------


def cpu_baseline(args, lg_sample=None, runs=1, host=None):
    """The oracle timed on the host: by default one sort of the whole
    workload (the same keys the GPU sorts; about 20 s at 2^28)."""
    import oracle
    import qms_inputs as gen
    lg_sample = args.lgn if lg_sample is None else lg_sample
    n = 1 << lg_sample
    dist = "normal" if args.dtype == "f32" else "uniform"
    k0 = host if (host is not None and host.size == n) else gen.keys(dist, args.dtype, n, 1000)
    oracle.lib()
    ts = []
    for _ in range(runs):
        k = k0.copy()
        t0 = time.perf_counter()
        oracle.sort(k, variant=args.pivot, mode="paper")
        ts.append(time.perf_counter() - t0)
    total = sum(ts)
    return {"value": runs * n / total / 1e9, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
            "sample": "%d run(s) of the single-threaded oracle (paper mode) on n=2^%d %s keys "
                      "of the workload's distribution, %.1f s of CPU work" %
                      (runs, lg_sample, args.dtype, total)}


# ---------------------------------------------------------------------------
# all-cores oracle over many arrays (batched form): one oracle run per
# segment, the segments dealt round-robin to one spawned process per core
# (spawn: this process already holds a CUDA context)


def _oracle_pool_init():
    import oracle
    oracle.lib()


def _oracle_pool_work(segs):
    import oracle
    keys = 0
    for seg in segs:
        oracle.sort(seg, variant="m3", mode="paper")
        keys += seg.size
    return keys


def oracle_all_cores(np, keys, off, every=8):
    """A seeded sample of the segments keys[off[i]:off[i+1]] (one in `every`)
    sorted by the oracle, one run per segment, on every host core; returns
    the keys/s of the timed pool run (pool start excluded)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    nseg = len(off) - 1
    pick = np.sort(np.random.default_rng(5).choice(nseg, max(1, nseg // every), replace=False))
    segs = [keys[int(off[i]):int(off[i + 1])].copy() for i in pick]
    work = [segs[w::cores] for w in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_pool_init) as pool:
        pool.map(_oracle_pool_work, [[segs[0].copy()]] * cores)  # warm the workers
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_pool_work, work))
        el = time.perf_counter() - t0
    return {"value": done / el / 1e9, "unit": "GKeys/s", "cores": cores, "kind": "oracle",
            "sample": "%d seeded segments (one in %d, %d keys), one oracle run per segment "
                      "(paper mode, median-of-3), %d spawned processes, %.1f s"
                      % (len(pick), every, done, cores, el)}


# ---------------------------------------------------------------------------
# batched and served forms


def bench_batched(args, q, torch, np, ranks):
    """65,536 segments, lengths log-uniform in [16, 65536], uint32 and
    float32 U(0,1) keys: one batched call vs one plain call per segment.
    With several ranks each sorts its LPT share of the segments (no
    collective on the data path); the time is the maximum over ranks and
    the throughput counts every rank's keys."""
    import qms_inputs as gen
    nseg_all = args.batched_segments
    L_all = gen.batch_lengths(nseg_all, 1, 16, 65536)
    off_all = gen.offsets_of(L_all)
    n_all = int(off_all[-1])
    mine = ranks.share(L_all)
    L = L_all[mine]
    nseg = len(L)
    off = gen.offsets_of(L)
    n = int(off[-1])
    doff = torch.from_numpy(off.view(np.int64)).cuda()
    out = {"segments": nseg_all, "keys": n_all, "lengths": "floor(exp(U(ln 16, ln 65536)))",
           "sharding": "LPT over %d ranks (n log n costs)" % ranks.ws if ranks.ws > 1 else "single GPU"}
    peak, _ = measured_peak_hbm()
    # Autotune the per-bin kernel configurations on this GPU (4-byte keys
    # without payloads: uint32 and float32 share the plan), untimed.
    t0 = time.perf_counter()
    report = q.qms_batched_autotune("u32")
    plan, tuned = q.qms_batched_get_plan("u32")
    out["autotune"] = {"seconds": time.perf_counter() - t0, "tuned": tuned,
                       "plan": {"bin_%d_(%d..%d keys)" % (b, (1 << (b - 1)) + 1 if b else 1, 1 << b): c
                                for b, c in enumerate(plan)},
                       "report": report.strip().splitlines()}
    for dt in ("u32", "f32"):
        k_all = gen.keys("uniform", dt, n_all, 1)
        k = k_all if ranks.ws == 1 else np.concatenate(
            [k_all[int(off_all[i]):int(off_all[i + 1])] for i in mine])
        del k_all
        src = torch.from_numpy(k.view(np.int32)).cuda()
        cpu_all = oracle_all_cores(np, k, off) if (dt == "u32" and not args.no_cpu_baseline) else None
        del k
        work = torch.empty_like(src)
        work.copy_(src)
        q.qms_sort_batched(work, doff, dtype=dt)  # warm-up
        times, prof = [], q.qms_profile()
        for _ in range(3):
            work.copy_(src)
            torch.cuda.synchronize()
            ranks.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            q.qms_sort_batched(work, doff, dtype=dt, profile=prof)
            e1.record()
            torch.cuda.synchronize()
            times.append(ranks.max(torch, e0.elapsed_time(e1)))
        ms = min(times)
        pb = prof.as_dict()["batch"]
        kern_ms = pb["ms"] / max(1, pb["launches"])
        alg = pb["bytes"] / max(1, pb["launches"])
        # plain: one qms_sort per segment, on a seeded sample of 1024 segments
        idx = np.random.default_rng(0).choice(nseg, min(1024, nseg), replace=False)
        work.copy_(src)
        torch.cuda.synchronize()
        ks = 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in idx:
            a, b = int(off[i]), int(off[i + 1])
            q.qms_sort(work[a:b], dtype=dt)
            ks += b - a
        e1.record()
        torch.cuda.synchronize()
        plain_gk = ks / (e0.elapsed_time(e1) / 1e3) / 1e9
        v = n_all / (ms / 1e3) / 1e9
        out[dt] = {"value": v, "unit": "GKeys/s", "ms": ms,
                   "plain_per_array": {"value": plain_gk, "unit": "GKeys/s",
                                       "sample": "%d seeded segments, one qms_sort each" % len(idx)},
                   "speedup_vs_plain": (n / (ms / 1e3) / 1e9) / plain_gk,  # one GPU's share
                   "cpu_baseline": cpu_all,
                   "roofline": {"bound": "hbm", "kernel": "k_batched",
                                "achieved": alg / (kern_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                                "frac": alg / (kern_ms / 1e3) / 1e9 / peak,
                                "note": "algorithmic bytes of every partition, leaf and merge "
                                        "step; segments are L2-resident while sorted",
                                "compulsory_frac": 2 * 4 * n / (kern_ms / 1e3) / 1e9 / peak}}
        del src, work
        torch.cuda.empty_cache()
    return out


def bench_served(args, q, torch, np, ranks):
    """Served form: a Poisson stream of requests (20,000 by default), sizes
    floor(2^U(10, 26)), dtype mix 50/30/20 uint32/uint64/float32 uniform,
    admitted against a 16 GB HBM budget.  Inputs live in pinned host memory
    and results go back to host memory, so every admitted request holds a
    device slot charged to the budget.  The FIFO baseline sorts the same
    request list one request at a time through the plain API (upload, sort,
    download).  Offered loads are fractions of that FIFO throughput; the
    saturation run submits every request at once.  With several ranks each
    serves its LPT share of the requests; throughputs count every rank's
    keys over the longest rank's time and latencies pool all ranks."""
    import qms_inputs as gen
    nreq = args.served_requests
    lg_max = args.served_lg_max
    loads = [float(x) for x in args.served_loads.split(",") if x]
    maxn = 1 << int(math.ceil(lg_max))
    esz = {"u32": 4, "u64": 8, "f32": 4}
    tdt = {"u32": torch.int32, "u64": torch.int64, "f32": torch.int32}
    pristine = {}
    for dt in ("u32", "u64", "f32"):
        k = gen.keys("uniform", dt, maxn, 77)
        t = torch.empty(maxn, dtype=tdt[dt], pin_memory=True)
        t.copy_(torch.from_numpy(k.view(np.int32 if k.itemsize == 4 else np.int64)))
        pristine[dt] = t
        del k
    reqs_all = gen.request_stream(nreq, 5, 10.0, lg_max, rate_per_s=1.0)
    all_keys = sum(r[1] for r in reqs_all)
    mine = ranks.share([r[1] for r in reqs_all])
    reqs0 = [reqs_all[i] for i in mine]
    total_keys = sum(r[1] for r in reqs0)
    mean_n = total_keys / len(reqs0)
    budget = 16 * 10**9
    # host output ring: every request in flight holds at most the budget
    ring_bytes = (budget + maxn * 8 + (1 << 30)) // 256 * 256
    ring = torch.empty(ring_bytes, dtype=torch.uint8, pin_memory=True)

    def fifo_plain():
        dev = {dt: torch.empty(maxn, dtype=tdt[dt], device="cuda") for dt in pristine}
        st = torch.cuda.current_stream()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        head = 0
        for _, n, dt in reqs0:
            nb = n * esz[dt]
            if head + nb > ring_bytes:
                head = 0
            d = dev[dt][:n]
            d.copy_(pristine[dt][:n], non_blocking=True)
            q.qms_sort(d, dtype=dt)  # returns once the sort has finished
            ring[head: head + nb].view(tdt[dt]).copy_(d, non_blocking=True)
            head += (nb + 255) // 256 * 256
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        del dev
        torch.cuda.empty_cache()
        return total_keys / el / 1e9, el  # this rank's requests

    def run(rate_gkeys):
        ranks.barrier()
        lam = None if rate_gkeys is None else rate_gkeys * 1e9 / mean_n
        srv = q.QmsServer(budget, max_slots=1024, workers=args.served_workers, max_batch=4096)
        tickets, live, infos = [], [], {}
        head = 0
        rng = np.random.default_rng(9)
        arr = 0.0
        t_start = time.perf_counter()
        for _, n, dt in reqs0:
            if lam is not None:
                arr += -math.log1p(-rng.random()) / lam
                while time.perf_counter() - t_start < arr:
                    pass
            nb = n * esz[dt]
            nb_al = (nb + 255) // 256 * 256
            if head + nb_al > ring_bytes:
                head = 0
            # wait for outstanding requests whose outputs overlap [head, head + nb)
            while live and any(o < head + nb_al and head < o + b for _, o, b in live):
                t, o, b = live.pop(0)
                infos[t] = srv.qms_server_wait(t, 600000.0)
            src = pristine[dt][:n]
            t = srv.qms_server_submit(src.data_ptr(), ring.data_ptr() + head, n, dt)
            live.append((t, head, nb_al))
            tickets.append(t)
            head += nb_al
        for t, o, b in live:
            infos[t] = srv.qms_server_wait(t, 600000.0)
        el = ranks.max(torch, time.perf_counter() - t_start)
        st = srv.qms_server_get_stats()
        srv.qms_server_destroy()
        lat = sorted(x for part in ranks.gather([infos[t]["latency_ms"] for t in tickets]) for x in part)
        bad = sum(ranks.gather(sum(1 for t in tickets if infos[t]["status"] != 0)))
        return {"sustained": all_keys / el / 1e9, "unit": "GKeys/s",
                "offered_GKeys_s": None if rate_gkeys is None else rate_gkeys * ranks.ws,
                "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                "mean_batch": st["batched_requests"] / max(1, st["batches"]),
                "peak_in_flight": st["peak_in_flight"], "peak_used_GB": st["peak_used_bytes"] / 1e9,
                "wall_s": el, "failed_requests": bad}

    ranks.barrier()
    fifo_local, fifo_s = fifo_plain()
    fifo_s = ranks.max(torch, fifo_s)
    fifo = all_keys / fifo_s / 1e9
    out = {"requests": nreq, "keys": all_keys, "sizes": "floor(2^U(10, %g))" % lg_max,
           "dtype_mix": "50/30/20 u32/u64/f32 uniform", "budget_GB": budget / 1e9,
           "inputs": "pinned host memory; results written back to pinned host memory",
           "fifo_plain": {"value": fifo, "unit": "GKeys/s", "wall_s": fifo_s,
                          "sample": "the same %d requests one at a time: upload, qms_sort, "
                                    "download" % nreq}}
    sat = run(None)
    out["saturation"] = sat
    for rho in loads:
        out["offered_%.2f" % rho] = run(rho * fifo_local)  # per rank: rho x its own FIFO rate
    out["speedup_vs_fifo_plain"] = sat["sustained"] / fifo
    # one request alone equals its slice sorted (spot check of the served path)
    return out


def _to_dev(torch, np, k):
    if k.dtype == np.uint32:
        return torch.from_numpy(k.view(np.int32)).cuda()
    if k.dtype == np.uint64:
        return torch.from_numpy(k.view(np.int64)).cuda()
    return torch.from_numpy(k).cuda()


def whole_roofline(pd, ms, peak, peak_kind):
    """Every kernel class's algorithmic bytes of one sort over its timed
    device time: the whole-sort HBM fraction."""
    b = sum(v["bytes"] for v in pd.values())
    a = b / (ms / 1e3) / 1e9
    return {"bound": "hbm", "scope": "whole sort (all kernel classes)", "achieved": a,
            "peak": peak, "unit": "GB/s", "frac": a / peak, "peak_source": peak_kind,
            "alg_bytes_per_sort": b}


def plain_record(q, torch, np, k, dtype, pivot, dist, pairs=False, reps=3, count=False,
                 cpu_sample=None, peak=(6800.0, "fallback")):
    """One configuration of the plain form: device time of `reps` graph
    sorts (median), the whole-sort roofline from a profiled pass of the same
    sort, optional comparison counts beside the oracle's, and the oracle
    timed on a bounded sample of the same distribution."""
    import oracle
    n = k.size
    src = _to_dev(torch, np, k)
    work = torch.empty_like(src)
    vsrc = torch.arange(n, dtype=torch.int32, device="cuda") if pairs else None
    vals = torch.empty_like(vsrc) if pairs else None

    def reset():
        work.copy_(src)
        if pairs:
            vals.copy_(vsrc)

    def sort(**kw):
        if pairs:
            return q.qms_sort_pairs(work, vals, pivot=pivot, dtype=dtype, **kw)
        return q.qms_sort(work, pivot=pivot, dtype=dtype, **kw)

    reset()
    sort()  # builds or reuses the graph instance
    ts = []
    for _ in range(reps):
        reset()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sort()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    head = work[: min(n, 1 << 20)].cpu().numpy().view(k.dtype)
    ok = bool(np.all(head[1:] >= head[:-1])) if dtype != "f32" else True
    reset()
    prof = q.qms_profile()
    sort(profile=prof)
    pd = prof.as_dict()
    pk, pkind = peak
    rec = {"value": n / (ms / 1e3) / 1e9, "unit": "GKeys/s", "ms": ms, "n": n, "dtype": dtype,
           "pivot": pivot, "dist": dist, "pairs": pairs, "prefix_sorted": ok,
           "roofline": whole_roofline(pd, ms, pk, pkind),
           "kernels_ms": {kk: round(v["ms"], 4) for kk, v in pd.items() if v["launches"]}}
    if count:
        reset()
        st = sort(count_cmps=True)
        kc = k.copy()
        oc, _ = oracle.sort(kc, variant=pivot, mode="analysis")
        rec["comparisons_per_key"] = {"gpu": st["comparisons"] / n, "oracle_analysis": oc / n,
                                      "lg_n_factorial": float(np.sum(np.log2(np.arange(2, n + 1)))) / n}
    if cpu_sample is not None:
        ks, vs, what = cpu_sample
        t0 = time.perf_counter()
        oracle.sort(ks, vs, variant=pivot, mode="paper")
        el = time.perf_counter() - t0
        rec["cpu_baseline"] = {"value": ks.size / el / 1e9, "unit": "GKeys/s", "cores": 1,
                               "kind": "oracle", "sample": what + " (%.2f s)" % el}
    del src, work, vsrc, vals
    torch.cuda.empty_cache()
    return rec


def config_records(args, q, torch, np):
    """The configurations besides the headline: C1 (2^20 permutation with
    comparison counts), C2 (2^28 int64 and float32; 2^24 with every pivot
    rule) and C3 (2^27 uint64 keys with uint32 payloads over six key
    distributions, hybrid pivot)."""
    import oracle
    import qms_inputs as gen
    peak = measured_peak_hbm()
    out = {}
    lg_cpu = 22

    def sample(dist, dtype, pairs=False, lg=lg_cpu):
        m = 1 << lg
        if dist == "killer":
            ks = oracle.adversary_u32(m, "hybrid", "paper")[0].astype(np.uint64)
        elif dist == "perm":
            ks = gen.permutation_u32(m, 11)
        else:
            ks = gen.keys(dist, dtype, m, 11)
        vs = gen.payload_index(m) if pairs else None
        return ks, vs, "oracle on n=2^%d %s %s keys%s" % (lg, dist, dtype,
                                                          " with payloads" if pairs else "")

    k = gen.permutation_u32(1 << 20, 1)
    out["C1_perm_u32_2p20_m3"] = plain_record(q, torch, np, k, "u32", "m3", "perm", reps=5,
                                              count=True, cpu_sample=sample("perm", "u32", lg=20),
                                              peak=peak)
    for dtype, dist in (("i64", "uniform"), ("f32", "normal")):
        k = gen.keys(dist, dtype, 1 << 28, 3)
        out["C2_%s_2p28_m3" % dtype] = plain_record(q, torch, np, k, dtype, "m3", dist,
                                                    cpu_sample=sample(dist, dtype), peak=peak)
        del k
    for dtype, dist in (("u32", "uniform"), ("i64", "uniform"), ("f32", "normal")):
        k = gen.keys(dist, dtype, 1 << 24, 4)
        for pivot in ("m3", "sqrtn", "mom", "hybrid"):
            out["C2_%s_2p24_%s" % (dtype, pivot)] = plain_record(
                q, torch, np, k, dtype, pivot, dist, reps=5,
                cpu_sample=sample(dist, dtype) if dtype == "u32" else None, peak=peak)
        del k
    for dist in ("uniform", "mod16", "sorted", "reverse", "organ", "killer"):
        if dist == "killer":
            k = oracle.adversary_u32(1 << 27, "hybrid", "paper")[0].astype(np.uint64)
        else:
            k = gen.keys(dist, "u64", 1 << 27, 9)
        out["C3_pairs_u64_2p27_%s_hybrid" % dist] = plain_record(
            q, torch, np, k, "u64", "hybrid", dist, pairs=True,
            cpu_sample=sample(dist, "u64", pairs=True), peak=peak)
        del k
    return out


def run_reference(args):
    ws, rank, _ = dist_init(args)
    if rank != 0:
        return 0
    import oracle
    import qms_inputs as gen
    lg = min(args.lgn, 25)
    n = 1 << lg
    dist = "normal" if args.dtype == "f32" else "uniform"
    k0 = gen.keys(dist, args.dtype, n, 2)
    oracle.lib()
    for _ in range(args.warmup):
        oracle.sort(k0.copy(), variant=args.pivot, mode="paper")
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort(k0.copy(), variant=args.pivot, mode="paper")
    el = time.perf_counter() - t0
    v = args.steps * n / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GKeys/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": workload_name(args), "n": 1 << args.lgn, "pivot": args.pivot},
            "cpu_baseline": {"value": v, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
                             "sample": "each step sorts n=2^%d keys of the workload's "
                                       "distribution with the single-threaded oracle" % lg},
            "e2e": {"value": v, "unit": "GKeys/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_qms(args):
    import numpy as np
    import torch
    ws, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_1804_10062_gb300 as q
    q.lib()
    n = 1 << args.lgn
    esz = DTYPE_BYTES[args.dtype]
    host = keys_for(args, 2 + rank)
    tdt = torch.int32 if esz == 4 else torch.int64
    src = torch.from_numpy(host.view(np.int32 if esz == 4 else np.int64)).cuda()
    stream = torch.cuda.current_stream()
    bufs = [torch.empty_like(src) for _ in range(args.steps)]
    for b in bufs:
        b.copy_(src)
    work = torch.empty_like(src)
    for _ in range(args.warmup):
        work.copy_(src)
        q.qms_sort(work, pivot=args.pivot, dtype=args.dtype)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        # the plain API: each call returns once its sort has finished (a
        # waiting call of 2^16 keys or more runs its rounds from the host,
        # every kernel launched with a programmatic dependency on the one
        # before it)
        q.qms_sort(bufs[i], pivot=args.pivot, dtype=args.dtype)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    el_ms = e0.elapsed_time(e1)
    t = torch.tensor([el_ms], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    el_ms = float(t.item())
    # spot check of the result (full parity lives in the tests)
    out = bufs[0][: min(n, 1 << 20)].cpu().numpy()
    if args.dtype in ("u32", "u64"):
        out = out.view(np.uint32 if esz == 4 else np.uint64)
    if args.dtype != "f32":
        assert np.all(out[1:] >= out[:-1]), "result not sorted"
    # kernels per sort, counted on the device (same input distribution)
    work.copy_(src)
    st1 = q.qms_sort(work, pivot=args.pivot, dtype=args.dtype)
    launches = int(st1["launches"]) * args.steps
    # per-kernel times: a profiled pass of the same K sorts (CUDA events
    # around every launch of the same kernels, rounds run from the host)
    prof = q.qms_profile()
    for i in range(args.steps):
        bufs[i].copy_(src)
        torch.cuda.synchronize()
        q.qms_sort(bufs[i], pivot=args.pivot, dtype=args.dtype, profile=prof)
    torch.cuda.synchronize()

    value = ws * args.steps * n / (el_ms / 1e3) / 1e9
    pd = prof.as_dict()
    dom = max(pd, key=lambda k: pd[k]["ms"])
    peak, peak_kind = measured_peak_hbm()
    achieved = pd[dom]["bytes"] / (pd[dom]["ms"] / 1e3) / 1e9 if pd[dom]["ms"] > 0 else 0.0
    tpb = ncu_traffic_per_byte(dom, args.lgn, args.dtype, args.pivot)
    per_launch_alg = pd[dom]["bytes"] / max(1, pd[dom]["launches"])
    # the profiled pass ran K sorts: per-sort bytes over the timed pass's time per sort
    per_sort = {k: {"bytes": v["bytes"] / args.steps} for k, v in pd.items()}
    whole = whole_roofline(per_sort, el_ms / args.steps, peak, peak_kind)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                "timing": "CUDA events around every launch, in a profiled pass of the same K "
                          "sorts run right after the timed region (the timed pass launches the "
                          "same kernels from the host loop without events, each with a "
                          "programmatic dependency on the one before it)",
                "traffic": (tpb * per_launch_alg) if tpb is not None else None,
                "alg_bytes_per_launch": per_launch_alg,
                "kernels": {k: {"ms": round(v["ms"] / args.steps, 4),
                                "share": round(v["ms"] / max(1e-9, sum(x["ms"] for x in pd.values())), 4),
                                "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None,
                                "launches": v["launches"] // args.steps}
                            for k, v in pd.items() if v["launches"]}}

    e2e = None
    if not args.no_e2e:
        # Each step: the array crosses host -> device, is sorted through the
        # C ABI and crosses back.  Double-buffered over three streams, as an
        # application would run it: the next array's upload and the previous
        # result's download overlap the current sort.
        hbuf = torch.empty(n, dtype=tdt, pin_memory=True)
        hbuf.copy_(torch.from_numpy(host.view(np.int32 if esz == 4 else np.int64)))
        hout = torch.empty(n, dtype=tdt, pin_memory=True)
        dbuf = [torch.empty(n, dtype=tdt, device="cuda") for _ in range(2)]
        s_up, s_sort, s_down = (torch.cuda.Stream() for _ in range(3))
        # the link alone: uploads and downloads of a whole array (the best of
        # three; the first copy on a fresh buffer can be several times slower)
        link = {}
        for name, dst, src, stream in (("h2d_GBps", dbuf[0], hbuf, s_up),
                                       ("d2h_GBps", hout, dbuf[0], s_down)):
            best = 0.0
            for _ in range(3):
                torch.cuda.synchronize()
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    c0.record(stream)
                    dst.copy_(src, non_blocking=True)
                    c1.record(stream)
                torch.cuda.synchronize()
                best = max(best, n * esz / (c0.elapsed_time(c1) / 1e3) / 1e9)
            link[name] = best
        ksteps = max(8, min(args.steps, 16))

        def pipeline(steps):
            up = [torch.cuda.Event() for _ in range(steps)]
            srt = [torch.cuda.Event() for _ in range(steps)]
            down = [torch.cuda.Event() for _ in range(steps)]

            def upload(i):
                with torch.cuda.stream(s_up):
                    if i >= 2:
                        s_up.wait_event(down[i - 2])  # this buffer's previous result is out
                    dbuf[i % 2].copy_(hbuf, non_blocking=True)
                    up[i].record(s_up)

            upload(0)
            for i in range(steps):
                d = dbuf[i % 2]
                if i + 1 < steps:
                    upload(i + 1)  # enqueued before the sort, so it overlaps it
                s_sort.wait_event(up[i])
                # the plain API; it returns once the sort has finished
                q.qms_sort(d, pivot=args.pivot, dtype=args.dtype, stream=s_sort)
                srt[i].record(s_sort)
                with torch.cuda.stream(s_down):
                    s_down.wait_event(srt[i])
                    hout.copy_(d, non_blocking=True)
                    down[i].record(s_down)

        # Untimed warm-up steps of the same pipeline: the first steps of a
        # fresh pipeline stalled on the host link (a 1 GiB upload once took
        # 59 ms and a download 93 ms, against 5-6 ms in steady state).
        pipeline(2)
        barrier()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(s_up)
        pipeline(ksteps)
        a1.record(s_down)
        torch.cuda.synchronize()
        e_ms = a0.elapsed_time(a1)
        tt = torch.tensor([e_ms], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e_ms = float(tt.item())
        out_e2e = hout[: min(n, 1 << 20)].numpy()
        if args.dtype in ("u32", "u64"):
            out_e2e = out_e2e.view(np.uint32 if esz == 4 else np.uint64)
        if args.dtype != "f32":
            assert np.all(out_e2e[1:] >= out_e2e[:-1]), "e2e result not sorted"
        e2e = {"value": ws * ksteps * n / (e_ms / 1e3) / 1e9, "unit": "GKeys/s",
               "h2d_bytes_per_step": n * esz, "d2h_bytes_per_step": n * esz,
               "steps": ksteps, "warmup_steps": 2, **link,
               "api": "qms_sort via the C ABI; host pinned buffers; double-buffered, uploads "
                      "and downloads on their own streams overlapping the sorts"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, host=host)

    configs = None
    if rank == 0 and not args.no_configs:
        del bufs, work
        torch.cuda.empty_cache()
        bufs, work = [], None
        configs = config_records(args, q, torch, np)

    forms = None
    if not args.no_forms:
        bufs, work = [], None
        torch.cuda.empty_cache()
        ranks = Ranks(ws, rank, dist)
        which = [f.strip() for f in args.forms.split(",") if f.strip()]
        forms = {}
        if "batched" in which:
            forms["batched"] = bench_batched(args, q, torch, np, ranks)
        if "served" in which:
            forms["served"] = bench_served(args, q, torch, np, ranks)

    if rank == 0:
        line = {"metric": METRIC,
                "value": value, "unit": "GKeys/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": el_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": workload_name(args), "n": n, "pivot": args.pivot,
                           "arrays_per_gpu_step": 1, "l2": "inputs larger than L2 (%d MiB per "
                           "array), no flush" % (n * esz >> 20),
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "roofline": roofline, "roofline_whole_sort": whole, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": ck, "configs": configs,
                "forms": forms}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_qms(args)


if __name__ == "__main__":
    sys.exit(main())
