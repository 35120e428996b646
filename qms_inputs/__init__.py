"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the bench.

This module holds random-number generation and input shapes only: no part of
the sorting method.  Every stream is SplitMix64 (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), computed with numpy
uint64 arithmetic so that any caller can regenerate the same bytes from the
same seed.

The paper's own workload is random permutations of {1..n} of integers
(Sec. 5); the other shapes (uniform 32/64-bit keys, normal and uniform floats,
few-distinct, presorted, reverse, organ-pipe, uneven batches, Poisson request
streams) are the synthetic stand-ins for the workloads this library is
measured on.  NaN is never produced.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the SplitMix64 stream of ``seed``."""
    out = np.empty(n, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for c0 in range(0, n, _CHUNK):
            c1 = min(n, c0 + _CHUNK)
            z = np.arange(offset + c0 + 1, offset + c1 + 1, dtype=np.uint64)
            z *= _GOLDEN
            z += s
            z ^= z >> np.uint64(30)
            z *= _M1
            z ^= z >> np.uint64(27)
            z *= _M2
            z ^= z >> np.uint64(31)
            out[c0:c1] = z
    return out


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def permutation_u32(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of 0..n-1 (ranks of a SplitMix64 stream)."""
    r = splitmix64(seed, n)
    return np.argsort(r, kind="stable").astype(np.uint32)


def uniform_u32(n: int, seed: int) -> np.ndarray:
    return (splitmix64(seed, n) >> np.uint64(32)).astype(np.uint32)


def uniform_u64(n: int, seed: int) -> np.ndarray:
    return splitmix64(seed, n)


def uniform_i64(n: int, seed: int) -> np.ndarray:
    return splitmix64(seed, n).view(np.int64)


def normal_f32(n: int, seed: int) -> np.ndarray:
    """N(0, 1) floats by Box-Muller in double, rounded to float32."""
    out = np.empty(n, dtype=np.float32)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        x = splitmix64(seed, 2 * (c1 - c0), 2 * c0)
        u1 = ((x[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
        u2 = (x[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        out[c0:c1] = (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).astype(np.float32)
    return out


def uniform01_f32(n: int, seed: int) -> np.ndarray:
    """U(0, 1) floats with 24 random bits (exactly representable)."""
    return ((splitmix64(seed, n) >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)).astype(np.float32)


def few_distinct_u64(n: int, seed: int, k: int = 16) -> np.ndarray:
    return splitmix64(seed, n) % np.uint64(k)


def sorted_u64(n: int, seed: int) -> np.ndarray:
    return np.sort(splitmix64(seed, n))


def reverse_u64(n: int, seed: int) -> np.ndarray:
    return np.ascontiguousarray(np.sort(splitmix64(seed, n))[::-1])


def organ_pipe_u64(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.uint64)
    return np.where(i < n // 2, i, np.uint64(n - 1) - i).astype(np.uint64)


def keys(dist: str, dtype: str, n: int, seed: int) -> np.ndarray:
    """Named key distributions; ``dtype`` in {u32, u64, i64, f32}."""
    if dist == "perm":
        assert dtype == "u32"
        return permutation_u32(n, seed)
    if dist == "uniform":
        return {"u32": uniform_u32, "u64": uniform_u64, "i64": uniform_i64,
                "f32": uniform01_f32}[dtype](n, seed)
    if dist == "normal":
        assert dtype == "f32"
        return normal_f32(n, seed)
    base = {"mod16": lambda: few_distinct_u64(n, seed),
            "sorted": lambda: sorted_u64(n, seed),
            "reverse": lambda: reverse_u64(n, seed),
            "organ": lambda: organ_pipe_u64(n)}[dist]()
    if dtype == "u64":
        return base
    if dtype == "i64":
        return base.view(np.int64)
    if dtype == "u32":
        if dist in ("sorted", "reverse"):
            return (base >> np.uint64(32)).astype(np.uint32)
        return base.astype(np.uint32)
    raise ValueError((dist, dtype))


def payload_index(n: int) -> np.ndarray:
    """Payload = original index, so a key-value result identifies each pair."""
    return np.arange(n, dtype=np.uint32)


def batch_lengths(nseg: int, seed: int, lo: int = 16, hi: int = 65536) -> np.ndarray:
    """Segment lengths floor(exp(U(ln lo, ln hi))), clipped to [lo, hi]."""
    u = uniform01(seed, nseg)
    L = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(L, lo, hi)


def offsets_of(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    np.cumsum(lengths, out=off[1:])
    return off


def request_stream(nreq: int, seed: int, lg_lo: float = 10.0, lg_hi: float = 26.0,
                   mix=(("u32", 0.5), ("u64", 0.3), ("f32", 0.2)), rate_per_s: float = 1000.0):
    """Poisson request stream: (arrival_s, n, dtype) with sizes floor(2^U(lo, hi))."""
    u = uniform01(seed, 3 * nreq).reshape(nreq, 3)
    sizes = np.floor(np.exp2(lg_lo + u[:, 0] * (lg_hi - lg_lo))).astype(np.int64)
    gaps = -np.log1p(-u[:, 1]) / rate_per_s
    arrivals = np.cumsum(gaps)
    cum = np.cumsum([p for _, p in mix])
    names = [d for d, _ in mix]
    dts = [names[int(np.searchsorted(cum, x, side="right"))] if x < cum[-1] else names[-1]
           for x in u[:, 2]]
    return [(float(arrivals[i]), int(sizes[i]), dts[i]) for i in range(nreq)]
