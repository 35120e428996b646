"""Pins for the oracle's four-way swap-merge Mergesort (the multi-way merging
that Sec. 6 of arXiv 1804.10062 leaves as future work) and for
QuickMergesort with it as the Mergesort step.

What fixes the oracle here, besides the plain definition of sorted output:
- every permutation (and every word over a small alphabet) up to seven keys;
- the buffer's contents survive as a multiset and the slots between the two
  regions are untouched;
- comparisons: a tournament over the pairs (0, 1) and (2, 3) compares
  exactly as often as merging those pairs and then the two results with a
  plain two-way merge, so an independent two-level merge sort written here
  must count the same on every input;
- moves: two per output of a four-way merge plus one for the saved hole, a
  recurrence that the oracle must meet exactly on any input;
- the information-theoretic bound: on average over all n! inputs a
  comparison sort makes at least lg(n!) comparisons;
- moves: the four-way levels halve the number of merge passes, so the
  whole QuickMergesort moves clearly fewer elements than with Fig. 3's
  two-way Mergesort (about 0.55-0.6 of them at 2^14 to 2^17 keys).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import qms_inputs as gen


def _quarters(n):
    off = [0]
    for i in range(4):
        off.append(off[-1] + n // 4 + (1 if i < n % 4 else 0))
    return off


def _merge2(a, b):
    out, i, j, c = [], 0, 0, 0
    while i < len(a) and j < len(b):
        c += 1
        if b[j] < a[i]:
            out.append(b[j])
            j += 1
        else:
            out.append(a[i])
            i += 1
    return out + a[i:] + b[j:], c


def _two_level_mergesort(xs):
    """Sorted copy and comparison count of a merge sort that cuts a range
    into the same four parts, sorts them, merges parts 0 and 1, parts 2 and
    3, then the two results (two-way merges only)."""
    n = len(xs)
    if n < 2:
        return list(xs), 0
    off = _quarters(n)
    parts, c = [], 0
    for i in range(4):
        p, ci = _two_level_mergesort(xs[off[i]:off[i + 1]])
        parts.append(p)
        c += ci
    m01, c1 = _merge2(parts[0], parts[1])
    m23, c2 = _merge2(parts[2], parts[3])
    m, c3 = _merge2(m01, m23)
    return m, c + c1 + c2 + c3


def _moves(n, to_target):
    """Moves of the four-way Mergesort in analysis mode: a merge of n
    outputs moves 2n + 1 elements; a single key sorted into the other
    region is one such merge (3 moves), in place it needs none."""
    if n == 0:
        return 0
    if n == 1:
        return 3 if to_target else 0
    off = _quarters(n)
    return sum(_moves(off[i + 1] - off[i], not to_target) for i in range(4)) + 2 * n + 1


def _run(keys, to_target, mode="analysis", gap=5, seed=0):
    n = len(keys)
    rng = np.random.default_rng(seed)
    buf = rng.integers(0, 2 ** 32, size=n, dtype=np.uint32)
    fill = rng.integers(0, 2 ** 32, size=gap, dtype=np.uint32)
    a = np.concatenate([np.asarray(keys, dtype=np.uint32), fill, buf])
    c, m = oracle.msort4_u32(a, 0, n, n + gap, to_target=to_target, mode=mode)
    res = a[n + gap:] if to_target else a[:n]
    rest = a[:n] if to_target else a[n + gap:]
    assert a[n:n + gap].tobytes() == fill.tobytes()  # the gap is untouched
    assert np.array_equal(np.sort(rest), np.sort(buf))  # the buffer survives
    return res, c, m


@pytest.mark.parametrize("to_target", [False, True])
def test_every_small_permutation_and_word(to_target):
    for n in range(0, 8):
        for p in itertools.permutations(range(n)):
            res, _, _ = _run(p, to_target)
            assert list(res) == sorted(p)
    for n in range(1, 7):
        for w in itertools.product(range(3), repeat=n):
            res, _, _ = _run(w, to_target)
            assert list(res) == sorted(w)


@pytest.mark.parametrize("mode", ["analysis", "paper"])
def test_random_inputs_with_duplicates(mode):
    rng = np.random.default_rng(7)
    for n in list(range(0, 70)) + [255, 256, 257, 1000, 4096, 5003]:
        for hi in (4, 2 ** 32):
            keys = rng.integers(0, hi, size=n, dtype=np.uint32)
            for to_target in (False, True):
                res, _, _ = _run(keys, to_target, mode=mode, seed=n)
                assert res.tobytes() == np.sort(keys).tobytes()


def test_comparisons_equal_two_level_merging():
    rng = np.random.default_rng(11)
    for n in list(range(0, 80)) + [127, 300, 1024, 2049, 3001]:
        for hi in (3, 50, 2 ** 32):
            keys = rng.integers(0, hi, size=n, dtype=np.uint32)
            ref, cref = _two_level_mergesort([int(x) for x in keys])
            for to_target in (False, True):
                res, c, _ = _run(keys, to_target)
                assert list(res) == ref
                assert c == cref, (n, hi, to_target)


def test_moves_follow_the_recurrence():
    rng = np.random.default_rng(13)
    for n in range(0, 300):
        keys = rng.integers(0, 2 ** 32, size=n, dtype=np.uint32)
        for to_target in (False, True):
            _, _, m = _run(keys, to_target)
            assert m == _moves(n, to_target), (n, to_target)


def test_average_comparisons_meet_the_information_bound():
    for n in range(2, 8):
        tot = 0
        perms = list(itertools.permutations(range(n)))
        for p in perms:
            _, c, _ = _run(p, False)
            tot += c
        assert tot / len(perms) >= math.log2(math.factorial(n)) - 1e-9


@pytest.mark.parametrize("variant", ["m3", "sqrtn", "mom", "hybrid"])
@pytest.mark.parametrize("mode", ["analysis", "paper"])
def test_quickmergesort_with_four_way_mergesort_sorts(variant, mode):
    for dist, n in (("uniform", 20000), ("mod16", 7777), ("sorted", 5000), ("reverse", 5001),
                    ("organ", 4097)):
        k = gen.keys(dist, "u32", n, 5)
        kk = k.copy()
        c, r, m = oracle.sort4_u32(kk, variant=variant, mode=mode)
        assert kk.tobytes() == np.sort(k).tobytes(), (variant, mode, dist)
        assert r >= 1


def test_four_way_levels_move_fewer_elements():
    rng = np.random.default_rng(17)
    for n in (1 << 14, 1 << 17):
        k = rng.integers(0, 2 ** 32, size=n, dtype=np.uint32)
        c4, _, m4 = oracle.sort4_u32(k.copy())
        c2, m2 = oracle.sort_moves_u32(k.copy())
        assert m4 < 0.7 * m2, (n, m4, m2)
        # the comparisons stay those of a binary Mergesort (within 2% of n lg n)
        assert abs(c4 - c2) < 0.02 * n * math.log2(n)
