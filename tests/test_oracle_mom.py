"""Pins for the oracle's worst-case machinery (Sec. 4): the median of five,
the groups-of-five selection (plain and adaptive), the median-of-medians
pivot of every MoM round, the partition of only the 2n/3 non-medians, the
hybrid's switching rule, and the element-move counter (Sec. 5).  CPU only.

Each check ties the oracle to something outside it: the definition of a
median and of an order statistic (brute force over all small inputs), the
counting argument of Sec. 4 (at least 2 floor(n/6) elements on each side of
a median-of-medians pivot), the BFPRT discard guarantee, and closed forms of
Fig. 3's moves derived by hand for reverse-sorted input."""
import itertools
import math

import numpy as np
import pytest

import oracle
import qms_inputs as gen


# --------------------------------------------------------------------------
# median of five


def test_median5_all_permutations_of_distinct_keys():
    for p in itertools.permutations(range(5)):
        pos, c = oracle.median5_u32(p)
        assert p[pos] == 2, p
        assert c <= 6, (p, c)


def test_median5_all_tied_words():
    for w in itertools.product(range(3), repeat=5):
        pos, c = oracle.median5_u32(w)
        assert w[pos] == sorted(w)[2], w
        assert c <= 6


# --------------------------------------------------------------------------
# groups-of-five selection


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    yield "random", rng.permutation(n).astype(np.uint32)
    yield "tied", (rng.integers(0, 7, n)).astype(np.uint32)
    yield "sorted", np.arange(n, dtype=np.uint32)
    yield "reverse", np.arange(n, dtype=np.uint32)[::-1].copy()
    yield "organ", np.concatenate([np.arange(n // 2), np.arange(n - n // 2)[::-1]]).astype(np.uint32)


@pytest.mark.parametrize("adaptive", [False, True])
def test_select_returns_the_order_statistic(adaptive):
    for n in (1, 2, 5, 6, 11, 26, 125, 1000, 4099):
        for name, a0 in _inputs(n, n):
            ref = np.sort(a0)
            ranks = sorted({0, n - 1, n // 2, n // 3, (7 * n) // 10, n // 20, n - 1 - n // 20})
            for i in ranks:
                a = a0.copy()
                pos, _, _ = oracle.select_u32(a, i, adaptive=adaptive)
                assert a[pos] == ref[i], (name, n, i)
                np.testing.assert_array_equal(np.sort(a), ref)
                assert np.all(a[:pos] <= a[pos]) and np.all(a[pos + 1:] >= a[pos]), (name, n, i)


@pytest.mark.parametrize("adaptive", [False, True])
def test_select_discards_three_tenths_per_iteration(adaptive):
    # Distinct keys: each iteration continues on at most about 0.7 of its
    # range (at least 3 ceil(g/2) elements of the g = floor(n/5) groups lie on
    # the discarded side of a median of medians; the adaptive pivot keeps
    # the same guarantee, Sec. 4).
    for seed in range(4):
        n = 20000
        a0 = np.random.default_rng(seed).permutation(n).astype(np.uint32)
        for i in (0, n // 50, n // 7, n // 2, n - 1 - n // 7, n - 1 - n // 50, n - 1):
            _, _, tr = oracle.select_u32(a0.copy(), i, adaptive=adaptive)
            for m, kept in tr.tolist():
                if m >= 25:
                    assert kept <= 0.7 * m + 4, (seed, i, m, kept)


def _bfprt_tight(g):
    """5g distinct keys in groups of five built so that the median of the
    group medians has the smallest rank the groups-of-five argument allows:
    every group whose median lies above it has its two smaller keys just
    above it, and every other group has its two larger keys above all
    medians.  Selecting the maximum must then continue on 5g - 3 floor(g/2)
    - 3 keys, about 0.7 of the range and no more."""
    j0 = g // 2
    base, step = 10 ** 6, 10 ** 4
    out = []
    for k in range(g):
        m = base + step * k
        if k <= j0:
            small = [m - 2, m - 1]
            big = [10 ** 9 + 2 * k, 10 ** 9 + 2 * k + 1]
        else:
            pv = base + step * j0
            small = [pv + 1 + 2 * (k - j0), pv + 2 + 2 * (k - j0)]
            big = [m + 1, m + 2]
        out += [big[0], small[0], m, big[1], small[1]]
    return np.array(out, dtype=np.uint32), j0


def test_select_discard_bound_is_tight_on_a_constructed_input():
    for g in (20, 101, 400, 1000):
        a0, j0 = _bfprt_tight(g)
        n = a0.size
        _, _, tr = oracle.select_u32(a0.copy(), n - 1, adaptive=False)
        top = [k for m, k in tr.tolist() if m == n]  # the outermost first iteration
        assert top[0] == n - 3 * j0 - 3, (g, top)
        for m, kept in tr.tolist():
            if m >= 25:
                assert kept <= 0.7 * m + 4, (g, m, kept)
        pos, _, tr = oracle.select_u32(a0.copy(), n - 1, adaptive=True)
        for m, kept in tr.tolist():
            if m >= 25:
                assert kept <= 0.7 * m + 4, (g, m, kept)


def test_adaptive_select_narrows_extreme_ranks():
    # For a rank far from the middle the adaptive pivot sits just above the
    # sought element: the first iteration keeps a small part, and the whole
    # selection compares less than with the median of the group medians.
    n = 20000
    less = 0
    for seed in range(6):
        a0 = np.random.default_rng(100 + seed).permutation(n).astype(np.uint32)
        for i in (n // 20, n - 1 - n // 20):
            _, c0, t0 = oracle.select_u32(a0.copy(), i, adaptive=False)
            _, c1, t1 = oracle.select_u32(a0.copy(), i, adaptive=True)
            top0 = [k for m, k in t0.tolist() if m == n][0]
            top1 = [k for m, k in t1.tolist() if m == n][0]
            assert top1 <= 0.25 * n, (seed, i, top1)
            assert top0 >= 0.4 * n, (seed, i, top0)
            less += c1 < c0
    assert less >= 10


# --------------------------------------------------------------------------
# median-of-medians rounds


def _dists(n, seed):
    yield "uniform", np.random.default_rng(seed).integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    yield "perm", gen.permutation_u32(n, seed)
    yield "mod16", (np.random.default_rng(seed).integers(0, 16, n)).astype(np.uint32)
    yield "sorted", np.arange(n, dtype=np.uint32)
    yield "reverse", np.arange(n, dtype=np.uint32)[::-1].copy()
    yield "organ", np.concatenate([np.arange(n // 2), np.arange(n - n // 2)[::-1]]).astype(np.uint32)
    yield "adversary", oracle.adversary_u32(n, "m3", "analysis")[0]


@pytest.mark.parametrize("variant", ["mom", "hybrid"])
@pytest.mark.parametrize("mode", ["analysis", "paper"])
@pytest.mark.parametrize("mom", ["basic", "faithful"])
def test_mom_pivot_leaves_two_sixths_on_each_side(variant, mode, mom):
    # Sec. 4: the median of the floor(n/3) medians of three has at least
    # 2 floor(n/6) elements <= it and as many >= it (pivot included), so the
    # larger side can be Mergesorted with the smaller side as buffer.
    # With duplicate keys the bound holds for the pivot block of a three-way
    # split over all elements (paper mode, basic); a two-way split sends the
    # keys equal to the pivot right, and the faithful split leaves medians
    # equal to it on both sides, so those runs are checked on distinct keys.
    n = 3001 if variant == "mom" else 4096
    seen = 0
    for name, k0 in _dists(n, 9):
        if name == "mod16" and not (mode == "paper" and mom == "basic"):
            continue
        k = k0.copy()
        rec, _ = oracle.rounds_u32(k, variant=variant, mode=mode, mom=mom)
        np.testing.assert_array_equal(k, np.sort(k0))
        for b, e, lt, gt, ism, _, _, left in rec.tolist():
            if not ism:
                continue
            seen += 1
            m = e - b
            need = 2 * (m // 6)
            assert gt - b >= need and e - lt >= need, (name, b, e, lt, gt)
            nl, nr = lt - b, e - gt
            big, small = max(nl, nr), min(nl, nr)
            if (big + 1) // 2 <= small:  # the larger side is Mergesorted
                assert bool(left) == (nl >= nr), (name, b, e, lt, gt, left)
    assert seen > 0


def test_faithful_mom_partitions_only_the_non_medians():
    # Sec. 4: after the selection, the side of each of the n/3 medians is
    # known, so partitioning compares only the remaining n - floor(n/3)
    # elements (once each with a two-way partition).
    for seed in range(3):
        k = gen.permutation_u32(30001, seed)
        rec, _ = oracle.rounds_u32(k.copy(), variant="mom", mode="analysis", mom="faithful")
        for b, e, lt, gt, ism, _, part, _ in rec.tolist():
            assert ism
            assert part == (e - b) - (e - b) // 3, (b, e, part)
        rec, _ = oracle.rounds_u32(k.copy(), variant="mom", mode="analysis", mom="basic")
        for b, e, lt, gt, ism, _, part, _ in rec.tolist():
            assert part == (e - b) - 1
        rec, _ = oracle.rounds_u32(k.copy(), variant="mom", mode="paper", mom="faithful")
        for b, e, lt, gt, ism, _, part, _ in rec.tolist():
            r = (e - b) - (e - b) // 3
            assert r <= part <= 2 * r


@pytest.mark.parametrize("dist", ["uniform", "mod16", "sorted", "reverse", "organ"])
def test_faithful_mom_worst_case_bound_and_gain(dist):
    n = 1 << 14
    k = gen.keys(dist, "u64", n, 3)
    v = gen.payload_index(n)
    k0 = k.copy()
    c1, _ = oracle.sort(k, v, variant="mom", mode="paper", mom="faithful")
    np.testing.assert_array_equal(k, np.sort(k0))
    np.testing.assert_array_equal(k0[v], k)
    assert c1 <= n * math.log2(n) + 16.1 * n
    c0, _ = oracle.sort(k0.copy(), variant="mom", mode="paper", mom="basic")
    if dist in ("uniform", "sorted", "reverse"):  # distinct keys
        assert c1 < c0  # the n/3 medians are not compared with the pivot again


def test_hybrid_switches_after_an_unbalanced_pivot():
    # HQMS (Sec. 4, delta = 1/16): a median-of-3 pivot whose rank in its range
    # lies outside [floor(n/16), n - 1 - floor(n/16)] makes the next round a
    # median-of-medians round; every other round uses median-of-3.
    for name, k0 in _dists(4096, 5):
        rec, _ = oracle.rounds_u32(k0.copy(), variant="hybrid", mode="paper")
        for r0, r1 in zip(rec.tolist(), rec.tolist()[1:]):
            b, e, lt, gt, ism = r0[:5]
            m = e - b
            d = m // 16
            bad = (not ism) and ((gt - 1 - b) < d or (lt - b) > m - 1 - d)
            assert bool(r1[4]) == bad, (name, r0, r1)


# --------------------------------------------------------------------------
# element moves (Sec. 5)


def _msort_reverse(m):
    """Moves and comparisons of Fig. 3 msort on m reverse-sorted keys
    (analysis mode, leaves of one element swapped into place): at every
    level the target-side run holds the smaller keys, is taken first and
    runs out first, so a merge of s elements costs s - q comparisons (q the
    first half) and 2 s + 1 moves; a leaf swap costs 3 moves."""
    if m == 0:
        return 0, 0
    if m == 1:
        return 3, 0
    q = m // 2
    r = m - q
    mq, cq = _msort_reverse(q)
    mr, cr = _msort_reverse(r)
    return mq + mr + 2 * m + 1, cq + cr + r


def _out_reverse(n):
    """Fig. 3 out on n reverse-sorted keys: the second half (the smaller
    keys) is sorted into the buffer and is taken first by the final merge,
    which stops as soon as it runs out: r comparisons, 2 r + 2 moves."""
    if n <= 1:
        return 0, 0
    q = n // 2
    r = n - q
    m1, c1 = _msort_reverse(r)
    m2, c2 = _msort_reverse(q)
    return m1 + m2 + 2 * r + 2, c1 + c2 + r


def test_out_moves_on_reverse_input_match_closed_form():
    for n in range(1, 300):
        r = n - n // 2
        a = np.concatenate([np.arange(n, dtype=np.uint32)[::-1] + 1000,
                            np.zeros(r, dtype=np.uint32)])
        c, mv = oracle.out_moves_u32(a, 0, n, n)
        np.testing.assert_array_equal(a[:n], np.arange(n, dtype=np.uint32) + 1000)
        want_m, want_c = _out_reverse(n)
        assert (mv, c) == (want_m, want_c), n


def test_moves_small_cases_by_hand():
    # n = 2: one compare-and-swap (3 moves when it swaps, none otherwise).
    a = np.array([1, 0], dtype=np.uint32)
    assert oracle.sort_moves_u32(a) == (1, 3)
    a = np.array([0, 1], dtype=np.uint32)
    assert oracle.sort_moves_u32(a) == (1, 0)
    # Every permutation: at least one move per misplaced key, and the sort's
    # comparisons agree with the uncounted oracle.
    for n in range(3, 7):
        for p in itertools.permutations(range(n)):
            a = np.array(p, dtype=np.uint32)
            c, mv = oracle.sort_moves_u32(a)
            assert a.tolist() == list(range(n))
            assert mv >= sum(1 for i, x in enumerate(p) if x != i)
            b = np.array(p, dtype=np.uint32)
            assert oracle.sort(b)[0] == c


def test_moves_counter_agrees_with_uncounted_sort():
    for variant in ("m3", "sqrtn", "mom", "hybrid"):
        for mom in ("basic", "faithful"):
            k = gen.permutation_u32(5000, 3)
            a = k.copy()
            c, mv = oracle.sort_moves_u32(a, variant=variant, mode="paper", mom=mom)
            b = k.copy()
            c2, _ = oracle.sort(b, variant=variant, mode="paper", mom=mom)
            assert c == c2 and a.tobytes() == b.tobytes()
            assert 5000 <= mv < 60 * 5000
