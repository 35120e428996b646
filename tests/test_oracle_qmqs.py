"""Pins for QuickMergeXsort (Sec. 3, Thm. 3) in the oracle (no GPU): Mergesort
stops below a threshold and X = CleverQuicksort (median-of-3 quicksort) sorts
the block.  The exact average over all permutations equals a recurrence
derived the way the proof of Thm. 1 does (partitioning keeps both sides
random; a merge of random runs a, b costs a + b - a/(b+1) - b/(a+1)); Monte
Carlo means agree with it at larger n; and its leading term lies between
Mergesort's (1) and CleverQuicksort's (12/7 ln 2 = 1.188), approaching Thm.
3's (alpha + 1)/2 = 1.094 with the threshold at sqrt(n)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import qms_inputs as gen


def _frac_dp(nmax, thresh):
    """The recurrence in exact arithmetic (independent of the oracle's C++)."""
    def P(n, k):
        return Fraction((k - 1) * (n - k) * 6, n * (n - 1) * (n - 2))
    Q = [Fraction(0)] * (nmax + 1)
    for n in range(2, nmax + 1):
        if n == 2:
            Q[n] = Fraction(1)
            continue
        Q[n] = Fraction(8, 3) + (n - 3) + sum(P(n, k) * (Q[k - 1] + Q[n - k]) for k in range(1, n + 1))
    E = lambda a, b: a + b - Fraction(a, b + 1) - Fraction(b, a + 1)
    MX = [Fraction(0)] * (nmax + 1)
    MO = [Fraction(0)] * (nmax + 1)
    for n in range(2, nmax + 1):
        q, r = n // 2, n - n // 2
        MX[n] = Q[n] if n < thresh else MX[q] + MX[r] + E(q, r)
        MO[n] = MX[q] + MX[r] + E(q, r)
    T = [Fraction(0)] * (nmax + 1)
    for n in range(2, nmax + 1):
        if n == 2:
            T[n] = Fraction(1)
            continue
        s = Fraction(0)
        for k in range(1, n + 1):
            rest = (MO[k - 1] + T[n - k]) if (k - 1 < n // 2) else (MO[n - k] + T[k - 1])
            s += P(n, k) * rest
        T[n] = Fraction(8, 3) + (n - 3) + s
    return T, Q


@pytest.mark.parametrize("thresh", [2, 3, 4, 5])
def test_exhaustive_average_equals_recurrence(thresh):
    T, _ = _frac_dp(8, thresh)
    Td, _ = oracle.dp_qmqs(8, thresh)
    for n in range(1, 9):
        tot = 0
        for p in itertools.permutations(range(n)):
            a = np.array(p, dtype=np.uint32)
            tot += oracle.qmqs_u32(a, thresh)
            assert a.tolist() == list(range(n))
        assert Fraction(tot, math.factorial(n)) == T[n], (thresh, n)
        assert abs(Td[n] - float(T[n])) < 1e-9


def _frac_msort(nmax, thresh):
    """Exact averages of Fig. 3's out with the stopper: X-msort(n) is
    CleverQuicksort's Q(n) below thresh, else the halves plus the merge."""
    _, Q = _frac_dp(nmax, thresh)
    E = lambda a, b: a + b - Fraction(a, b + 1) - Fraction(b, a + 1)
    MX = [Fraction(0)] * (nmax + 1)
    MO = [Fraction(0)] * (nmax + 1)
    for n in range(2, nmax + 1):
        q, r = n // 2, n - n // 2
        MX[n] = Q[n] if n < thresh else MX[q] + MX[r] + E(q, r)
        MO[n] = MX[q] + MX[r] + E(q, r)
    return MO, Q


@pytest.mark.parametrize("thresh", [2, 4, 5, 6, 11])
def test_mergesort_with_stopper_exhaustive(thresh):
    # out(m) over all m! permutations: its two msort halves use X exactly
    # when they are shorter than thresh.  CleverQuicksort and Mergesort cost
    # differently from 5 keys on (Q(5) = 106/15, M(5) = 43/6), so thresholds
    # 5, 6 and 11 separate X from Mergesort and pin the boundary.
    MO, Q = _frac_msort(10, thresh)
    assert Q[5] == Fraction(106, 15)
    for m in range(2, 11):
        if m > 8 and thresh not in (5, 6, 11):
            continue
        r = m - m // 2
        tot = 0
        vals = []
        rng = np.random.default_rng(m)
        perms = itertools.permutations(range(m)) if m <= 8 else \
            (rng.permutation(m) for _ in range(20000))
        cnt = 0
        for p in perms:
            a = np.concatenate([np.array(p, dtype=np.uint32), np.full(r, 99, dtype=np.uint32)])
            c = oracle.out_x_u32(a, 0, m, m, thresh)
            tot += c
            vals.append(c)
            assert a[:m].tolist() == list(range(m))
            cnt += 1
        if m <= 8:
            assert Fraction(tot, cnt) == MO[m], (thresh, m)
        else:  # sampled: within 4 standard errors of the exact average
            se = float(np.std(vals, ddof=1)) / math.sqrt(cnt)
            assert abs(tot / cnt - float(MO[m])) < 4 * se, (thresh, m, tot / cnt, float(MO[m]), se)


def test_double_precision_table_equals_exact_recurrence():
    for thresh in range(2, 13):
        T, Q = _frac_dp(40, thresh)
        Td, Qd = oracle.dp_qmqs(40, thresh)
        for n in range(41):
            assert abs(Td[n] - float(T[n])) < 1e-9 * max(1.0, float(T[n])), (thresh, n)
            assert abs(Qd[n] - float(Q[n])) < 1e-9 * max(1.0, float(Q[n])), (thresh, n)


@pytest.mark.parametrize("n,seeds", [(1000, 200), (4096, 80)])
def test_mc_mean_matches_recurrence(n, seeds):
    th = int(math.ceil(math.sqrt(n)))
    T, _ = oracle.dp_qmqs(n, th)
    cs = []
    for s in range(seeds):
        a = gen.permutation_u32(n, 131 * s + n)
        cs.append(oracle.qmqs_u32(a, th))
        assert np.all(a[1:] > a[:-1])
    cs = np.array(cs, dtype=np.float64)
    se = cs.std(ddof=1) / math.sqrt(seeds)
    assert abs(cs.mean() - T[n]) <= 4 * se + 1e-9, (cs.mean(), T[n], se)


def test_leading_term_between_mergesort_and_quicksort():
    res = {}
    for k in (10, 12, 14):
        n = 1 << k
        T, Q = oracle.dp_qmqs(n, 1 << (k // 2))
        res[k] = (T[n] / n, Q[n] / n)
    qmqs_slope = (res[14][0] - res[12][0]) / 2
    quick_slope = (res[14][1] - res[12][1]) / 2
    assert abs(quick_slope - 12 / 7 * math.log(2)) < 0.01       # CleverQuicksort
    assert 1.04 < qmqs_slope < 1.10                             # Thm. 3: 1.094 in the limit
    T0, _ = oracle.dp(1 << 14)
    assert T0[1 << 14] < res[14][0] * (1 << 14) < res[14][1] * (1 << 14)


@pytest.mark.parametrize("dtype_dist", [("uniform", 5), ("mod16", 6), ("sorted", 7)])
def test_sorts_like_a_library_sort(dtype_dist):
    dist, seed = dtype_dist
    for n in (2, 3, 17, 1000, 5000):
        k = gen.keys(dist, "u32", n, seed)
        a = k.copy()
        oracle.qmqs_u32(a, 64, mode="paper")
        assert a.tobytes() == np.sort(k).tobytes()
