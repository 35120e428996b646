// QuickMergesort oracle (Edelkamp & Weiss, "QuickMergesort: Practically
// Efficient Constant-Factor Optimal Sorting", arXiv 1804.10062).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
// reference that the CUDA path is checked against.  Only the tests, the
// smoke check and the CPU-baseline leg of the benchmark may load it.  It
// shares no code, header, table or helper with the CUDA library.
//
// What it computes (paper sections in brackets):
//   * QuickXsort skeleton with X = Mergesort [Sec. 2]: choose a pivot,
//     partition, sort one side with Mergesort using the other side as the
//     swap buffer, continue on the remaining side.
//   * merge / msort / out / sort as in the C++ implementation figure of
//     Sec. 3 (Fig. 3), with two corrections:
//       - msort for odd n uses r = n - floor(n/2) slots for the first half
//         target (the printed version reads a buffer element as data);
//       - merge does not read one slot past its target range on its last
//         step (the printed version reads, then overwrites, that slot).
//   * Pivot rules: median-of-3 [Sec. 2, proof of Thm. 1], median-of-sqrt(n)
//     [Sec. 2, Thm. 2], MoMQuickMergesort (median of the n/3 medians of
//     three, found with the groups-of-five median-of-medians selection)
//     [Sec. 4], HybridQuickMergesort with delta = 1/16 [Sec. 4].
//   * An element-comparison counter [Sec. 5]: every call of the order
//     predicate adds one.
//   * An element-move counter [Sec. 5, the moves experiment]: the sort run on
//     a key type whose construction and assignment from another element
//     count one move each, so a swap counts three.
//   * QuickMergeXsort [Sec. 3, Thm. 3]: an option x_thresh > 0 stops the
//     Mergesort recursion (msort) below x_thresh elements and sorts such a
//     block with X = CleverQuicksort (median-of-3 quicksort: the same sort3,
//     Lomuto partition and recursion on both sides), then moves it into its
//     target; the paper's QMQS takes x_thresh near sqrt(n).
//   * The multi-way merging that Sec. 6 names as future work, as an option:
//     a four-way swap-merge Mergesort in the full-buffer form (four parts
//     sorted into the other region, merged back by a tournament over the
//     pairs (0, 1) and (2, 3), each output swapped with a buffer element
//     through one hole), and QuickMergesort with it as the Mergesort step
//     (the side with a buffer at least as large as itself is sorted).
//   * The MoM details of Sec. 4 as an option ("faithful" MoM): adaptive
//     selection inside the median-of-medians routine, and a partition of
//     only the 2n/3 elements that are not medians of triples (the medians
//     are already on the correct side once the selection has run).
//
// Readings of points the paper leaves open (each also listed in the design
// notes of the repository):
//   * Median-of-3 samples positions b, b + floor(n/2), e - 1.  sort3 compares
//     (mid, lo), then (hi, mid) and, only if that swapped, (mid, lo) again.
//     The pivot is parked at b + 1 and the n - 3 non-sample elements are
//     partitioned with one comparison each (Lomuto movement), so one round
//     costs sort3 + (n - 3) comparisons as in the proof of Thm. 1.
//   * The driver partitions only ranges of >= 3 elements; a range of 2 gets
//     one compare-and-swap.  Side choice follows Fig. 3: Mergesort the left
//     side iff the pivot index is below the integer midpoint.
//   * "paper" mode adds what the experiments describe but the listing omits:
//     insertion sort below 10 elements (driver and msort leaves) and a
//     duplicate guard (a tie between the pivot and a neighbouring sample
//     switches the round to a three-way partition whose equal block is
//     final).  "analysis" mode is the listing alone (leaf n <= 1).
//   * Median-of-sqrt(n): k = largest odd number <= ceil(sqrt n), samples at
//     b + i * floor(n/k), moved to the front and sorted by this same sort.
//   * MoM: triples (3i, 3i+1, 3i+2), i < floor(n/3), medians moved to slot
//     b + i; median of medians by groups-of-five selection (6-comparison
//     median of five); all n - 1 other elements are compared with the pivot.
//     MoM rounds Mergesort the larger side when its ceil(m/2) buffer fits
//     in the smaller side, else the smaller side.
//   * Faithful MoM (Sec. 4, last paragraphs): the selection looks for rank k
//     among n elements; for k <= 0.3n it takes as pivot the group median of
//     rank ceil((k+1)/3) - 1 (the smallest rank that still places at least
//     k + 1 elements at or below the pivot, so the sought element stays on
//     the kept side while about 0.3n elements or more are discarded), and
//     mirrored for k >= 0.7n; otherwise the median of the group medians.
//     After the selection the n/3 medians are split around the pivot, so
//     only the other elements are compared with it; blocks are then put in
//     place by rotations (moves, no comparisons).
//   * HQMS: a median-of-3 pivot whose rank inside the current range lies
//     outside [floor(n/16), n - 1 - floor(n/16)] makes the next round MoM;
//     the round after that is median-of-3 again.
//   * Key order: ascending; float keys use IEEE order with -0 < +0 (NaN is
//     never generated); int64 is signed.

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

namespace {

enum Variant { M3 = 0, SQRTN = 1, MOM = 2, HYBRID = 3 };
enum Mode { ANALYSIS = 0, PAPER = 1 };

// ---- plain order predicates on the raw key types -------------------------

struct LessU32 {
  bool operator()(uint32_t x, uint32_t y) const { return x < y; }
};
struct LessU64 {
  bool operator()(uint64_t x, uint64_t y) const { return x < y; }
};
struct LessI64 {
  bool operator()(int64_t x, int64_t y) const { return x < y; }
};
struct LessF32 {
  // IEEE "<" for non-NaN values, with -0 ordered before +0.
  bool operator()(float x, float y) const {
    if (x < y) return true;
    if (y < x) return false;
    return std::signbit(x) && !std::signbit(y);
  }
};

// An element is a key, or a (key, payload) pair moved as one unit.
template <class K>
struct Pair {
  K key;
  uint32_t val;
};

template <class K, class KLess>
struct ByKey {
  KLess kl;
  bool operator()(const K& x, const K& y) const { return kl(x, y); }
  bool operator()(const Pair<K>& x, const Pair<K>& y) const {
    return kl(x.key, y.key);
  }
};

struct Split {
  size_t lt, gt;  // [b,lt) left side, [lt,gt) pivot block, [gt,e) right side
  bool mom;       // the round used a MoM pivot
};

// One partition round as seen by the tests: the range, the pivot block, the
// rule, the comparisons spent choosing the pivot and partitioning, and the
// side that was Mergesorted.
struct RoundRec {
  uint64_t b, e, lt, gt, mom, cmp_pivot, cmp_part, left;
};

// One iteration of the groups-of-five selection: the range size and the size
// of the part it continues on (0 once the element is found).
struct SelRec {
  uint64_t n, kept;
};

// An element type whose moves are counted: every construction from, or
// assignment of, another element adds one (so std::swap adds three).
template <class K>
struct Counted {
  K v;
  static thread_local uint64_t moves;
  Counted() : v() {}
  Counted(const Counted& o) : v(o.v) { ++moves; }
  Counted& operator=(const Counted& o) {
    v = o.v;
    ++moves;
    return *this;
  }
};
template <class K>
thread_local uint64_t Counted<K>::moves = 0;

template <class E, class Less>
class QuickMergesort {
 public:
  QuickMergesort(E* a, Less less, int variant, int mode, int side, int mom = 0, size_t x_thresh = 0)
      : a_(a), less_(less), variant_(variant), mode_(mode), side_(side), mom_(mom),
        x_thresh_(x_thresh) {}

  uint64_t comparisons() const { return cmps_; }
  uint64_t rounds() const { return rounds_; }
  // 2: Fig. 3's two-way Mergesort; 4: the four-way swap-merge (Sec. 6).
  void set_kway(int k) { kway_ = k; }
  std::vector<RoundRec>* round_log = nullptr;  // filled when set
  std::vector<SelRec>* select_log = nullptr;   // filled when set

  // Sorts a[b, e) ascending.
  void sort(size_t b, size_t e) {
    bool mom_next = false;
    const size_t stop = (mode_ == PAPER) ? 10 : 3;
    while (e - b >= stop) {
      ++rounds_;
      const size_t n = e - b;
      const bool mom_round =
          variant_ == MOM || (variant_ == HYBRID && mom_next);
      const uint64_t c0 = cmps_;
      Split s;
      if (variant_ == SQRTN) {
        s = partition_sqrtn(b, e);
      } else if (mom_round) {
        s = partition_mom(b, e);
      } else {
        s = partition_m3(b, e);
      }
      if (variant_ == HYBRID) {
        // Rank of the pivot block inside [b, e), 0-based.
        const size_t d = n / 16;
        const size_t r_lo = s.lt - b, r_hi = s.gt - 1 - b;
        mom_next = !mom_round && (r_hi < d || r_lo > n - 1 - d);
      }
      const size_t nl = s.lt - b, nr = e - s.gt;
      bool left;
      if (kway_ == 4 && (s.mom || side_ == 1 || s.gt != s.lt + 1)) {
        // The four-way Mergesort takes a buffer as large as its input.
        left = nl <= nr;
      } else if (s.mom || side_ == 1) {
        // Larger side if its ceil(m/2) buffer fits in the other side.
        const size_t big = std::max(nl, nr), small = std::min(nl, nr);
        const bool big_fits = (big + 1) / 2 <= small;
        left = big_fits ? (nl >= nr) : (nl < nr);
      } else if (s.gt == s.lt + 1) {
        // Fig. 3: Mergesort the left side iff the pivot is left of the
        // integer midpoint.
        left = s.lt < (b + e) / 2;
      } else {
        left = nl <= nr;  // three-way split: the smaller side
      }
      if (round_log) {
        const uint64_t part = s.mom ? part_cmps_ : 0;
        round_log->push_back(RoundRec{b, e, s.lt, s.gt, s.mom ? 1u : 0u,
                                      cmps_ - c0 - part, part, left ? 1u : 0u});
      }
      if (left) {
        if (kway_ == 4) msort4_in(b, s.lt - b, s.gt); else out(b, s.lt, s.gt);
        b = s.gt;
      } else {
        if (kway_ == 4) msort4_in(s.gt, e - s.gt, b); else out(s.gt, e, b);
        e = s.lt;
      }
    }
    if (mode_ == PAPER) {
      insertion_sort(b, e);
    } else if (e - b == 2) {
      if (lt(a_[b + 1], a_[b])) std::swap(a_[b], a_[b + 1]);
    }
  }

  // Four-way swap-merge Mergesort (the multi-way merging that Sec. 6 names
  // as future work), in the full-buffer form: the buffer has as many slots
  // as the input.  A range is cut into four parts of n/4 elements (the first
  // n mod 4 parts one more); the parts are sorted into the other region and
  // merged back by a four-way merge whose every output takes the place of a
  // buffer element, which moves into the slot the output came from.
  //
  // msort4_in: sorts a[b, b + n) in place; a[t, t + n) is the buffer (its
  // contents are permuted).  msort4_to: sorts a[b, b + n) into a[t, t + n);
  // the old buffer contents end up in a[b, b + n).  Base: in "paper" mode
  // insertion sort below 10 elements, else single elements.
  void msort4_in(size_t b, size_t n, size_t t) {
    const size_t leaf = (mode_ == PAPER) ? 10 : 2;
    if (n < leaf) {
      if (mode_ == PAPER) insertion_sort(b, b + n);
      return;
    }
    size_t off[5];
    quarters(n, off);
    for (int i = 0; i < 4; ++i) msort4_to(b + off[i], off[i + 1] - off[i], t + off[i]);
    merge4(t, off, b);
  }
  void msort4_to(size_t b, size_t n, size_t t) {
    const size_t leaf = (mode_ == PAPER) ? 10 : 2;
    if (n < leaf) {
      if (mode_ == PAPER) insertion_sort(b, b + n);
      if (n > 0) {
        size_t off1[5] = {0, n, n, n, n};  // one run: a plain block move
        merge4(b, off1, t);
      }
      return;
    }
    size_t off[5];
    quarters(n, off);
    for (int i = 0; i < 4; ++i) msort4_in(b + off[i], off[i + 1] - off[i], t + off[i]);
    merge4(b, off, t);
  }

  // Internal Mergesort of a[b, e) using the ceil(n/2) slots at a[temp, ...)
  // as swap buffer (Fig. 3, "out").  Buffer contents are permuted.
  void out(size_t b, size_t e, size_t temp) {
    const size_t n = e - b;
    if (n > 1) {
      const size_t q = n / 2, r = n - q;
      msort(b + q, e, temp);
      msort(b, b + q, b + r);
      merge(temp, temp + r, b, e);
    }
  }

 private:
  bool lt(const E& x, const E& y) {
    ++cmps_;
    return less_(x, y);
  }

  // Fig. 3 "merge": run1 = a[b1, e1) (in the buffer), run2 sits at the tail
  // of the target range a[t, et); the first (e1 - b1) target slots hold
  // buffer elements.  One hole (temp) carries a buffer element; buffer
  // elements end in run1's slots.
  void merge(size_t b1, size_t e1, size_t t, size_t et) {
    size_t i1 = b1, i2 = t + (e1 - b1), r = t;
    E temp = a_[t];
    while (i1 != e1 && i2 != et) {
      size_t src = lt(a_[i1], a_[i2]) ? i1++ : i2++;
      a_[r++] = a_[src];
      a_[src] = a_[r];
    }
    while (i1 < e1) {
      a_[r++] = a_[i1];
      if (r != et) a_[i1] = a_[r];  // the printed loop reads a[et] here
      ++i1;
    }
    a_[i1 - 1] = temp;
  }

  // Part boundaries of a four-way split of n: off[0] = 0 <= ... <= off[4] = n.
  static void quarters(size_t n, size_t off[5]) {
    off[0] = 0;
    for (int i = 0; i < 4; ++i) off[i + 1] = off[i] + n / 4 + (static_cast<size_t>(i) < n % 4 ? 1 : 0);
  }

  // Four-way merge: run i is a[s + off[i], s + off[i+1]); the n = off[4]
  // outputs go to a[d, d + n), which holds buffer elements (disjoint from the
  // runs).  Each output moves into the hole left by the previous step and
  // the next buffer element moves into the consumed run slot (one hole, as
  // in Fig. 3's merge: two moves per output).  The smallest head is found by
  // a tournament over the pairs (0, 1) and (2, 3): after an output only the
  // consumed run's pair and the final match are replayed, one comparison
  // each while both sides have elements left; equal keys go to the lower
  // run.
  void merge4(size_t s, const size_t off[5], size_t d) {
    const size_t n = off[4];
    if (n == 0) return;
    size_t h[4], end[4];
    for (int i = 0; i < 4; ++i) {
      h[i] = s + off[i];
      end[i] = s + off[i + 1];
    }
    auto alive = [&](int i) { return i >= 0 && h[i] != end[i]; };
    auto match = [&](int x, int y) {  // winner of runs x < y (or -1)
      const bool ax = alive(x), ay = alive(y);
      if (ax && ay) return lt(a_[h[y]], a_[h[x]]) ? y : x;
      return ax ? x : (ay ? y : -1);
    };
    int w01 = match(0, 1), w23 = match(2, 3);
    int win = match_winners(w01, w23, h, end);
    E temp = a_[d];
    for (size_t p = 0; p < n; ++p) {
      const size_t src = h[win]++;
      a_[d + p] = a_[src];
      a_[src] = (p + 1 < n) ? a_[d + p + 1] : temp;
      if (p + 1 == n) break;
      if (win < 2) w01 = match(0, 1); else w23 = match(2, 3);
      win = match_winners(w01, w23, h, end);
    }
  }
  int match_winners(int x, int y, const size_t* h, const size_t* end) {
    const bool ax = x >= 0 && h[x] != end[x], ay = y >= 0 && h[y] != end[y];
    if (ax && ay) return lt(a_[h[y]], a_[h[x]]) ? y : x;
    return ax ? x : (ay ? y : -1);
  }

  // Fig. 3 "msort": sorts a[b, e) into a[t, t + n); the old target contents
  // end up in a[b, e).  r = n - floor(n/2) is used for the odd case.
  void msort(size_t b, size_t e, size_t t) {
    const size_t n = e - b;
    if (x_thresh_ > 0 && n < x_thresh_) {
      // QuickMergeXsort: X sorts the block, which then moves to its target.
      clever_quicksort(b, e);
      for (size_t i = 0; i < n; ++i) std::swap(a_[b + i], a_[t + i]);
      return;
    }
    const size_t leaf = (mode_ == PAPER) ? 10 : 2;
    if (n < leaf) {
      if (mode_ == PAPER) insertion_sort(b, e);
      for (size_t i = 0; i < n; ++i) std::swap(a_[b + i], a_[t + i]);
      return;
    }
    const size_t q = n / 2, r = n - q;
    msort(b + q, e, t + q);
    msort(b, b + q, b + r);
    merge(b + r, b + n, t, t + n);
  }

  // X = CleverQuicksort [Sec. 3]: median-of-3 quicksort.  A range of two
  // gets one compare-and-swap; from three on, sort3 on the first, middle and
  // last element, the median parked at b + 1, the other n - 3 elements
  // compared once each (Lomuto), and both sides sorted the same way.  The
  // smaller side recurses, the larger one loops (O(log n) stack).
  void clever_quicksort(size_t b, size_t e) {
    while (e - b >= 3) {
      const size_t n = e - b, m = b + n / 2;
      sort3(b, m, e - 1);
      std::swap(a_[m], a_[b + 1]);
      size_t i = lomuto(b + 1, b + 2, e - 1);
      std::swap(a_[b + 1], a_[i - 1]);
      const size_t k = i - 1;  // the pivot's final index
      if (k - b < e - (k + 1)) {
        clever_quicksort(b, k);
        b = k + 1;
      } else {
        clever_quicksort(k + 1, e);
        e = k;
      }
    }
    if (e - b == 2 && lt(a_[b + 1], a_[b])) std::swap(a_[b], a_[b + 1]);
  }

  void insertion_sort(size_t b, size_t e) {
    for (size_t i = b + 1; i < e; ++i) {
      E x = a_[i];
      size_t j = i;
      while (j > b && lt(x, a_[j - 1])) {
        a_[j] = a_[j - 1];
        --j;
      }
      a_[j] = x;
    }
  }

  // Lomuto partition of a[from, to) around the pivot parked at a[p]:
  // elements less than the pivot are moved to a[from, i).  Returns i.
  size_t lomuto(size_t p, size_t from, size_t to) {
    size_t i = from;
    for (size_t j = from; j < to; ++j) {
      if (lt(a_[j], a_[p])) {
        std::swap(a_[i], a_[j]);
        ++i;
      }
    }
    return i;
  }

  // Three-way partition of a[b, e) around the value v (Dijkstra): at most
  // two comparisons per element.
  Split three_way(size_t b, size_t e, E v) {
    size_t l = b, i = b, g = e;
    while (i < g) {
      if (lt(a_[i], v)) {
        std::swap(a_[l++], a_[i++]);
      } else if (lt(v, a_[i])) {
        std::swap(a_[i], a_[--g]);
      } else {
        ++i;
      }
    }
    return Split{l, g, false};
  }

  // Two-way partition with the pivot at a[b]: the other n - 1 elements are
  // compared once each; the pivot ends at its final index k.
  Split two_way_front(size_t b, size_t e) {
    size_t i = lomuto(b, b + 1, e);
    std::swap(a_[b], a_[i - 1]);
    return Split{i - 1, i, false};
  }

  // sort3 on positions lo, mid, hi; afterwards a[lo] <= a[mid] <= a[hi].
  void sort3(size_t lo, size_t mid, size_t hi) {
    if (lt(a_[mid], a_[lo])) std::swap(a_[mid], a_[lo]);
    if (lt(a_[hi], a_[mid])) {
      std::swap(a_[hi], a_[mid]);
      if (lt(a_[mid], a_[lo])) std::swap(a_[mid], a_[lo]);
    }
  }

  Split partition_m3(size_t b, size_t e) {
    const size_t n = e - b, m = b + n / 2;
    sort3(b, m, e - 1);
    if (mode_ == PAPER) {
      // Duplicate guard: a tie between the pivot and a neighbouring sample
      // selects a three-way partition.
      const bool strict = lt(a_[b], a_[m]) && lt(a_[m], a_[e - 1]);
      if (!strict) return three_way(b, e, a_[m]);
    }
    std::swap(a_[m], a_[b + 1]);
    size_t i = lomuto(b + 1, b + 2, e - 1);
    std::swap(a_[b + 1], a_[i - 1]);
    return Split{i - 1, i, false};
  }

  Split partition_sqrtn(size_t b, size_t e) {
    const size_t n = e - b;
    size_t c = static_cast<size_t>(std::sqrt(static_cast<double>(n)));
    while (c * c < n) ++c;
    while (c > 1 && (c - 1) * (c - 1) >= n) --c;  // c = ceil(sqrt(n))
    size_t k = (c % 2 == 1) ? c : c - 1;
    if (k == 0) k = 1;
    const size_t step = n / k;
    for (size_t i = 0; i < k; ++i) std::swap(a_[b + i], a_[b + i * step]);
    // Sort the sample with this same algorithm (counted).
    QuickMergesort inner(a_, less_, variant_, mode_, side_, mom_, x_thresh_);
    inner.sort(b, b + k);
    cmps_ += inner.comparisons();
    const size_t pm = b + k / 2;
    if (mode_ == PAPER && k >= 3) {
      const bool strict = lt(a_[pm - 1], a_[pm]) && lt(a_[pm], a_[pm + 1]);
      if (!strict) return three_way(b, e, a_[pm]);
    }
    std::swap(a_[b], a_[pm]);
    return two_way_front(b, e);
  }

  // (Test hooks: the selection routines below are public.)
 public:
  // Median of a[p0], a[p1], a[p2] with at most 3 comparisons; returns its
  // position.
  size_t median3_pos(size_t p0, size_t p1, size_t p2) {
    if (lt(a_[p1], a_[p0])) std::swap(p0, p1);  // now a[p0] <= a[p1]
    if (lt(a_[p2], a_[p1])) {
      return lt(a_[p2], a_[p0]) ? p0 : p2;
    }
    return p1;
  }

  // Median of the five elements at a[b, b+5) with 6 comparisons; returns
  // its position.
  size_t median5_pos(size_t b) {
    size_t p[5] = {b, b + 1, b + 2, b + 3, b + 4};
    auto L = [&](size_t i, size_t j) { return lt(a_[p[i]], a_[p[j]]); };
    if (L(1, 0)) std::swap(p[0], p[1]);  // p0 <= p1
    if (L(3, 2)) std::swap(p[2], p[3]);  // p2 <= p3
    if (L(2, 0)) {                       // make p0 the minimum of the four
      std::swap(p[0], p[2]);
      std::swap(p[1], p[3]);
    }
    // p0 is below p1, p2, p3 so it is not the median; the median is the
    // second smallest of {p1, p2, p3, p4}, where p2 <= p3.
    if (L(4, 1)) std::swap(p[1], p[4]);  // p1 <= p4
    if (L(2, 1)) {                       // p2 is the minimum of the four
      return L(3, 1) ? p[3] : p[1];
    }
    return L(4, 2) ? p[4] : p[2];  // p1 is the minimum of the four
  }

  // Groups-of-five selection (median of medians, [CLRS Sec. 9.3] as cited
  // in Sec. 4): rearranges a[b, e) and returns the position of an element of
  // rank i (0-based) in it.  Afterwards a[b, pos) <= a[pos] <= a[pos+1, e).
  // With mom_ = 1 the pivot of an iteration adapts to i (Sec. 4, last
  // paragraphs; the reading is in the header).
  size_t select(size_t b, size_t e, size_t i) {
    while (true) {
      const size_t n = e - b;
      if (n <= 5) {
        insertion_sort(b, e);
        if (select_log) select_log->push_back(SelRec{n, 0});
        return b + i;
      }
      const size_t g = n / 5;
      for (size_t j = 0; j < g; ++j) {
        std::swap(a_[b + j], a_[median5_pos(b + 5 * j)]);
      }
      size_t rank = g / 2;
      if (mom_ == 1) {
        if (10 * i <= 3 * n) {
          rank = (i + 1 + 2) / 3 - 1;  // ceil((i + 1) / 3) - 1
        } else if (10 * i >= 7 * n) {
          rank = g - 1 - ((n - i + 2) / 3 - 1);  // the mirror image
        }
        if (rank > g - 1) rank = g - 1;
      }
      const size_t mm = select(b, b + g, rank);
      std::swap(a_[b], a_[mm]);
      Split s = three_way(b, e, a_[b]);
      if (i < s.lt - b) {
        if (select_log) select_log->push_back(SelRec{n, s.lt - b});
        e = s.lt;
      } else if (i < s.gt - b) {
        if (select_log) select_log->push_back(SelRec{n, 0});
        return b + i;
      } else {
        if (select_log) select_log->push_back(SelRec{n, e - s.gt});
        i -= s.gt - b;
        b = s.gt;
      }
    }
  }

 private:
  Split partition_mom(size_t b, size_t e) {
    const size_t n = e - b, t = n / 3;
    for (size_t i = 0; i < t; ++i) {
      const size_t p = median3_pos(b + 3 * i, b + 3 * i + 1, b + 3 * i + 2);
      std::swap(a_[b + i], a_[p]);
    }
    const size_t mm = select(b, b + t, t / 2);
    const uint64_t c0 = cmps_;
    Split s;
    if (mom_ == 1 && t >= 1) {
      s = partition_rest(b, e, t, mm);
    } else {
      std::swap(a_[b], a_[mm]);
      s = (mode_ == PAPER) ? three_way(b, e, a_[b]) : two_way_front(b, e);
    }
    part_cmps_ = cmps_ - c0;
    s.mom = true;
    return s;
  }

  // Sec. 4: once the selection has run, the medians a[b, b + t) are split
  // around the pivot a[mm] (those before it are <= it, those after >= it),
  // so only the n - t other elements are compared with the pivot: once each
  // in analysis mode, three-way (at most twice) in paper mode.  Rotations
  // then bring the blocks into partition order.
  Split partition_rest(size_t b, size_t e, size_t t, size_t mm) {
    const size_t m0 = b + t;  // first non-median
    const E v = a_[mm];
    size_t nl = m0, ne = m0, hi = e;
    // a[m0, nl) < v, a[nl, ne) == v, a[ne, hi) unknown, a[hi, e) > v
    while (ne < hi) {
      if (lt(a_[ne], v)) {
        std::swap(a_[nl++], a_[ne++]);
      } else if (mode_ == PAPER && lt(v, a_[ne])) {
        std::swap(a_[ne], a_[--hi]);
      } else if (mode_ == PAPER) {
        ++ne;
      } else {
        // analysis mode: two-way, ">= v" stays right
        ++ne;
      }
    }
    if (mode_ != PAPER) {  // no equal block: a[nl, e) >= v
      hi = nl;
      ne = nl;
    }
    // [b, mm) medians <= v, mm pivot, (mm, m0) medians >= v,
    // [m0, nl) < v, [nl, ne) == v (paper mode), [ne, e) > v / >= v.
    // 1. Move the left non-medians before the pivot.
    std::rotate(a_ + mm, a_ + m0, a_ + nl);
    const size_t p = mm + (nl - m0);  // the pivot's new index
    // 2. Move the equal non-medians right after the pivot.
    const size_t rm = m0 - mm - 1;  // medians right of the pivot
    std::rotate(a_ + p + 1, a_ + p + 1 + rm, a_ + p + 1 + rm + (ne - nl));
    return Split{p, p + 1 + (ne - nl), true};
  }

  E* a_;
  Less less_;
  int variant_, mode_, side_, mom_;
  size_t x_thresh_;
  int kway_ = 2;
  uint64_t cmps_ = 0;
  uint64_t rounds_ = 0;
  uint64_t part_cmps_ = 0;  // comparisons of the last MoM round's partition
};

template <class K, class KLess>
int sort_typed(void* keys, uint32_t* vals, size_t n, int variant, int mode,
               int side, int mom, uint64_t* cmps, uint64_t* rounds) {
  using Less = ByKey<K, KLess>;
  K* k = static_cast<K*>(keys);
  uint64_t c = 0, r = 0;
  if (vals == nullptr) {
    QuickMergesort<K, Less> s(k, Less{}, variant, mode, side, mom);
    if (n > 1) s.sort(0, n);
    c = s.comparisons();
    r = s.rounds();
  } else {
    std::vector<Pair<K>> e(n);
    for (size_t i = 0; i < n; ++i) e[i] = Pair<K>{k[i], vals[i]};
    QuickMergesort<Pair<K>, Less> s(e.data(), Less{}, variant, mode, side, mom);
    if (n > 1) s.sort(0, n);
    for (size_t i = 0; i < n; ++i) {
      k[i] = e[i].key;
      vals[i] = e[i].val;
    }
    c = s.comparisons();
    r = s.rounds();
  }
  if (cmps) *cmps = c;
  if (rounds) *rounds = r;
  return 0;
}

// McIlroy's adversary ("a killer adversary for quicksort", 1999), written
// here from its published description: every element starts as "gas"
// (larger than all solid values); when two gas elements meet, the current
// pivot candidate is frozen to the next solid value.  Run against this
// oracle it yields an input on which that exact sort variant performs
// badly.
struct Adversary {
  std::vector<uint32_t> val;
  uint32_t gas, nsolid = 0;
  size_t candidate = 0;
  explicit Adversary(size_t n) : val(n, static_cast<uint32_t>(n)), gas(static_cast<uint32_t>(n)) {}
  void freeze(uint32_t x) { val[x] = nsolid++; }
};

struct AdversaryLess {
  Adversary* adv;
  bool operator()(uint32_t x, uint32_t y) const {
    Adversary& A = *adv;
    if (A.val[x] == A.gas && A.val[y] == A.gas) {
      if (x == A.candidate) {
        A.freeze(x);
      } else {
        A.freeze(y);
      }
    }
    if (A.val[x] == A.gas) {
      A.candidate = x;
    } else if (A.val[y] == A.gas) {
      A.candidate = y;
    }
    return A.val[x] < A.val[y];
  }
};

struct LessCounted {
  bool operator()(const Counted<uint32_t>& x, const Counted<uint32_t>& y) const {
    return x.v < y.v;
  }
};
using CountedU32 = Counted<uint32_t>;

}  // namespace

extern "C" {

// dtype: 0 = uint32, 1 = uint64, 2 = int64, 3 = float32.
// variant: 0 = median-of-3, 1 = median-of-sqrt(n), 2 = MoM, 3 = hybrid.
// mode: 0 = analysis (Fig. 3 alone), 1 = paper (base cases + duplicate guard).
// side: 0 = Fig. 3 (Mergesort the side left of the midpoint test),
//       1 = larger side whenever its buffer fits.
// vals: NULL for key-only sorts, else payloads moved with their keys.
int qms_ref_sort2(void* keys, uint32_t* vals, size_t n, int dtype, int variant,
                  int mode, int side, int mom, uint64_t* cmps, uint64_t* rounds) {
  if (keys == nullptr && n > 0) return -1;
  if (variant < 0 || variant > 3 || mode < 0 || mode > 1 || mom < 0 || mom > 1) return -1;
  switch (dtype) {
    case 0:
      return sort_typed<uint32_t, LessU32>(keys, vals, n, variant, mode, side, mom, cmps, rounds);
    case 1:
      return sort_typed<uint64_t, LessU64>(keys, vals, n, variant, mode, side, mom, cmps, rounds);
    case 2:
      return sort_typed<int64_t, LessI64>(keys, vals, n, variant, mode, side, mom, cmps, rounds);
    case 3:
      return sort_typed<float, LessF32>(keys, vals, n, variant, mode, side, mom, cmps, rounds);
    default:
      return -1;
  }
}

int qms_ref_sort(void* keys, uint32_t* vals, size_t n, int dtype, int variant,
                 int mode, int side, uint64_t* cmps, uint64_t* rounds) {
  return qms_ref_sort2(keys, vals, n, dtype, variant, mode, side, 0, cmps, rounds);
}

// The same sort on uint32 keys with element moves counted (Sec. 5: a move
// is an assignment of an input element; a swap counts three).
int qms_ref_moves_u32(uint32_t* keys, size_t n, int variant, int mode, int side, int mom,
                      uint64_t* cmps, uint64_t* moves) {
  if (keys == nullptr && n > 0) return -1;
  if (variant < 0 || variant > 3 || mode < 0 || mode > 1 || mom < 0 || mom > 1) return -1;
  std::vector<CountedU32> e(n);
  for (size_t i = 0; i < n; ++i) e[i].v = keys[i];
  CountedU32::moves = 0;
  QuickMergesort<CountedU32, LessCounted> s(e.data(), LessCounted{}, variant, mode, side, mom);
  if (n > 1) s.sort(0, n);
  const uint64_t mv = CountedU32::moves;
  for (size_t i = 0; i < n; ++i) keys[i] = e[i].v;
  if (cmps) *cmps = s.comparisons();
  if (moves) *moves = mv;
  return 0;
}

// QuickMergesort with the four-way swap-merge Mergesort (Sec. 6's
// multi-way merging) on uint32 keys; comparisons, rounds and element moves
// (a swap counts three) are reported.
int qms_ref_sort4_u32(uint32_t* keys, size_t n, int variant, int mode, uint64_t* cmps,
                      uint64_t* rounds, uint64_t* moves) {
  if (keys == nullptr && n > 0) return -1;
  if (variant < 0 || variant > 3 || mode < 0 || mode > 1) return -1;
  std::vector<CountedU32> e(n);
  for (size_t i = 0; i < n; ++i) e[i].v = keys[i];
  CountedU32::moves = 0;
  QuickMergesort<CountedU32, LessCounted> s(e.data(), LessCounted{}, variant, mode, 0);
  s.set_kway(4);
  if (n > 1) s.sort(0, n);
  const uint64_t mv = CountedU32::moves;
  for (size_t i = 0; i < n; ++i) keys[i] = e[i].v;
  if (cmps) *cmps = s.comparisons();
  if (rounds) *rounds = s.rounds();
  if (moves) *moves = mv;
  return 0;
}

// The four-way Mergesort alone: a[b, b + n) sorted in place with the buffer
// a[t, t + n) (to_target = 0), or into a[t, t + n) (to_target = 1).
int qms_ref_msort4_u32(uint32_t* a, size_t b, size_t n, size_t t, int to_target, int mode,
                       uint64_t* cmps, uint64_t* moves) {
  if (a == nullptr || mode < 0 || mode > 1) return -1;
  if (t < b + n && b < t + n) return -1;  // the regions must not overlap
  const size_t len = std::max(b + n, t + n);
  std::vector<CountedU32> v(len);
  for (size_t i = 0; i < len; ++i) v[i].v = a[i];
  CountedU32::moves = 0;
  QuickMergesort<CountedU32, LessCounted> s(v.data(), LessCounted{}, M3, mode, 0);
  if (to_target) s.msort4_to(b, n, t); else s.msort4_in(b, n, t);
  const uint64_t mv = CountedU32::moves;
  for (size_t i = 0; i < len; ++i) a[i] = v[i].v;
  if (cmps) *cmps = s.comparisons();
  if (moves) *moves = mv;
  return 0;
}

// Fig. 3 "out" alone with moves counted (see qms_ref_out_u32).
int qms_ref_out_moves_u32(uint32_t* a, size_t b, size_t e, size_t temp, int mode,
                          uint64_t* cmps, uint64_t* moves) {
  if (a == nullptr || e < b) return -1;
  const size_t r = (e - b) - (e - b) / 2;
  if (temp < e && temp + r > b) return -1;
  const size_t len = std::max(e, temp + r);
  std::vector<CountedU32> v(len);
  for (size_t i = 0; i < len; ++i) v[i].v = a[i];
  CountedU32::moves = 0;
  QuickMergesort<CountedU32, LessCounted> s(v.data(), LessCounted{}, M3, mode, 0);
  s.out(b, e, temp);
  const uint64_t mv = CountedU32::moves;
  for (size_t i = 0; i < len; ++i) a[i] = v[i].v;
  if (cmps) *cmps = s.comparisons();
  if (moves) *moves = mv;
  return 0;
}

// Test hook: the 6-comparison median of five used by the selection.  *pos
// receives the index (0..4) of the median within v[0..5) (v is not changed).
int qms_ref_median5_u32(const uint32_t* v, int* pos, uint64_t* cmps) {
  if (v == nullptr || pos == nullptr) return -1;
  uint32_t a[5];
  std::memcpy(a, v, sizeof(a));
  using Less = ByKey<uint32_t, LessU32>;
  QuickMergesort<uint32_t, Less> s(a, Less{}, MOM, ANALYSIS, 0);
  *pos = static_cast<int>(s.median5_pos(0));
  if (cmps) *cmps = s.comparisons();
  return 0;
}

// Test hook: groups-of-five selection of rank i in a[0, n) (rearranged in
// place); *pos receives the position of the selected element.  adaptive = 1
// uses the Sec. 4 adaptation.  trace (may be NULL) receives up to cap
// (n, kept) pairs, one per iteration at every recursion depth; *len their
// number.
int qms_ref_select_u32(uint32_t* a, size_t n, size_t i, int adaptive, size_t* pos,
                       uint64_t* cmps, uint64_t* trace, size_t cap, size_t* len) {
  if (a == nullptr || pos == nullptr || i >= n || adaptive < 0 || adaptive > 1) return -1;
  using Less = ByKey<uint32_t, LessU32>;
  QuickMergesort<uint32_t, Less> s(a, Less{}, MOM, PAPER, 0, adaptive);
  std::vector<SelRec> log;
  s.select_log = &log;
  *pos = s.select(0, n, i);
  if (cmps) *cmps = s.comparisons();
  if (len) *len = log.size();
  for (size_t j = 0; trace != nullptr && j < log.size() && j < cap; ++j) {
    trace[2 * j] = log[j].n;
    trace[2 * j + 1] = log[j].kept;
  }
  return 0;
}

// Test hook: sorts uint32 keys and records every partition round as eight
// words (b, e, lt, gt, mom, cmp_pivot, cmp_part, left): the range, the
// pivot block, whether the pivot was a median of medians, the comparisons
// spent choosing the pivot (everything but the partition of a MoM round),
// the partition comparisons of a MoM round, and whether the left side was
// Mergesorted.  Up to cap rounds are written; *len receives their number.
int qms_ref_rounds_u32(uint32_t* keys, size_t n, int variant, int mode, int side, int mom,
                       uint64_t* rec, size_t cap, size_t* len, uint64_t* cmps) {
  if (keys == nullptr && n > 0) return -1;
  if (variant < 0 || variant > 3 || mode < 0 || mode > 1 || mom < 0 || mom > 1) return -1;
  using Less = ByKey<uint32_t, LessU32>;
  QuickMergesort<uint32_t, Less> s(keys, Less{}, variant, mode, side, mom);
  std::vector<RoundRec> log;
  s.round_log = &log;
  if (n > 1) s.sort(0, n);
  if (len) *len = log.size();
  if (cmps) *cmps = s.comparisons();
  for (size_t j = 0; rec != nullptr && j < log.size() && j < cap; ++j) {
    const RoundRec& r = log[j];
    const uint64_t w[8] = {r.b, r.e, r.lt, r.gt, r.mom, r.cmp_pivot, r.cmp_part, r.left};
    std::memcpy(rec + 8 * j, w, sizeof(w));
  }
  return 0;
}

// Fig. 3 "out" with the QuickMergeXsort stopper: Mergesort of a[b, e) with
// the buffer at a[temp, ...), X = CleverQuicksort for msort calls below
// x_thresh elements.
int qms_ref_out_x_u32(uint32_t* a, size_t b, size_t e, size_t temp, int mode, size_t x_thresh,
                      uint64_t* cmps) {
  if (a == nullptr || e < b) return -1;
  const size_t r = (e - b) - (e - b) / 2;
  if (temp < e && temp + r > b) return -1;
  using Less = ByKey<uint32_t, LessU32>;
  QuickMergesort<uint32_t, Less> s(a, Less{}, M3, mode, 0, 0, x_thresh);
  s.out(b, e, temp);
  if (cmps) *cmps = s.comparisons();
  return 0;
}

// QuickMergeXsort on uint32 keys [Sec. 3]: the sort with x_thresh (X =
// CleverQuicksort below x_thresh elements inside Mergesort).
int qms_ref_qmqs_u32(uint32_t* keys, size_t n, int variant, int mode, size_t x_thresh,
                     uint64_t* cmps) {
  if ((keys == nullptr && n > 0) || variant < 0 || variant > 3 || mode < 0 || mode > 1) return -1;
  using Less = ByKey<uint32_t, LessU32>;
  QuickMergesort<uint32_t, Less> s(keys, Less{}, variant, mode, 0, 0, x_thresh);
  if (n > 1) s.sort(0, n);
  if (cmps) *cmps = s.comparisons();
  return 0;
}

// Exact average comparisons of the analysis-mode median-of-3 QuickMergeXsort
// with X = CleverQuicksort below x_thresh, on random permutations, by the
// same argument as qms_ref_dp: partitioning keeps both sides random, so
//   Q(n) = 8/3 + (n - 3) + sum_k Pr[k] (Q(k-1) + Q(n-k)),  Q(2) = 1,
//   X-msort(n) = Q(n) for n < x_thresh, else the two halves plus E,
//   out(n) = X-msort(floor(n/2)) + X-msort(ceil(n/2)) + E,
// and T(n) as in qms_ref_dp with out in place of Mergesort.
int qms_ref_dp_qmqs(size_t nmax, size_t x_thresh, double* T, double* Q) {
  if (T == nullptr || Q == nullptr) return -1;
  std::vector<double> MX(nmax + 1, 0.0), MO(nmax + 1, 0.0);
  auto pk = [](size_t n, size_t k) {
    const double nd = static_cast<double>(n);
    return static_cast<double>(k - 1) * static_cast<double>(n - k) / (nd * (nd - 1.0) * (nd - 2.0) / 6.0);
  };
  for (size_t n = 0; n <= nmax; ++n) {
    if (n <= 1) { Q[n] = 0.0; continue; }
    if (n == 2) { Q[n] = 1.0; continue; }
    double s = 0.0;
    for (size_t k = 1; k <= n; ++k) s += pk(n, k) * (Q[k - 1] + Q[n - k]);
    Q[n] = 8.0 / 3.0 + static_cast<double>(n - 3) + s;
  }
  auto E = [](double a, double b) { return a + b - a / (b + 1.0) - b / (a + 1.0); };
  for (size_t n = 0; n <= nmax; ++n) {
    if (n <= 1) { MX[n] = 0.0; MO[n] = 0.0; continue; }
    const size_t q = n / 2, r = n - q;
    const double e = E(static_cast<double>(q), static_cast<double>(r));
    MX[n] = (x_thresh > 0 && n < x_thresh) ? Q[n] : MX[q] + MX[r] + e;
    MO[n] = MX[q] + MX[r] + e;
  }
  for (size_t n = 0; n <= nmax; ++n) {
    if (n <= 1) { T[n] = 0.0; continue; }
    if (n == 2) { T[n] = 1.0; continue; }
    double s = 0.0;
    for (size_t k = 1; k <= n; ++k) {
      const double rest = (k - 1 < n / 2) ? (MO[k - 1] + T[n - k]) : (MO[n - k] + T[k - 1]);
      s += pk(n, k) * rest;
    }
    T[n] = 8.0 / 3.0 + static_cast<double>(n - 3) + s;
  }
  return 0;
}

// Mergesort alone (Fig. 3 "out"): sorts a[b, e) using the ceil((e-b)/2)
// slots a[temp, ...) as swap buffer; the buffer contents are permuted.  The
// buffer must not overlap [b, e).
int qms_ref_out_u32(uint32_t* a, size_t b, size_t e, size_t temp, int mode,
                    uint64_t* cmps) {
  if (a == nullptr || e < b) return -1;
  const size_t r = (e - b) - (e - b) / 2;
  if (temp < e && temp + r > b) return -1;
  using Less = ByKey<uint32_t, LessU32>;
  QuickMergesort<uint32_t, Less> s(a, Less{}, M3, mode, 0);
  s.out(b, e, temp);
  if (cmps) *cmps = s.comparisons();
  return 0;
}

// Exact average comparisons of the analysis-mode median-of-3 sort on
// random permutations of distinct keys, derived from the proof of Thm. 1:
// Pr[pivot rank = k] = (k-1)(n-k)/C(n,3), partitioning keeps both sides
// uniformly random, and the Mergesort of m elements costs M(m) on average
// with M(n) = M(floor(n/2)) + M(ceil(n/2)) + E(floor(n/2), ceil(n/2)),
// E(a, b) = a + b - a/(b+1) - b/(a+1) (expected comparisons of a merge
// that stops when one run is exhausted).  Fills T[0..nmax], M[0..nmax].
int qms_ref_dp(size_t nmax, double* T, double* M) {
  if (T == nullptr || M == nullptr) return -1;
  for (size_t n = 0; n <= nmax; ++n) {
    if (n <= 1) {
      M[n] = 0.0;
      continue;
    }
    const double a = static_cast<double>(n / 2), b = static_cast<double>(n - n / 2);
    M[n] = M[n / 2] + M[n - n / 2] + a + b - a / (b + 1.0) - b / (a + 1.0);
  }
  for (size_t n = 0; n <= nmax; ++n) {
    if (n <= 1) {
      T[n] = 0.0;
      continue;
    }
    if (n == 2) {
      T[n] = 1.0;
      continue;
    }
    const double nd = static_cast<double>(n);
    const double c3 = nd * (nd - 1.0) * (nd - 2.0) / 6.0;
    double s = 0.0;
    for (size_t k = 1; k <= n; ++k) {
      const double w = static_cast<double>(k - 1) * static_cast<double>(n - k);
      if (w == 0.0) continue;
      const double rest = (k - 1 < n / 2) ? (M[k - 1] + T[n - k]) : (M[n - k] + T[k - 1]);
      s += w * rest;
    }
    T[n] = 8.0 / 3.0 + (nd - 3.0) + s / c3;
  }
  return 0;
}

// Builds an input of n distinct uint32 keys (a permutation of 0..n-1) by
// running McIlroy's adversary against this oracle's sort with the given
// variant and mode.  Returns the comparisons the sort made on it.
int qms_ref_adversary_u32(uint32_t* out, size_t n, int variant, int mode,
                          uint64_t* cmps) {
  if (out == nullptr && n > 0) return -1;
  Adversary adv(n);
  std::vector<uint32_t> ids(n);
  for (size_t i = 0; i < n; ++i) ids[i] = static_cast<uint32_t>(i);
  AdversaryLess less{&adv};
  QuickMergesort<uint32_t, AdversaryLess> s(ids.data(), less, variant, mode, 0);
  if (n > 1) s.sort(0, n);
  // Elements never frozen keep their relative gas order: freeze them now in
  // index order so that the result is a permutation.
  for (size_t i = 0; i < n; ++i) {
    if (adv.val[i] == adv.gas) adv.freeze(static_cast<uint32_t>(i));
  }
  for (size_t i = 0; i < n; ++i) out[i] = adv.val[i];
  if (cmps) *cmps = s.comparisons();
  return 0;
}

}  // extern "C"
