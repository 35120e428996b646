// Host side of the GB300 QuickMergesort library: the C ABI declared in
// include/qms.h and the round driver that queues the kernels of
// qms_kernels.cuh.
//
// Driver (Fig. 3 "sort" of arXiv 1804.10062): while the remaining range is
// larger than one tile, choose a pivot, partition in place, Mergesort one
// side using the other side as swap buffer, continue on the other side; a
// last range of at most one tile is finished by the base case.  The host
// reads the left count of each partition (one small device-to-host copy per
// round) to size the Mergesort launches.

#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <random>
#include <string>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/qms.h"
#include "qms_cta.cuh"
#include "qms_merge.cuh"
#include "qms_graph.cuh"
#include "qms_batch.h"
#include "qms_host.h"

namespace qms {
namespace {

struct Err {
  int code;
};

inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw Err{QMS_ECUDA};
}

inline int xform_of(int dtype) {
  return dtype == QMS_F32 ? XF_F32 : (dtype == QMS_I64 ? XF_I64 : XF_NONE);
}

// Raises the dynamic shared-memory limit of a kernel on the current device.
template <class F>
void allow_smem(F* f, size_t bytes) {
  ck(smem_attr(reinterpret_cast<const void*>(f), bytes));
}

// Host mirror of the descriptor fields the driver reads back each round.
struct DescHead {
  unsigned long long cmp, L, mis, pivot;
};

// Device workspace for one sort: descriptor + per-tile counters.
constexpr size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of one sort's workspace: round descriptor, per-tile left
// counts, the two misplaced-rank prefixes, merge splits, overlapped-merge
// tile flags and the exchange warps' start tiles.
struct WsLayout {
  size_t counts = 0, pml = 0, pmr = 0, splits = 0, flags = 0, wtl = 0, wtr = 0, total = 0;
  constexpr explicit WsLayout(uint64_t n) {
    const uint64_t nt = n / PT + 2;
    const uint64_t ns = n / 1024 + 3;  // merge tiles of at least 1024 outputs
    const uint64_t nw = n / EXJ + 2;   // at most n / 2 misplaced ranks
    size_t off = round256(sizeof(Desc));
    counts = off;
    off += round256(nt * 4);
    pml = off;
    off += round256((nt + 1) * 8);
    pmr = off;
    off += round256((nt + 1) * 8);
    splits = off;
    off += round256(ns * 8);
    flags = off;  // overlapped-merge tile flags, one per split
    off += round256(ns * 4);
    wtl = off;
    off += round256(nw * 4);
    wtr = off;
    off += round256(nw * 4);
    total = off;
  }
};

// Status of a finished sort from the descriptor's error bits.
inline int err_code(unsigned err) {
  if (err == 0) return QMS_OK;
  return (err & kErrOvlWait) ? QMS_ETIMEOUT : QMS_EINTERNAL;
}

struct Workspace {
  unsigned char* base = nullptr;
  size_t bytes = 0;
  Desc* desc = nullptr;
  uint32_t* counts = nullptr;
  uint64_t* pml = nullptr;
  uint64_t* pmr = nullptr;
  uint64_t* splits = nullptr;
  unsigned* flags = nullptr;
  uint32_t* wtl = nullptr;
  uint32_t* wtr = nullptr;
  cudaStream_t st = nullptr;

  static size_t size_for(uint64_t n) { return WsLayout(n).total; }
  // Points the arrays into [p, p + size_for(n)).
  void place(unsigned char* p, uint64_t n) {
    const WsLayout w(n);
    desc = reinterpret_cast<Desc*>(p);
    counts = reinterpret_cast<uint32_t*>(p + w.counts);
    pml = reinterpret_cast<uint64_t*>(p + w.pml);
    pmr = reinterpret_cast<uint64_t*>(p + w.pmr);
    splits = reinterpret_cast<uint64_t*>(p + w.splits);
    flags = reinterpret_cast<unsigned*>(p + w.flags);
    wtl = reinterpret_cast<uint32_t*>(p + w.wtl);
    wtr = reinterpret_cast<uint32_t*>(p + w.wtr);
  }
  void alloc(uint64_t n, cudaStream_t s) {
    st = s;
    bytes = size_for(n);
    if (cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, s) != cudaSuccess) {
      base = nullptr;
      (void)cudaGetLastError();
      throw Err{QMS_ENOMEM};
    }
    place(base, n);
    ck(cudaMemsetAsync(desc, 0, sizeof(Desc), s));
  }
  ~Workspace() {
    if (base) cudaFreeAsync(base, st);
  }
};

// Records CUDA events around launches (profiling only) and accumulates the
// device time of each kernel class into a qms_profile after the stream has
// been synchronised.
class Profiler {
 public:
  explicit Profiler(qms_profile* out) : out_(out) {}
  bool active() const { return out_ != nullptr; }
  ~Profiler() {
    for (auto& r : recs_) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  }
  void begin(cudaStream_t st) {
    if (!out_) return;
    Rec r{};
    ck(cudaEventCreate(&r.a));
    ck(cudaEventCreate(&r.b));
    ck(cudaEventRecord(r.a, st));
    recs_.push_back(r);
  }
  void end(cudaStream_t st, int kind, uint64_t bytes) {
    if (!out_) return;
    Rec& r = recs_.back();
    r.kind = kind;
    r.bytes = bytes;
    ck(cudaEventRecord(r.b, st));
  }
  // Call after the stream has been synchronised.
  void flush() {
    if (!out_) return;
    for (auto& r : recs_) {
      float ms = 0.f;
      ck(cudaEventElapsedTime(&ms, r.a, r.b));
      out_->ms[r.kind] += ms;
      out_->bytes[r.kind] += r.bytes;
      out_->launches[r.kind] += 1;
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    recs_.clear();
  }

 private:
  struct Rec {
    cudaEvent_t a, b;
    int kind;
    uint64_t bytes;
  };
  qms_profile* out_;
  std::vector<Rec> recs_;
};

// Stores a partition pass's result (left count, misplaced pairs, tie and
// error bits) into mapped host memory for the host-driven driver.
__global__ void k_report(Desc* d, unsigned long long* out) {
  grid_dep_wait();
  grid_dep_trigger();
  if (threadIdx.x != 0) return;
  out[0] = d->L;
  out[1] = d->mis;
  out[2] = static_cast<unsigned long long>(d->tie) | (static_cast<unsigned long long>(d->err) << 32);
  d->L = 0;  // a further pass of the round counts from zero
  __threadfence_system();
}

// Mapped pinned host words for k_report, one block per host thread and
// device (host-driven sorts are synchronous, so a thread runs one at a time);
// allocated on first use and kept.  Null if the allocation fails.
unsigned long long* report_words() {
  struct Slots {
    std::map<int, unsigned long long*> by_dev;
    ~Slots() {
      for (auto& kv : by_dev) cudaFreeHost(kv.second);
    }
  };
  thread_local Slots slots;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  auto it = slots.by_dev.find(dev);
  if (it != slots.by_dev.end()) return it->second;
  void* p = nullptr;
  if (cudaHostAlloc(&p, 64, cudaHostAllocMapped) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  slots.by_dev[dev] = static_cast<unsigned long long*>(p);
  return static_cast<unsigned long long*>(p);
}

template <class K, bool HV, bool CNT>
class Sorter {
 public:
  Sorter(K* keys, uint32_t* vals, int xf, cudaStream_t st, Workspace& ws, Profiler& prof)
      : keys_(keys), vals_(vals), xf_(xf), st_(st), ws_(ws), prof_(prof) {
    allow_smem(k_leaf_sort<K, HV, CNT>,
               tile_smem_bytes<K, HV, LeafCfg<K, HV>::LT, LeafCfg<K, HV>::VL>());
    allow_smem(k_pivot_sample<K, HV, CNT>, tile_smem_bytes<K, true, SAMPLE_T, V>());
  }

  uint64_t rounds = 0, mom_rounds = 0, launches = 0;
  uint64_t exchanged_bytes = 0;  // algorithmic bytes of the exchange steps
  bool fig3_side = true;         // Fig. 3's side rule; false: the larger side when it fits
  unsigned spin_limit = kOvlSpinLimit;  // polls of one flag in a bounded device wait
  int withhold = 0;                     // test hook (QMS_FLAG_TEST_WITHHOLD)
  // Mapped pinned host words the round results are stored to (null: the
  // results are copied back with cudaMemcpyAsync instead).
  unsigned long long* report_ = nullptr;

  // ---- steps ------------------------------------------------------------

  static constexpr uint64_t ES = sizeof(K) + (HV ? 4 : 0);  // bytes per element

  void leaf(uint64_t P, uint64_t m, bool to_buf, uint64_t Bb) {
    if (m == 0) return;
    using LC = LeafCfg<K, HV>;
    const uint64_t nt = (m + LC::TILE_L - 1) / LC::TILE_L;
    prof_.begin(st_);
    launch(k_leaf_sort<K, HV, CNT>, grid_of(nt), LC::LT, tile_smem_bytes<K, HV, LC::LT, LC::VL>(), keys_,
           vals_, P, m, Bb, to_buf ? 1 : 0, xf_, ws_.desc);
    prof_.end(st_, QMS_K_LEAF, (to_buf ? 4 : 2) * m * ES);
    launched();
  }

  // Mergesort of P[0, m) with the disjoint buffer Bb[0, m) (Fig. 3 "out"
  // with a full-size buffer: every level merges one region into the other).
  // The sorted keys end in P, or with into_buf in Bb (and Bb's old contents
  // in P).
  void mergesort(uint64_t P, uint64_t m, uint64_t Bb, bool into_buf = false) {
    if (m == 0 || (m == 1 && !into_buf)) return;
    constexpr uint64_t TL = LeafCfg<K, HV>::TILE_L;
    if (m <= TL && !into_buf) {
      leaf(P, m, false, 0);
      return;
    }
    const uint64_t leaves = (m + TL - 1) / TL;
    int levels = 0;
    while ((1ull << levels) < leaves) ++levels;
    // each level moves the runs to the other region
    const bool to_buf = ((levels & 1) != 0) != into_buf;
    leaf(P, m, to_buf, Bb);
    uint64_t X = to_buf ? Bb : P, Y = to_buf ? P : Bb;
    constexpr uint64_t MT = MergeCfg<K, HV>::MT;
    const uint64_t mtiles = (m + MT - 1) / MT;
    for (int l = 0; l < levels; ++l) {
      const uint64_t L = TL << l;
      prof_.begin(st_);
      launch(k_merge_split3<K, HV, CNT>, grid_of((mtiles + 255) / 256), 256, 0,
             static_cast<const K*>(keys_), X, m, L, xf_, ws_.splits, ws_.desc);
      prof_.end(st_, QMS_K_MERGE_SPLIT, 0);
      prof_.begin(st_);
      launch_merge(X, Y, m, L, mtiles);
      prof_.end(st_, QMS_K_MERGE, 4 * m * ES);
      launched(2);
      std::swap(X, Y);
    }
  }

  // Fig. 3 "out" with its half-size buffer: sorts P[0, m) using the
  // ceil(m/2) slots Bb[0, ceil(m/2)) (disjoint from the part).  The second
  // half is sorted into the buffer, the first half into the tail of the
  // part, then the overlapped merge fills the part; the buffer's elements
  // end, permuted, in Bb.
  void out_half(uint64_t P, uint64_t m, uint64_t Bb) {
    if (m <= 1) return;
    const uint64_t q = m / 2, r = m - q;
    mergesort(P + q, r, Bb, true);
    mergesort(P, q, P + r, true);
    constexpr uint64_t MT = MergeCfg<K, HV>::MT;
    const uint64_t mtiles = (m + MT - 1) / MT;
    prof_.begin(st_);
    k_ovl_split<K, HV, CNT><<<grid_of((mtiles + 255) / 256), 256, 0, st_>>>(
        keys_, Bb, r, P, q, xf_, ws_.splits, ws_.flags, ws_.desc);
    // wait ranges in the exchange start tables (unused outside partitions)
    k_ovl_deps<K, HV><<<grid_of((mtiles + 255) / 256), 256, 0, st_>>>(r, q, ws_.splits, ws_.wtl,
                                                                      ws_.wtr);
    prof_.end(st_, QMS_K_MERGE_SPLIT, 0);
    prof_.begin(st_);
    k_ovl_merge<K, HV, CNT><<<grid_of(mtiles), MBT, 0, st_>>>(
        keys_, vals_, Bb, r, P, q, ws_.splits, ws_.wtl, ws_.wtr, ws_.flags, xf_, ws_.desc,
        spin_limit, withhold);
    prof_.end(st_, QMS_K_MERGE, 4 * m * ES);
    launched(3);
  }

  // Parks a pivot of [b, e) at e - 1 (rule: QMS_PIVOT_*, MOM for HYBRID's
  // fallback rounds).
  void pivot(uint64_t b, uint64_t e, int rule) {
    const uint64_t n = e - b;
    prof_.begin(st_);
    if (rule == QMS_PIVOT_SQRTN) {
      uint64_t c = 1;
      while (c * c < n) ++c;  // ceil(sqrt(n)); n < 2^40 here
      uint64_t k = (c & 1) ? c : c - 1;
      if (k > static_cast<uint64_t>(SAMPLE_MAX)) k = SAMPLE_MAX;
      if (k < 1) k = 1;
      const uint64_t step = n / k;
      launch(k_pivot_sample<K, HV, CNT>, 1, SAMPLE_T, tile_smem_bytes<K, true, SAMPLE_T, V>(), keys_, vals_,
             b, e, static_cast<int>(k), step, xf_, ws_.desc);
      launched();
    } else if (rule == QMS_PIVOT_MOM) {
      const uint64_t t = n / 3;
      const unsigned g = static_cast<unsigned>(std::min<uint64_t>((t + 255) / 256, 1u << 20));
      k_mom_triples<K, HV, CNT><<<g, 256, 0, st_>>>(keys_, vals_, b, t, xf_, ws_.desc);
      launched();
      // radix select of rank floor(t/2) among the medians
      unsigned long long init[4] = {0ull, 0ull, static_cast<unsigned long long>(t / 2), 0ull};
      ck(cudaMemcpyAsync(&ws_.desc->sel_prefix, init, sizeof(init), cudaMemcpyHostToDevice, st_));
      ck(cudaMemsetAsync(ws_.desc->hist, 0, sizeof(ws_.desc->hist), st_));
      for (int shift = static_cast<int>(sizeof(K) * 8) - 8; shift >= 0; shift -= 8) {
        k_sel_hist<K><<<g, 256, 0, st_>>>(keys_, b, t, xf_, shift, ws_.desc);
        k_sel_pick<<<1, 32, 0, st_>>>(shift, ws_.desc);
        launched(2);
      }
      const unsigned long long big = ~0ull;
      ck(cudaMemcpyAsync(&ws_.desc->pos, &big, sizeof(big), cudaMemcpyHostToDevice, st_));
      k_mom_locate<K><<<g, 256, 0, st_>>>(keys_, b, t, xf_, ws_.desc);
      k_mom_place<K, HV><<<1, 32, 0, st_>>>(keys_, vals_, b, e, t, ws_.desc);
      launched(2);
      ++mom_rounds;
    } else {
      launch(k_pivot_m3<K, HV, CNT>, 1, 32, 0, keys_, vals_, b, e, xf_, ws_.desc);
      launched();
    }
    prof_.end(st_, QMS_K_PIVOT, 0);
  }

  // Partitions [lo, hi) around the descriptor's pivot (le: "<=" pass);
  // when parked != ~0 the pivot parked there moves to lo + L afterwards.
  // Returns L, the number of left elements.
  uint64_t partition(uint64_t lo, uint64_t hi, bool le, uint64_t parked, unsigned* tie) {
    const uint64_t n = hi - lo;
    const uint64_t nt = (n + PT - 1) / PT;
    if (n > 0) {
      // L starts at zero: reset by the pivot kernel before a round's first
      // pass and by k_report after it (else here)
      if (!report_) ck(cudaMemsetAsync(&ws_.desc->L, 0, sizeof(unsigned long long), st_));
      prof_.begin(st_);
      launch(k_part_local<K, HV, CNT>, grid_of(nt), PNT, 0, keys_, vals_, lo, hi, le ? 1 : 0, xf_,
             ws_.desc, ws_.counts);
      prof_.end(st_, QMS_K_PART_LOCAL, 2 * n * ES);
      const uint64_t ch = scan_chunk(nt);
      const unsigned nch = static_cast<unsigned>((nt + ch - 1) / ch);
      prof_.begin(st_);
      launch(k_part_chunks, nch, NT, 0, lo, hi, static_cast<const uint32_t*>(ws_.counts), ws_.desc);
      launch(k_part_prefix, nch, NT, 0, lo, hi, static_cast<const uint32_t*>(ws_.counts), ws_.pml,
             ws_.pmr, ws_.wtl, ws_.wtr, ws_.desc);
      prof_.end(st_, QMS_K_PART_SCAN, nt * 20);
      launched();
      const uint64_t maxmis = n / 2 + 1;
      const uint64_t per = static_cast<uint64_t>(EXB) * EXW;
      prof_.begin(st_);
      const unsigned gx = grid_of((maxmis + per - 1) / per);
      const uint32_t* cnts = ws_.counts;
      const uint64_t* pl = ws_.pml;
      const uint64_t* pr = ws_.pmr;
      const uint32_t* tl = ws_.wtl;
      const uint32_t* tr = ws_.wtr;
      const Desc* dc = ws_.desc;
      if (n < (1ull << 32)) {
        launch(k_part_exchange<K, HV, uint32_t>, gx, EXB, 0, keys_, vals_, lo, cnts, pl, pr, tl, tr, dc);
      } else {
        launch(k_part_exchange<K, HV, uint64_t>, gx, EXB, 0, keys_, vals_, lo, cnts, pl, pr, tl, tr, dc);
      }
      prof_.end(st_, QMS_K_PART_EXCHANGE, 0);  // bytes added once mis is known
      launched(3);
    } else if (!report_) {
      ck(cudaMemsetAsync(&ws_.desc->L, 0, sizeof(unsigned long long), st_));
    }
    if (parked != ~0ull) {
      prof_.begin(st_);
      launch(k_place_pivot<K, HV>, 1, 32, 0, keys_, vals_, lo, parked, ws_.desc);
      prof_.end(st_, QMS_K_PIVOT, 0);
      launched();
    }
    struct {
      unsigned long long L, mis;
      unsigned tie, err;
    } h;
    if (report_) {
      // A kernel stores the round's result into mapped host memory: no copy
      // engine is involved, so the read-back does not queue behind large
      // copies that other streams may have in flight.
      launch(k_report, 1, 32, 0, ws_.desc, report_);
      ck(cudaStreamSynchronize(st_));
      const volatile unsigned long long* r = report_;
      h.L = r[0];
      h.mis = r[1];
      h.tie = static_cast<unsigned>(r[2]);
      h.err = static_cast<unsigned>(r[2] >> 32);
    } else {
      ck(cudaMemcpyAsync(&h.L, &ws_.desc->L, 2 * sizeof(h.L), cudaMemcpyDeviceToHost, st_));
      ck(cudaMemcpyAsync(&h.tie, &ws_.desc->tie, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st_));
      ck(cudaStreamSynchronize(st_));
    }
    ck(cudaGetLastError());
    if (h.err) throw Err{err_code(h.err)};
    if (tie) *tie = h.tie;
    exchanged_bytes += (n > 0) ? 4 * h.mis * ES : 0;
    return h.L;
  }

  // One round on [b, e): returns the pivot block [k, k + 1 + eq).
  void split(uint64_t b, uint64_t e, int rule, uint64_t* k, uint64_t* eq) {
    pivot(b, e, rule);
    unsigned tie = 0;
    const uint64_t L = partition(b, e - 1, false, e - 1, &tie);
    *k = b + L;
    *eq = 0;
    if (tie && *k + 1 < e) *eq = partition(*k + 1, e, true, ~0ull, nullptr);
  }

  void sort(uint64_t n, int rule) {
    uint64_t b = 0, e = n;
    bool mom_next = false;
    while (e - b > static_cast<uint64_t>(LeafCfg<K, HV>::TILE_L)) {
      ++rounds;
      const uint64_t nn = e - b;
      const bool mom = rule == QMS_PIVOT_MOM || (rule == QMS_PIVOT_HYBRID && mom_next);
      const int r = mom ? QMS_PIVOT_MOM : (rule == QMS_PIVOT_SQRTN ? QMS_PIVOT_SQRTN : QMS_PIVOT_M3);
      uint64_t k, eq;
      split(b, e, r, &k, &eq);
      if (rule == QMS_PIVOT_HYBRID) {
        const uint64_t d = nn / 16, rlo = k - b, rhi = k + eq - b;
        mom_next = !mom && (rhi < d || rlo > nn - 1 - d);
      }
      const uint64_t rb = k + 1 + eq;
      const uint64_t nl = k - b, nr = e - rb;
      const int side = choose_side(b, e, k, eq, fig3_side);
      if (side == SIDE_LARGER_LEFT) {
        out_half(b, nl, rb);
        b = rb;
      } else if (side == SIDE_LARGER_RIGHT) {
        out_half(rb, nr, b);
        e = k;
      } else if (side == SIDE_LEFT) {
        mergesort(b, nl, rb);
        b = rb;
      } else {
        mergesort(rb, nr, b);
        e = k;
      }
    }
    if (e - b > 1) leaf(b, e - b, false, 0);
  }

  void launched(int c = 1) { launches += c; }

  // Launches a kernel of the round loop.  Unless its time is being
  // profiled, with a programmatic dependency on the kernel before it: the
  // kernel's blocks may start during the previous kernel's last wave and
  // wait (grid_dep_wait) for its results, which hides the launch gap; the
  // merge kernel loads its buffer tile before that wait.
  template <class... KA, class... A>
  void launch(void (*k)(KA...), unsigned grid, unsigned block, size_t smem, A... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st_;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (prof_.active() || no_pdl()) ? 0 : 1;
    ck(cudaLaunchKernelEx(&cfg, k, static_cast<KA>(args)...));
  }
  static bool no_pdl() {
    static const bool v = std::getenv("QMS_NO_PDL") != nullptr;
    return v;
  }
  void launch_merge(uint64_t X, uint64_t Y, uint64_t m, uint64_t L, uint64_t mtiles) {
    launch(k_merge_level3<K, HV, CNT>, grid_of(mtiles), MBT, 0, keys_, vals_, X, Y, m, L,
           static_cast<const uint64_t*>(ws_.splits), xf_, ws_.desc);
  }

 private:
  static unsigned grid_of(uint64_t blocks) {
    if (blocks < 1) blocks = 1;
    return static_cast<unsigned>(std::min<uint64_t>(blocks, 1u << 30));
  }

  K* keys_;
  uint32_t* vals_;
  int xf_;
  cudaStream_t st_;
  Workspace& ws_;
  Profiler& prof_;
};

// ---------------------------------------------------------------------------
// Device-driven sort: one instantiated CUDA graph per (key type, payload,
// counting, pivot rule, device) instance, holding the whole round loop
// (qms_graph.cuh).  A call writes the keys' address and size into the
// instance's device state and launches the graph; the host does not wait
// between rounds.  Graphs with conditional nodes allow one instantiation
// each, so concurrent calls use separate instances from a pool.

struct GraphInst {
  cudaGraphDeviceNode_t dn[DN_COUNT] = {};
  unsigned int gcap[DN_COUNT] = {};  // built-in grid of each work node
  unsigned int dyn = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DState* d_state = nullptr;
  DState* h_state = nullptr;  // pinned copy read back for the statistics
  unsigned char* ws = nullptr;
  uint64_t cap = 0;
  size_t ws_bytes = 0;
  cudaEvent_t done = nullptr;    // recorded after the instance's last launch
  cudaStream_t last = nullptr;   // stream of that launch
  bool used = false;             // launched at least once
  bool wide = false;             // built for arrays of 2^32 keys or more
  bool busy = false;             // a call is setting it up on the host
};

inline size_t graph_ws_bytes(uint64_t cap) { return WsLayout(cap).total; }

std::mutex g_graph_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::vector<GraphInst*>> g_graphs;

// Adds a kernel node after `dep`.  programmatic: the edge is a programmatic
// dependency (the kernel may start once every block of `dep` has called
// griddepcontrol.launch_dependents, and waits for dep's completion with
// griddepcontrol.wait); if the runtime refuses that edge, an ordinary one.
cudaGraphNode_t add_kernel(cudaGraph_t g, cudaGraphNode_t dep, const void* func, unsigned grid,
                           unsigned block, size_t smem, void** args,
                           cudaGraphDeviceNode_t* devnode = nullptr, bool programmatic = false) {
  cudaKernelNodeParams p{};
  p.func = const_cast<void*>(func);
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.sharedMemBytes = static_cast<unsigned>(smem);
  p.kernelParams = args;
  p.extra = nullptr;
  cudaGraphNode_t n = nullptr;
  if (programmatic && dep) {
    ck(cudaGraphAddKernelNode(&n, g, nullptr, 0, &p));
    cudaGraphEdgeData e{};
    e.from_port = cudaGraphKernelNodePortProgrammatic;
    e.type = cudaGraphDependencyTypeProgrammatic;
    if (cudaGraphAddDependencies(g, &dep, &n, &e, 1) != cudaSuccess) {
      (void)cudaGetLastError();
      ck(cudaGraphAddDependencies(g, &dep, &n, nullptr, 1));
    }
  } else {
    ck(cudaGraphAddKernelNode(&n, g, dep ? &dep : nullptr, dep ? 1 : 0, &p));
  }
  if (devnode) {
    // Device-updatable: the control kernels size its grid to the work.
    cudaKernelNodeAttrValue v{};
    v.deviceUpdatableKernelNode.deviceUpdatable = 1;
    *devnode = nullptr;
    if (cudaGraphKernelNodeSetAttribute(n, cudaLaunchAttributeDeviceUpdatableKernelNode, &v) ==
        cudaSuccess) {
      cudaKernelNodeAttrValue o{};
      if (cudaGraphKernelNodeGetAttribute(n, cudaLaunchAttributeDeviceUpdatableKernelNode, &o) ==
          cudaSuccess)
        *devnode = o.deviceUpdatableKernelNode.devNode;
    }
    (void)cudaGetLastError();
  }
  return n;
}

cudaGraphNode_t add_cond(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
                         cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t n = nullptr;
  ck(cudaGraphAddNode(&n, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &cp));
  *body = cp.conditional.phGraph_out[0];
  return n;
}

template <class K, bool HV, bool CNT>
class GraphRunner {
 public:
  // Builds the graph of one instance (kernel arguments: the instance's
  // device state and the three condition handles).
  static void build(GraphInst* gi, int pivot, bool half) {
    build_impl(gi, pivot, true, half, std::getenv("QMS_NO_PDL") == nullptr);
  }

  // The exchange kernel of this graph: 32-bit positions unless the graph
  // serves arrays of 2^32 keys or more.
  static const void* exchange_kernel(bool wide) {
    return wide ? reinterpret_cast<const void*>(k_g_part_exchange<K, HV, uint64_t>)
                : reinterpret_cast<const void*>(k_g_part_exchange<K, HV, uint32_t>);
  }

  // half: the round body also holds the larger-side machinery (two Mergesort
  // phases and the overlapped merge); without it a round runs Fig. 3's rule
  // with no extra conditional nodes.  pdl: the merge node depends on the
  // split node programmatically (it starts while the split runs and loads
  // its buffer tiles first).
  static void build_impl(GraphInst* gi, int pivot, bool dyn, bool half, bool pdl) {
    int dev = 0, sms = 0;
    ck(cudaGetDevice(&dev));
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    using LC = LeafCfg<K, HV>;
    const size_t tsm = tile_smem_bytes<K, HV>(), tsm_s = tile_smem_bytes<K, true, SAMPLE_T, V>();
    const size_t tsm_l = tile_smem_bytes<K, HV, LC::LT, LC::VL>();
    allow_smem(k_g_leaf<K, HV, CNT>, tsm_l);
    allow_smem(k_g_final<K, HV, CNT>, tsm_l);
    allow_smem(k_g_pivot_sample<K, HV, CNT>, tsm_s);
    auto occ = [&](const void* f, int block, size_t smem) {
      int o = 0;
      ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, f, block, smem));
      return static_cast<unsigned>(sms * std::max(o, 1));
    };
    // Grid caps in waves of resident blocks (the control kernels size each
    // node to its work up to these), from sweeps at 2^28 keys: leaves 8
    // waves (2: 18.72 ms per sort, 8: 18.65), partition tiles 4 (18.68).
    // (QMS_*_WAVES environment variables override the caps for experiments.)
    auto waves = [&](const char* env, unsigned dflt, unsigned per_wave) {
      const char* v = std::getenv(env);
      const unsigned w = (v && dyn) ? static_cast<unsigned>(std::max(1, std::atoi(v))) : dflt;
      return per_wave * w;
    };
    const unsigned g_part =
        waves("QMS_PART_WAVES", 4, occ(reinterpret_cast<const void*>(k_g_part_local<K, HV, CNT>), PNT, 0));
    const unsigned g_leaf =
        waves("QMS_LEAF_WAVES", 8, occ(reinterpret_cast<const void*>(k_g_leaf<K, HV, CNT>), LC::LT, tsm_l));
    const unsigned g_exch =
        waves("QMS_EXCH_WAVES", 2, occ(exchange_kernel(gi->wide), EXB, 0));
    const unsigned g_split = static_cast<unsigned>(sms) * 4;
    // Eight waves of merge blocks that loop over the tiles: one block per tile
    // costs more in the level-end counter (one atomic per block) than it
    // gains, two waves too few (2^28 keys: 18.6 / 18.4 / 19.0 ms per sort).
    // With fixed grids every block of the node runs on every level, however
    // small, so there it stays at two waves.
    const unsigned g_merge = dyn ? waves("QMS_MERGE_WAVES", 8,
                                         occ(reinterpret_cast<const void*>(k_g_merge<K, HV, CNT>), MBT, 0))
                                 : occ(reinterpret_cast<const void*>(k_g_merge<K, HV, CNT>), MBT, 0) * 2;
    // Tiles are handed out through a ticket: with device-sized grids one
    // block per tile, else one wave of blocks that loop.
    const unsigned g_omerge =
        dyn ? (1u << 30) : occ(reinterpret_cast<const void*>(k_g_ovl_merge<K, HV, CNT>), MBT, 0);
    const unsigned g_mom = static_cast<unsigned>(sms) * 8;

    cudaGraph_t g = nullptr;
    ck(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h_round, h_pass2, h_level, h_phase = 0, h_ovl = 0;
    ck(cudaGraphConditionalHandleCreate(&h_round, g, 0, cudaGraphCondAssignDefault));
    ck(cudaGraphConditionalHandleCreate(&h_pass2, g, 0, cudaGraphCondAssignDefault));
    ck(cudaGraphConditionalHandleCreate(&h_level, g, 0, cudaGraphCondAssignDefault));
    if (half) {
      ck(cudaGraphConditionalHandleCreate(&h_phase, g, 0, cudaGraphCondAssignDefault));
      ck(cudaGraphConditionalHandleCreate(&h_ovl, g, 0, cudaGraphCondAssignDefault));
    }
    DState* S = gi->d_state;
    void* a_s[] = {&S};
    void* a_round[] = {&S, &h_round};
    void* a_pass2[] = {&S, &h_pass2};
    void* a_level[] = {&S, &h_level};
    void* a_side[] = {&S, &h_level, &h_phase, &h_ovl};
    void* a_phase[] = {&S, &h_phase, &h_level};
    cudaGraph_t body = nullptr;
    cudaGraphNode_t start = add_kernel(g, nullptr, reinterpret_cast<const void*>(k_g_start<K, HV>), 1,
                                       32, 0, a_round);
    cudaGraphNode_t w_round = add_cond(g, start, h_round, cudaGraphCondTypeWhile, &body);
    cudaGraphNode_t n = add_kernel(body, nullptr, reinterpret_cast<const void*>(k_g_begin<K, HV, CNT>),
                                   1, 32, 0, a_round);
    if (pivot == QMS_PIVOT_SQRTN) {
      n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_pivot_sample<K, HV, CNT>), 1, SAMPLE_T,
                     tsm_s, a_s);
    }
    if (pivot == QMS_PIVOT_MOM || pivot == QMS_PIVOT_HYBRID) {
      n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_mom_triples<K, HV, CNT>), g_mom, 256,
                     0, a_s);
      for (int shift = static_cast<int>(sizeof(K) * 8) - 8; shift >= 0; shift -= 8) {
        int sh = shift;
        void* a_sh[] = {&S, &sh};
        n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_sel_hist<K>), g_mom, 256, 0, a_sh);
        n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_sel_pick), 1, 32, 0, a_sh);
      }
      n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_mom_locate<K>), g_mom, 256, 0, a_s);
      n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_mom_place<K, HV>), 1, 32, 0, a_s);
    }
    cudaGraphDeviceNode_t* dn = dyn ? gi->dn : nullptr;
    gi->gcap[DN_PART1] = gi->gcap[DN_PART2] = g_part;
    gi->gcap[DN_EXCH1] = gi->gcap[DN_EXCH2] = g_exch;
    gi->gcap[DN_LEAF] = g_leaf;
    gi->gcap[DN_SPLIT] = g_split;
    gi->gcap[DN_MERGE] = g_merge;
    gi->gcap[DN_OSPLIT] = gi->gcap[DN_ODEPS] = g_split;
    gi->gcap[DN_OMERGE] = g_omerge;
    const unsigned g_scan = 1024;  // at most 1024 chunks
    gi->gcap[DN_CHUNK1] = gi->gcap[DN_PREF1] = gi->gcap[DN_CHUNK2] = gi->gcap[DN_PREF2] = g_scan;
    auto add_pass = [&](cudaGraph_t gr, cudaGraphNode_t d, int ip, int ie) {
      d = add_kernel(gr, d, reinterpret_cast<const void*>(k_g_part_local<K, HV, CNT>), g_part, PNT, 0,
                     a_s, dn ? dn + ip : nullptr);
      const int ic = (ip == DN_PART1) ? DN_CHUNK1 : DN_CHUNK2;
      const int ipf = (ip == DN_PART1) ? DN_PREF1 : DN_PREF2;
      d = add_kernel(gr, d, reinterpret_cast<const void*>(k_g_part_chunks), g_scan, NT, 0, a_s,
                     dn ? dn + ic : nullptr);
      d = add_kernel(gr, d, reinterpret_cast<const void*>(k_g_part_prefix), g_scan, NT, 0, a_s,
                     dn ? dn + ipf : nullptr);
      d = add_kernel(gr, d, exchange_kernel(gi->wide), g_exch, EXB, 0, a_s, dn ? dn + ie : nullptr);
      return d;
    };
    n = add_pass(body, n, DN_PART1, DN_EXCH1);
    n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_mid<K, HV>), 1, 32, 0, a_pass2);
    cudaGraph_t p2 = nullptr;
    n = add_cond(body, n, h_pass2, cudaGraphCondTypeIf, &p2);
    add_pass(p2, nullptr, DN_PART2, DN_EXCH2);
    auto add_levels = [&](cudaGraph_t gr, cudaGraphNode_t d) {
      d = add_kernel(gr, d, reinterpret_cast<const void*>(k_g_leaf<K, HV, CNT>), g_leaf, LC::LT, tsm_l,
                     a_s, dn ? dn + DN_LEAF : nullptr);
      cudaGraph_t lv = nullptr;
      d = add_cond(gr, d, h_level, cudaGraphCondTypeWhile, &lv);
      cudaGraphNode_t q = add_kernel(lv, nullptr, reinterpret_cast<const void*>(k_g_split<K, HV, CNT>),
                                     g_split, 256, 0, a_s, dn ? dn + DN_SPLIT : nullptr);
      add_kernel(lv, q, reinterpret_cast<const void*>(k_g_merge<K, HV, CNT>), g_merge, MBT, 0, a_level,
                 dn ? dn + DN_MERGE : nullptr, pdl);
      return d;
    };
    if (!half) {
      n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_side<K, HV, false>), 1, 32, 0, a_side);
      n = add_levels(body, n);
    } else {
      n = add_kernel(body, n, reinterpret_cast<const void*>(k_g_side<K, HV, true>), 1, 32, 0, a_side);
      // Mergesort phases: one (Fig. 3 rule) or two (half-buffer rounds)
      cudaGraph_t ph = nullptr;
      n = add_cond(body, n, h_phase, cudaGraphCondTypeWhile, &ph);
      cudaGraphNode_t p = add_levels(ph, nullptr);
      add_kernel(ph, p, reinterpret_cast<const void*>(k_g_phase_end<K, HV>), 1, 32, 0, a_phase);
      // the overlapped final merge of half-buffer rounds
      cudaGraph_t ov = nullptr;
      n = add_cond(body, n, h_ovl, cudaGraphCondTypeIf, &ov);
      cudaGraphNode_t q = add_kernel(ov, nullptr, reinterpret_cast<const void*>(k_g_ovl_split<K, HV, CNT>),
                                     g_split, 256, 0, a_s, dn ? dn + DN_OSPLIT : nullptr);
      q = add_kernel(ov, q, reinterpret_cast<const void*>(k_g_ovl_deps<K, HV>), g_split, 256, 0, a_s,
                     dn ? dn + DN_ODEPS : nullptr);
      add_kernel(ov, q, reinterpret_cast<const void*>(k_g_ovl_merge<K, HV, CNT>), g_omerge, MBT, 0, a_s,
                 dn ? dn + DN_OMERGE : nullptr);
    }
    add_kernel(body, n, reinterpret_cast<const void*>(k_g_end<K, HV>), 1, 32, 0, a_round);
    add_kernel(g, w_round, reinterpret_cast<const void*>(k_g_final<K, HV, CNT>), 1, LC::LT, tsm_l, a_s);
    bool all = dyn;
    for (int i = 0; i < DN_COUNT && dyn; ++i) {
      const bool ovl_node = (i == DN_OSPLIT || i == DN_ODEPS || i == DN_OMERGE);
      if (!half && ovl_node) continue;  // not part of this graph
      all = all && gi->dn[i] != nullptr;
    }
    if (dyn && !all) {  // some node is not device-updatable: fixed grids throughout
      cudaGraphDestroy(g);
      for (int i = 0; i < DN_COUNT; ++i) gi->dn[i] = nullptr;
      build_impl(gi, pivot, false, half, pdl);
      return;
    }
    gi->dyn = all ? 1u : 0u;
    if (cudaGraphInstantiate(&gi->exec, g, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaGraphDestroy(g);
      for (int i = 0; i < DN_COUNT; ++i) gi->dn[i] = nullptr;
      if (pdl) {  // programmatic edges not accepted here: ordinary edges
        build_impl(gi, pivot, dyn, half, false);
        return;
      }
      if (dyn) {  // device-updatable nodes not accepted here: fixed grids
        build_impl(gi, pivot, false, half, false);
        return;
      }
      throw Err{QMS_ECUDA};
    }
    if (gi->dyn && cudaGraphUpload(gi->exec, nullptr) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaGraphExecDestroy(gi->exec);
      cudaGraphDestroy(g);
      for (int i = 0; i < DN_COUNT; ++i) gi->dn[i] = nullptr;
      build_impl(gi, pivot, false, half, false);
      return;
    }
    gi->graph = g;
    if (std::getenv("QMS_VERBOSE"))
      std::fprintf(stderr, "qms: graph built (K=%zu HV=%d CNT=%d pivot=%d): %s grids%s\n", sizeof(K),
                   HV ? 1 : 0, CNT ? 1 : 0, pivot, gi->dyn ? "device-sized" : "fixed",
                   pdl ? ", programmatic split-merge edge" : "");
  }

  // Takes a free instance able to hold n keys (creating or growing one).
  // An instance whose last launch went to the same stream can be taken at
  // once: the stream orders the new launch (and its state load) after the
  // old one.  Otherwise the last launch must have finished.  The per-thread
  // default stream is one handle for many streams, so it never counts as the
  // same stream.
  static GraphInst* acquire(uint64_t n, int pivot, bool half, cudaStream_t st) {
    int dev = 0;
    ck(cudaGetDevice(&dev));
    const bool wide = n >= (1ull << 32);
    const auto key = std::make_tuple(static_cast<int>(sizeof(K)), HV ? 1 : 0, CNT ? 1 : 0, pivot,
                                     (half ? 1 : 0) | (wide ? 2 : 0), dev);
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto& pool = g_graphs[key];
    GraphInst* gi = nullptr;
    const bool ordered = st != cudaStreamPerThread;
    for (GraphInst* c : pool) {  // same stream first
      if (!c->busy && ordered && c->used && c->last == st) {
        gi = c;
        break;
      }
    }
    for (GraphInst* c : pool) {
      if (gi != nullptr) break;
      if (c->busy) continue;
      if (cudaEventQuery(c->done) != cudaSuccess) {
        (void)cudaGetLastError();
        continue;
      }
      gi = c;
    }
    if (gi == nullptr) {
      gi = new GraphInst();
      ck(cudaMalloc(reinterpret_cast<void**>(&gi->d_state), sizeof(DState)));
      ck(cudaMallocHost(reinterpret_cast<void**>(&gi->h_state), sizeof(DState)));
      ck(cudaEventCreateWithFlags(&gi->done, cudaEventDisableTiming));
      gi->wide = wide;
      build(gi, pivot, half);
      pool.push_back(gi);
    }
    if (gi->cap < n) {
      if (gi->used) ck(cudaEventSynchronize(gi->done));  // its last launch still uses ws
      if (gi->ws) ck(cudaFree(gi->ws));
      gi->ws = nullptr;
      const uint64_t cap = std::max<uint64_t>(n, 1ull << 20);
      gi->ws_bytes = graph_ws_bytes(cap);
      if (cudaMalloc(reinterpret_cast<void**>(&gi->ws), gi->ws_bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        gi->cap = 0;
        throw Err{QMS_ENOMEM};
      }
      gi->cap = cap;
    }
    gi->busy = true;
    return gi;
  }

  static void release(GraphInst* gi) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    gi->busy = false;
  }

  // Enqueues the sort of keys[0, n) on st; with stats, waits and fills them.
  static int run(K* keys, uint32_t* vals, uint64_t n, int dtype, int pivot, bool fig3,
                 unsigned spin_limit, int withhold, cudaStream_t st, qms_stats* stats) {
    const auto t0 = std::chrono::steady_clock::now();
    GraphInst* gi = acquire(n, pivot, !fig3, st);
    struct Rel {
      GraphInst* g;
      ~Rel() { release(g); }
    } rel{gi};
    const uint64_t cap = gi->cap;
    unsigned char* w = gi->ws;
    DState h;  // passed by value to the state-load kernel
    std::memset(&h, 0, sizeof(DState));
    h.keys = keys;
    h.vals = vals;
    h.n = n;
    h.xf = xform_of(dtype);
    h.pivot = pivot;
    const WsLayout wl(cap);
    h.desc = reinterpret_cast<Desc*>(w);
    h.counts = reinterpret_cast<uint32_t*>(w + wl.counts);
    h.pml = reinterpret_cast<unsigned long long*>(w + wl.pml);
    h.pmr = reinterpret_cast<unsigned long long*>(w + wl.pmr);
    h.splits = reinterpret_cast<unsigned long long*>(w + wl.splits);
    h.flags = reinterpret_cast<unsigned*>(w + wl.flags);
    h.fig3 = fig3 ? 1 : 0;
    h.spin_limit = spin_limit;
    h.withhold = withhold;
    h.wtl = reinterpret_cast<uint32_t*>(w + wl.wtl);
    h.wtr = reinterpret_cast<uint32_t*>(w + wl.wtr);
    h.b = 0;
    h.e = n;
    for (int i = 0; i < DN_COUNT; ++i) {
      h.dn[i] = gi->dn[i];
      h.cap[i] = gi->gcap[i];
    }
    h.dyn = gi->dyn;
    k_g_load_state<<<1, 1, 0, st>>>(gi->d_state, h);
    ck(cudaMemsetAsync(h.desc, 0, sizeof(Desc), st));
    ck(cudaGraphLaunch(gi->exec, st));
    gi->last = st;
    gi->used = true;
    if (stats) {
      unsigned long long cmp = 0;
      unsigned err = 0;
      ck(cudaMemcpyAsync(&cmp, &h.desc->cmp, sizeof(cmp), cudaMemcpyDeviceToHost, st));
      ck(cudaMemcpyAsync(&err, &h.desc->err, sizeof(err), cudaMemcpyDeviceToHost, st));
      ck(cudaMemcpyAsync(gi->h_state, gi->d_state, sizeof(DState), cudaMemcpyDeviceToHost, st));
      ck(cudaEventRecord(gi->done, st));
      ck(cudaStreamSynchronize(st));
      ck(cudaGetLastError());
      if (err) throw Err{err_code(err)};
      stats->comparisons = cmp;
      stats->aux_bytes = gi->ws_bytes;
      stats->rounds = gi->h_state->rounds;
      stats->mom_rounds = gi->h_state->mom_rounds;
      stats->launches = gi->h_state->launches;
      stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    } else {
      ck(cudaEventRecord(gi->done, st));
      ck(cudaGetLastError());
    }
    return QMS_OK;
  }
};

struct Args {
  void* keys;
  uint32_t* vals;
  uint64_t n;
  int dtype;
  int pivot;
  bool count;
  cudaStream_t st;
  qms_profile* prof;
};

template <class K, bool HV, bool CNT, class Fn>
int run_typed(const Args& a, qms_stats* stats, Fn&& fn) {
  const auto t0 = std::chrono::steady_clock::now();
  Workspace ws;
  ws.alloc(a.n, a.st);
  Profiler prof(a.prof);
  Sorter<K, HV, CNT> s(static_cast<K*>(a.keys), a.vals, xform_of(a.dtype), a.st, ws, prof);
  s.report_ = report_words();
  fn(s);
  unsigned long long cmp = 0;
  unsigned err = 0;
  if (CNT) ck(cudaMemcpyAsync(&cmp, &ws.desc->cmp, sizeof(cmp), cudaMemcpyDeviceToHost, a.st));
  ck(cudaMemcpyAsync(&err, &ws.desc->err, sizeof(err), cudaMemcpyDeviceToHost, a.st));
  ck(cudaStreamSynchronize(a.st));
  ck(cudaGetLastError());
  prof.flush();
  if (err) throw Err{err_code(err)};
  if (a.prof) a.prof->bytes[QMS_K_PART_EXCHANGE] += s.exchanged_bytes;
  if (stats) {
    stats->comparisons = cmp;
    stats->aux_bytes = ws.bytes;
    stats->rounds = s.rounds;
    stats->mom_rounds = s.mom_rounds;
    stats->launches = s.launches;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return QMS_OK;
}

template <class Fn>
int dispatch(const Args& a, qms_stats* stats, Fn&& fn) {
  try {
    const bool u64 = (a.dtype == QMS_U64 || a.dtype == QMS_I64);
    const bool hv = a.vals != nullptr;
    if (u64) {
      if (hv) return a.count ? run_typed<uint64_t, true, true>(a, stats, fn) : run_typed<uint64_t, true, false>(a, stats, fn);
      return a.count ? run_typed<uint64_t, false, true>(a, stats, fn) : run_typed<uint64_t, false, false>(a, stats, fn);
    }
    if (hv) return a.count ? run_typed<uint32_t, true, true>(a, stats, fn) : run_typed<uint32_t, true, false>(a, stats, fn);
    return a.count ? run_typed<uint32_t, false, true>(a, stats, fn) : run_typed<uint32_t, false, false>(a, stats, fn);
  } catch (const Err& e) {
    return e.code;
  } catch (...) {
    return QMS_EINTERNAL;
  }
}

bool valid_dtype(int d) { return d >= QMS_U32 && d <= QMS_F32; }

// Arrays from this size on are sorted host-driven by calls that wait.
constexpr uint64_t kHostDrivenMinN = 1ull << 16;

// Polls of one flag before a bounded device wait gives up.
unsigned spin_limit_of(const qms_options* opt) {
  if (opt == nullptr || opt->spin_limit <= 0) return kOvlSpinLimit;
  return static_cast<unsigned>(opt->spin_limit);
}

// ---------------------------------------------------------------------------
// Batched-form plan: for each length bin (segments of (2^(b-1), 2^b] keys)
// the kernel configuration that sorts it (qms_batch.h).  The default takes
// the smallest thread group whose tile holds the bin; the autotuner
// (qms_batched_autotune) times every configuration per bin on this GPU and
// stores the fastest in a JSON file per key type, payload and SM count,
// which later processes load.

struct BatchPlan {
  int cfg[BATCH_BINS];
  bool tuned;
};

BatchPlan default_plan(int ksize, bool hv) {
  BatchPlan p{};
  for (int b = 0; b < BATCH_BINS; ++b) {
    int best = BC_QMS;
    for (int c = 0; c < BC_COUNT; ++c) {
      if (c == BC_QMS || !batch_cfg_valid(c, ksize, hv) || batch_cfg_capacity(c) < (1 << b)) continue;
      if (best == BC_QMS || batch_cfg_capacity(c) < batch_cfg_capacity(best)) best = c;
    }
    p.cfg[b] = best;
  }
  p.tuned = false;
  return p;
}

void mkdir_one(const char* d) { (void)::mkdir(d, 0755); }

std::string plan_dir() {
  if (const char* d = std::getenv("QMS_AUTOTUNE_DIR")) return d;
  const char* h = std::getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/qms_gb300";
}

std::string plan_path(int ksize, bool hv, int sms) {
  char buf[96];
  std::snprintf(buf, sizeof(buf), "/batched_k%d_v%d_sm%d.json", ksize, hv ? 1 : 0, sms);
  return plan_dir() + buf;
}

int cfg_by_name(const char* name) {
  for (int c = 0; c < BC_COUNT; ++c)
    if (std::strcmp(name, batch_cfg_name(c)) == 0) return c;
  return -1;
}

// Reads a plan file written by write_plan: one bin per line,
//   {"bin": B, "max_len": N, "config": "NAME", "ns_per_key": X}
// Lines that do not parse, or name a configuration that does not exist for
// these keys, leave the default for their bin.  Returns false when the
// file cannot be read or holds another key type or SM count.
bool read_plan(const std::string& path, int ksize, bool hv, int sms, BatchPlan* p) {
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return false;
  char line[512];
  bool header = false;
  while (std::fgets(line, sizeof(line), f)) {
    int k = 0, v = 0, sm = 0;
    if (std::sscanf(line, " {\"key_bytes\": %d, \"payload\": %d, \"sm_count\": %d", &k, &v, &sm) == 3) {
      header = (k == ksize && v == (hv ? 1 : 0) && sm == sms);
      continue;
    }
    int b = -1;
    char name[64] = {0};
    if (std::sscanf(line, " {\"bin\": %d, \"max_len\": %*d, \"config\": \"%63[^\"]\"", &b, name) == 2 &&
        b >= 0 && b < BATCH_BINS) {
      const int c = cfg_by_name(name);
      if (c >= 0 && batch_cfg_valid(c, ksize, hv) && batch_cfg_capacity(c) >= (1 << b)) p->cfg[b] = c;
    }
  }
  std::fclose(f);
  p->tuned = header;
  return header;
}

bool write_plan(const std::string& path, int ksize, bool hv, int sms, const BatchPlan& p,
                const double* ns_per_key) {
  FILE* f = std::fopen(path.c_str(), "w");
  if (!f) return false;
  std::fprintf(f, "{\"key_bytes\": %d, \"payload\": %d, \"sm_count\": %d,\n \"bins\": [\n", ksize,
               hv ? 1 : 0, sms);
  for (int b = 0; b < BATCH_BINS; ++b)
    std::fprintf(f, "  {\"bin\": %d, \"max_len\": %d, \"config\": \"%s\", \"ns_per_key\": %.6f}%s\n", b,
                 1 << b, batch_cfg_name(p.cfg[b]), ns_per_key ? ns_per_key[b] : 0.0,
                 b + 1 < BATCH_BINS ? "," : "");
  std::fprintf(f, " ]}\n");
  return std::fclose(f) == 0;
}

std::mutex g_plan_mu;
std::map<std::tuple<int, int, int>, BatchPlan> g_plans;  // (key bytes, payload, device)

BatchPlan plan_for(int ksize, bool hv) {
  int dev = 0, sms = 0;
  ck(cudaGetDevice(&dev));
  ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  std::lock_guard<std::mutex> lk(g_plan_mu);
  const auto key = std::make_tuple(ksize, hv ? 1 : 0, dev);
  auto it = g_plans.find(key);
  if (it != g_plans.end()) return it->second;
  BatchPlan p = default_plan(ksize, hv);
  BatchPlan q = p;
  if (read_plan(plan_path(ksize, hv, sms), ksize, hv, sms, &q)) p = q;
  g_plans[key] = p;
  return p;
}

void set_plan(int ksize, bool hv, const BatchPlan& p) {
  int dev = 0;
  ck(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_plans[std::make_tuple(ksize, hv ? 1 : 0, dev)] = p;
}

// Streams of the batched form's concurrent bins (per device, created once).
constexpr int kBatchStreams = BC_COUNT;
cudaStream_t batch_stream(int i) {
  static std::mutex mu;
  static std::map<int, std::vector<cudaStream_t>> streams;
  int dev = 0;
  ck(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto& v = streams[dev];
  if (v.empty()) {
    v.resize(kBatchStreams);
    for (auto& x : v) ck(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  }
  return v[i];
}

// ---------------------------------------------------------------------------
// Batched form: many independent segments of one array.  Every segment is
// one QuickMergesort.  The plan maps each length bin to a kernel
// configuration: segments that fit one group's tile are finished by the
// base case inside a warp or block-sized group (several groups per block);
// longer segments of at most CTA_MAX_TILES tiles are sorted by one block
// each running the rounds (longest first, from an atomic ticket); still
// longer ones run through the grid-wide driver.  The configurations' lists
// run concurrently on separate streams.

// Launches the block-per-segment QuickMergesort over order[0, n).
template <class K, bool HV, bool CNT>
void launch_cta_qms(K* keys, uint32_t* vals, const uint64_t* d_off, const uint32_t* d_order,
                    uint32_t n, unsigned int* ticket, int pivot, int xf, Desc* desc, cudaStream_t st) {
  constexpr size_t smem = cta_smem_bytes<K, HV>();
  allow_smem(k_batched<K, HV, CNT>, smem);
  int dev = 0, sms = 0, occ = 0;
  ck(cudaGetDevice(&dev));
  ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched<K, HV, CNT>, NT, smem));
  const unsigned grid = static_cast<unsigned>(
      std::max<uint64_t>(1, std::min<uint64_t>(n, static_cast<uint64_t>(sms) * std::max(occ, 1))));
  k_batched<K, HV, CNT><<<grid, NT, smem, st>>>(keys, vals, d_off, d_order, n, ticket, pivot, xf, desc);
  ck(cudaGetLastError());
}

inline int ceil_log2(uint64_t x) {
  int b = 0;
  while ((1ull << b) < x) ++b;
  return b;
}

template <class K, bool HV, bool CNT>
int run_batched(void* keys, uint32_t* vals, const uint64_t* d_off, size_t nseg, int dtype,
                int pivot, cudaStream_t st, qms_profile* profile, qms_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  constexpr uint64_t ES = sizeof(K) + (HV ? 4 : 0);
  std::vector<uint64_t> off(nseg + 1);
  ck(cudaMemcpyAsync(off.data(), d_off, (nseg + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  for (size_t i = 0; i < nseg; ++i)
    if (off[i + 1] < off[i]) throw Err{QMS_EINVAL};
  if (HV && off[nseg] >= (1ull << 32)) throw Err{QMS_EINVAL};
  const BatchPlan plan = plan_for(sizeof(K), HV);
  const uint64_t cta_max = static_cast<uint64_t>(CTA_MAX_TILES) * TILE;
  // Each configuration's segments, longest first: counting sort by length
  // bin (ceil(log2 length), at most 64), bins in descending order.
  std::vector<uint32_t> cnt_cb(static_cast<size_t>(BC_COUNT) * 65, 0);
  std::vector<uint32_t> big;
  uint64_t big_max = 0, group_keys = 0;
  auto cfg_of = [&](uint64_t len, int b) { return b < BATCH_BINS ? plan.cfg[b] : BC_QMS; };
  for (size_t i = 0; i < nseg; ++i) {
    const uint64_t len = off[i + 1] - off[i];
    if (len <= 1) continue;
    if (len > cta_max) {
      big.push_back(static_cast<uint32_t>(i));
      big_max = std::max(big_max, len);
      continue;
    }
    const int b = ceil_log2(len);
    const int c = cfg_of(len, b);
    ++cnt_cb[static_cast<size_t>(c) * 65 + b];
    if (c != BC_QMS) group_keys += len;
  }
  std::vector<uint32_t> cfg_start(BC_COUNT + 1, 0), pos(static_cast<size_t>(BC_COUNT) * 65, 0);
  uint32_t acc = 0;
  for (int c = 0; c < BC_COUNT; ++c) {
    cfg_start[c] = acc;
    for (int b = 64; b >= 0; --b) {
      pos[static_cast<size_t>(c) * 65 + b] = acc;
      acc += cnt_cb[static_cast<size_t>(c) * 65 + b];
    }
  }
  cfg_start[BC_COUNT] = acc;
  const uint32_t nlisted = acc;
  std::vector<uint32_t> order(nlisted ? nlisted : 1);
  for (size_t i = 0; i < nseg; ++i) {
    const uint64_t len = off[i + 1] - off[i];
    if (len <= 1 || len > cta_max) continue;
    const int b = ceil_log2(len);
    order[pos[static_cast<size_t>(cfg_of(len, b)) * 65 + b]++] = static_cast<uint32_t>(i);
  }
  // Workspace: descriptor, one ticket per configuration and the lists
  // (O(segments) words), plus the grid driver's workspace for the longest
  // large segment.
  const size_t desc_b = 256 * ((sizeof(Desc) + 255) / 256);
  const size_t hdr = desc_b + 256;
  const size_t bbytes = hdr + static_cast<size_t>(nlisted) * 4;
  unsigned char* bws = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&bws), bbytes, st) != cudaSuccess) {
    (void)cudaGetLastError();
    throw Err{QMS_ENOMEM};
  }
  struct Free {
    unsigned char* p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } free_bws{bws, st};
  Desc* desc = reinterpret_cast<Desc*>(bws);
  unsigned int* tickets = reinterpret_cast<unsigned int*>(bws + desc_b);
  uint32_t* d_order = reinterpret_cast<uint32_t*>(bws + hdr);
  ck(cudaMemsetAsync(bws, 0, hdr, st));
  uint64_t launches = 0;
  Profiler prof(profile);
  const int xf = xform_of(dtype);
  if (nlisted) {
    ck(cudaMemcpyAsync(d_order, order.data(), static_cast<size_t>(nlisted) * 4, cudaMemcpyHostToDevice, st));
    prof.begin(st);
    // fork: every non-empty list on its own stream, joined back into st
    cudaEvent_t fork = nullptr;
    ck(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    std::vector<cudaEvent_t> joins;
    struct Ev {
      cudaEvent_t& f;
      std::vector<cudaEvent_t>& j;
      ~Ev() {
        if (f) cudaEventDestroy(f);
        for (auto e : j) cudaEventDestroy(e);
      }
    } ev{fork, joins};
    ck(cudaEventRecord(fork, st));
    for (int c = 0; c < BC_COUNT; ++c) {
      const uint32_t n = cfg_start[c + 1] - cfg_start[c];
      if (n == 0) continue;
      cudaStream_t bs = batch_stream(c);
      ck(cudaStreamWaitEvent(bs, fork, 0));
      const uint32_t* lst = d_order + cfg_start[c];
      if (c == BC_QMS) {
        launch_cta_qms<K, HV, CNT>(static_cast<K*>(keys), vals, d_off, lst, n, tickets + c, pivot, xf,
                                   desc, bs);
      } else {
        ck(launch_group_cfg(c, sizeof(K), HV, CNT, keys, vals, d_off, lst, n, tickets + c, xf, desc, bs));
      }
      ++launches;
      cudaEvent_t j = nullptr;
      ck(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
      joins.push_back(j);
      ck(cudaEventRecord(j, bs));
      ck(cudaStreamWaitEvent(st, j, 0));
    }
    prof.end(st, QMS_K_BATCH, 0);
  }
  uint64_t rounds = 0, mom_rounds = 0, big_cmp = 0;
  if (!big.empty()) {
    Workspace ws;
    ws.alloc(big_max, st);
    for (uint32_t i : big) {
      ck(cudaMemsetAsync(ws.desc, 0, sizeof(Desc), st));
      Sorter<K, HV, CNT> srt(static_cast<K*>(keys) + off[i], HV ? vals + off[i] : nullptr, xf, st, ws,
                             prof);
      srt.report_ = report_words();
      srt.sort(off[i + 1] - off[i], pivot);
      rounds += srt.rounds;
      mom_rounds += srt.mom_rounds;
      launches += srt.launches;
      unsigned long long c = 0;
      if (CNT) {
        ck(cudaMemcpyAsync(&c, &ws.desc->cmp, sizeof(c), cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
      }
      big_cmp += c;
    }
  }
  struct {
    unsigned long long cmp, bytes;
    unsigned err;
  } h{};
  ck(cudaMemcpyAsync(&h.cmp, &desc->cmp, sizeof(h.cmp), cudaMemcpyDeviceToHost, st));
  ck(cudaMemcpyAsync(&h.bytes, &desc->bytes, sizeof(h.bytes), cudaMemcpyDeviceToHost, st));
  ck(cudaMemcpyAsync(&h.err, &desc->err, sizeof(h.err), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  ck(cudaGetLastError());
  prof.flush();
  // group-sorted segments move 2 * ES bytes per key (read once, written once)
  if (profile) profile->bytes[QMS_K_BATCH] += h.bytes + 2 * ES * group_keys;
  if (h.err) throw Err{QMS_EINTERNAL};
  if (stats) {
    stats->comparisons = h.cmp + big_cmp;
    stats->aux_bytes = bbytes + (big.empty() ? 0 : Workspace::size_for(big_max));
    stats->rounds = rounds;
    stats->mom_rounds = mom_rounds;
    stats->launches = launches;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return QMS_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the batched form.  For every length bin it sorts a synthetic
// batch of random keys (segment lengths uniform within the bin, enough
// segments to fill the GPU several times) with every configuration whose
// tile holds the bin, times each with CUDA events (median of three, keys
// refilled before every run), keeps the fastest per key, installs the plan
// for this device and writes it to the plan file.

template <class K>
__global__ void k_fill_random(K* a, uint64_t n, uint64_t seed) {
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;  // SplitMix64 (Steele, Lea, Flood)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    a[i] = static_cast<K>(z ^ (z >> 31));
  }
}

template <class K, bool HV>
int autotune_typed(cudaStream_t st, char* report, size_t report_len) {
  int dev = 0, sms = 0;
  ck(cudaGetDevice(&dev));
  ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  constexpr uint64_t kMaxKeys = 1ull << 24;
  // a bin's draw stops at the first total of at least kMaxKeys keys, so it
  // can pass it by one segment of the last bin, 2^(BATCH_BINS-1) keys
  const uint64_t cap_keys = kMaxKeys + (1ull << (BATCH_BINS - 1));
  const uint64_t max_seg = kMaxKeys / 2 + 2;
  // one allocation: keys, payloads, offsets, order, descriptor and tickets
  const size_t kb = cap_keys * sizeof(K), vb = HV ? cap_keys * 4 : 0;
  const size_t ob = (max_seg + 1) * 8, rb = max_seg * 4, db = 256 * ((sizeof(Desc) + 255) / 256) + 256;
  unsigned char* mem = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(&mem), kb + vb + ob + rb + db) != cudaSuccess) {
    (void)cudaGetLastError();
    throw Err{QMS_ENOMEM};
  }
  struct Free {
    unsigned char* p;
    ~Free() { cudaFree(p); }
  } fr{mem};
  K* keys = reinterpret_cast<K*>(mem);
  uint32_t* vals = HV ? reinterpret_cast<uint32_t*>(mem + kb) : nullptr;
  uint64_t* d_off = reinterpret_cast<uint64_t*>(mem + kb + vb);
  uint32_t* d_order = reinterpret_cast<uint32_t*>(mem + kb + vb + ob);
  Desc* desc = reinterpret_cast<Desc*>(mem + kb + vb + ob + rb);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(reinterpret_cast<unsigned char*>(desc) +
                                                         256 * ((sizeof(Desc) + 255) / 256));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaEventCreate(&e0));
  ck(cudaEventCreate(&e1));
  struct Evs {
    cudaEvent_t a, b;
    ~Evs() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evs{e0, e1};
  BatchPlan plan = default_plan(sizeof(K), HV);
  double ns[BATCH_BINS] = {0};
  std::mt19937_64 rng(0x5eedull);
  std::string rep;
  for (int b = 1; b < BATCH_BINS; ++b) {
    const uint64_t lo = (1ull << (b - 1)) + 1, hi = 1ull << b;
    const uint64_t target = std::min<uint64_t>(kMaxKeys, 1ull << (b + 13));
    std::vector<uint64_t> off(1, 0);
    std::uniform_int_distribution<uint64_t> len(std::max<uint64_t>(lo, 2), hi);
    while (off.back() < target && off.size() < max_seg) off.push_back(off.back() + len(rng));
    const uint32_t nseg = static_cast<uint32_t>(off.size() - 1);
    const uint64_t n = off.back();
    if (n > cap_keys || nseg > max_seg) throw Err{QMS_EINTERNAL};  // the buffers hold them
    std::vector<uint32_t> order(nseg);
    for (uint32_t i = 0; i < nseg; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
      return off[x + 1] - off[x] > off[y + 1] - off[y];
    });
    ck(cudaMemcpyAsync(d_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, st));
    ck(cudaMemcpyAsync(d_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice, st));
    double best = -1.0;
    int best_c = plan.cfg[b];
    for (int c = 0; c < BC_COUNT; ++c) {
      if (!batch_cfg_valid(c, sizeof(K), HV)) continue;
      if (c != BC_QMS && batch_cfg_capacity(c) < static_cast<int>(hi)) continue;
      if (c == BC_QMS && hi <= static_cast<uint64_t>(TILE)) continue;  // a single tile there
      float t[3] = {0, 0, 0};
      for (int r = -1; r < 3; ++r) {  // one warm-up run
        k_fill_random<K><<<1024, 256, 0, st>>>(keys, n, 77 + r);
        ck(cudaMemsetAsync(desc, 0, 256 * ((sizeof(Desc) + 255) / 256) + 256, st));
        ck(cudaEventRecord(e0, st));
        if (c == BC_QMS)
          launch_cta_qms<K, HV, false>(keys, vals, d_off, d_order, nseg, ticket, QMS_PIVOT_M3, XF_NONE,
                                       desc, st);
        else
          ck(launch_group_cfg(c, sizeof(K), HV, false, keys, vals, d_off, d_order, nseg, ticket,
                              XF_NONE, desc, st));
        ck(cudaEventRecord(e1, st));
        ck(cudaEventSynchronize(e1));
        if (r >= 0) ck(cudaEventElapsedTime(&t[r], e0, e1));
      }
      unsigned err = 0;
      ck(cudaMemcpy(&err, &desc->err, sizeof(err), cudaMemcpyDeviceToHost));
      if (err) throw Err{QMS_EINTERNAL};
      std::sort(t, t + 3);
      const double per = static_cast<double>(t[1]) * 1e6 / static_cast<double>(n);
      char line[160];
      std::snprintf(line, sizeof(line), "bin %2d (%llu..%llu keys, %u segments): %-12s %.4f ns/key\n", b,
                    static_cast<unsigned long long>(lo), static_cast<unsigned long long>(hi), nseg,
                    batch_cfg_name(c), per);
      rep += line;
      if (best < 0 || per < best) {
        best = per;
        best_c = c;
      }
    }
    plan.cfg[b] = best_c;
    ns[b] = best;
  }
  plan.tuned = true;
  set_plan(sizeof(K), HV, plan);
  const std::string path = plan_path(sizeof(K), HV, sms);
  std::string dir = plan_dir();
  // create the directory (one level below an existing one is enough here)
  for (size_t p = 1; p <= dir.size(); ++p) {
    if (p == dir.size() || dir[p] == '/') {
      const std::string d = dir.substr(0, p);
      mkdir_one(d.c_str());
    }
  }
  const bool saved = write_plan(path, sizeof(K), HV, sms, plan, ns);
  rep += saved ? ("plan written to " + path + "\n") : ("plan not written (" + path + ")\n");
  if (report && report_len) {
    std::snprintf(report, report_len, "%s", rep.c_str());
  }
  return QMS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of qms_sort (qms_sort_noalloc).
//
// Some callers cannot allocate device memory: an application that gives all
// of the GPU's memory to its own pool allocator and forbids any other
// cudaMalloc, or a latency-critical loop in which an allocation could
// synchronise the device or fail under memory pressure.  For them the round
// descriptor and the per-tile counters of one sort live in a fixed-size
// file-scope device array instead of a workspace allocated per call.

constexpr uint64_t kNoallocMaxN = QMS_NOALLOC_MAX_N;
constexpr size_t kNoallocBytes = WsLayout(kNoallocMaxN).total;

}  // namespace
}  // namespace qms

// Scratch of qms_sort_noalloc (about 900 KB).  Every GPU that loads this
// library holds it until the process exits.  All calls share it.
static __device__ __align__(256) unsigned char qms_noalloc_scratch[qms::kNoallocBytes];

namespace qms {
namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    (void)cudaGetLastError();
    return QMS_ECUDA;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, qms_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return QMS_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  return QMS_OK;
}

template <class K, bool CNT>
int run_noalloc(void* keys, uint64_t n, int dtype, int pivot, const qms_options* opt,
                cudaStream_t st, unsigned char* base, qms_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  Workspace ws;  // base stays null: nothing is allocated and nothing is freed
  ws.st = st;
  ws.bytes = kNoallocBytes;
  ws.place(base, kNoallocMaxN);
  // The array keeps the previous call's contents: the descriptor (counters,
  // flags, selection state) must start from zero.
  ck(cudaMemsetAsync(ws.desc, 0, sizeof(Desc), st));
  Profiler prof(nullptr);
  Sorter<K, false, CNT> s(static_cast<K*>(keys), nullptr, xform_of(dtype), st, ws, prof);
  s.fig3_side = !(opt && (opt->flags & QMS_FLAG_LARGER_SIDE));
  s.spin_limit = spin_limit_of(opt);
  s.withhold = (opt && (opt->flags & QMS_FLAG_TEST_WITHHOLD)) ? 1 : 0;
  s.sort(n, pivot);
  unsigned long long cmp = 0;
  unsigned err = 0;
  if (CNT) ck(cudaMemcpyAsync(&cmp, &ws.desc->cmp, sizeof(cmp), cudaMemcpyDeviceToHost, st));
  ck(cudaMemcpyAsync(&err, &ws.desc->err, sizeof(err), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  ck(cudaGetLastError());
  if (err) return err_code(err);
  if (stats) {
    stats->comparisons = cmp;
    stats->aux_bytes = kNoallocBytes;
    stats->rounds = s.rounds;
    stats->mom_rounds = s.mom_rounds;
    stats->launches = s.launches;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return QMS_OK;
}

}  // namespace
}  // namespace qms

using namespace qms;

extern "C" {

int qms_version(void) { return 10000; }

int qms_release_cached(void) {
  try {
    int dev = 0;
    ck(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto& kv : g_graphs) {
      if (std::get<5>(kv.first) != dev) continue;
      auto& pool = kv.second;
      std::vector<GraphInst*> keep;
      for (GraphInst* gi : pool) {
        if (gi->busy) {  // another thread is setting up a sort with it
          keep.push_back(gi);
          continue;
        }
        if (gi->used) ck(cudaEventSynchronize(gi->done));
        if (gi->exec) ck(cudaGraphExecDestroy(gi->exec));
        if (gi->graph) ck(cudaGraphDestroy(gi->graph));
        if (gi->ws) ck(cudaFree(gi->ws));
        ck(cudaFree(gi->d_state));
        ck(cudaFreeHost(gi->h_state));
        ck(cudaEventDestroy(gi->done));
        delete gi;
      }
      pool.swap(keep);
    }
    return QMS_OK;
  } catch (const Err& e) {
    return e.code;
  }
}

const char* qms_error_string(int code) {
  switch (code) {
    case QMS_OK: return "ok";
    case QMS_EINVAL: return "invalid argument";
    case QMS_ENOMEM: return "out of device memory";
    case QMS_EBUDGET: return "request exceeds the HBM budget";
    case QMS_ECUDA: return "CUDA error";
    case QMS_ETIMEOUT: return "bounded wait timed out";
    case QMS_EAGAIN: return "not finished";
    case QMS_EINTERNAL: return "internal consistency check failed";
    default: return "unknown error";
  }
}

static int sort_common(void* d_keys, uint32_t* d_vals, size_t n, int dtype, const qms_options* opt,
                       void* stream, qms_stats* stats) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (!valid_dtype(dtype)) return QMS_EINVAL;
  const int pivot = opt ? opt->pivot : QMS_PIVOT_M3;
  if (pivot < QMS_PIVOT_M3 || pivot > QMS_PIVOT_HYBRID) return QMS_EINVAL;
  if (n <= 1) return QMS_OK;
  if (d_keys == nullptr) return QMS_EINVAL;
  if (d_vals != nullptr && n >= (1ull << 32)) return QMS_EINVAL;
  Args a{d_keys, d_vals, n, dtype, pivot, opt && opt->count_cmps, static_cast<cudaStream_t>(stream),
         opt ? opt->profile : nullptr};
  // A call that waits for its result runs the rounds from the host: with
  // every kernel launched programmatically after the one before it, one
  // small read-back per round costs less than the graph's conditional nodes
  // (2^20 keys: 1.06 ms against 1.26; 2^24: 2.57 against 3.25; 2^28: 17.3
  // against 18.9).  Asynchronous calls take the graph, which needs no host
  // thread; so do arrays of less than 2^16 keys (at most a few leaves).
  const bool wait = !(opt && (opt->flags & QMS_FLAG_ASYNC)) || stats != nullptr;
  const bool big_sync =
      wait && n >= kHostDrivenMinN && !(opt && (opt->flags & QMS_FLAG_DEVICE_DRIVEN));
  const bool host_driven =
      (opt && (opt->profile || (opt->flags & QMS_FLAG_HOST_DRIVEN))) || big_sync;
  const bool fig3 = !(opt && (opt->flags & QMS_FLAG_LARGER_SIDE));
  const unsigned spin = spin_limit_of(opt);
  const int withhold = (opt && (opt->flags & QMS_FLAG_TEST_WITHHOLD)) ? 1 : 0;
  if (host_driven)
    return dispatch(a, stats, [&](auto& s) {
      s.fig3_side = fig3;
      s.spin_limit = spin;
      s.withhold = withhold;
      s.sort(n, pivot);
    });
  qms_stats local{};
  qms_stats* st = stats ? stats : ((opt && (opt->flags & QMS_FLAG_ASYNC)) ? nullptr : &local);
  try {
    const bool u64 = (dtype == QMS_U64 || dtype == QMS_I64);
    const bool hv = d_vals != nullptr, cnt = a.count;
    const cudaStream_t s = a.st;
#define QMS_G(K, H, C) \
  GraphRunner<K, H, C>::run(static_cast<K*>(d_keys), d_vals, n, dtype, pivot, fig3, spin, withhold, \
                            s, st)
    if (u64) {
      if (hv) return cnt ? QMS_G(uint64_t, true, true) : QMS_G(uint64_t, true, false);
      return cnt ? QMS_G(uint64_t, false, true) : QMS_G(uint64_t, false, false);
    }
    if (hv) return cnt ? QMS_G(uint32_t, true, true) : QMS_G(uint32_t, true, false);
    return cnt ? QMS_G(uint32_t, false, true) : QMS_G(uint32_t, false, false);
#undef QMS_G
  } catch (const Err& e) {
    return e.code;
  } catch (...) {
    return QMS_EINTERNAL;
  }
}

int qms_sort(void* d_keys, size_t n, int dtype, const qms_options* opt, void* stream,
             qms_stats* stats) {
  return sort_common(d_keys, nullptr, n, dtype, opt, stream, stats);
}

int qms_sort_pairs(void* d_keys, uint32_t* d_vals, size_t n, int dtype, const qms_options* opt,
                   void* stream, qms_stats* stats) {
  if (d_vals == nullptr && n > 1) return QMS_EINVAL;
  return sort_common(d_keys, d_vals, n, dtype, opt, stream, stats);
}

int qms_tile_sort(void* d_keys, uint32_t* d_vals, size_t n, int dtype, void* stream) {
  if (!valid_dtype(dtype) || n > static_cast<size_t>(TILE)) return QMS_EINVAL;
  if (n <= 1) return QMS_OK;
  if (d_keys == nullptr) return QMS_EINVAL;
  Args a{d_keys, d_vals, n, dtype, 0, false, static_cast<cudaStream_t>(stream), nullptr};
  return dispatch(a, nullptr, [&](auto& s) { s.leaf(0, n, false, 0); });
}

int qms_partition(void* d_keys, uint32_t* d_vals, size_t n, int dtype, int pivot, void* stream,
                  uint64_t* k_out, uint64_t* eq_out) {
  if (!valid_dtype(dtype) || n < 3 || d_keys == nullptr || k_out == nullptr || eq_out == nullptr)
    return QMS_EINVAL;
  if (pivot < QMS_PIVOT_M3 || pivot > QMS_PIVOT_MOM) return QMS_EINVAL;
  if (d_vals != nullptr && n >= (1ull << 32)) return QMS_EINVAL;
  Args a{d_keys, d_vals, n, dtype, pivot, false, static_cast<cudaStream_t>(stream), nullptr};
  return dispatch(a, nullptr, [&](auto& s) {
    uint64_t k, eq;
    s.split(0, n, pivot, &k, &eq);
    *k_out = k;
    *eq_out = eq;
  });
}

int qms_mergesort(void* d_keys, uint32_t* d_vals, size_t m, size_t buf, int dtype, void* stream) {
  if (!valid_dtype(dtype) || (m > 1 && d_keys == nullptr) || buf < m) return QMS_EINVAL;
  if (m <= 1) return QMS_OK;
  Args a{d_keys, d_vals, buf + m, dtype, 0, false, static_cast<cudaStream_t>(stream), nullptr};
  return dispatch(a, nullptr, [&](auto& s) { s.mergesort(0, m, buf); });
}

int qms_mergesort_half(void* d_keys, uint32_t* d_vals, size_t m, size_t buf, int dtype,
                       void* stream) {
  if (!valid_dtype(dtype) || (m > 1 && d_keys == nullptr) || buf < m) return QMS_EINVAL;
  if (m <= 1) return QMS_OK;
  Args a{d_keys, d_vals, buf + (m - m / 2), dtype, 0, false, static_cast<cudaStream_t>(stream),
         nullptr};
  return dispatch(a, nullptr, [&](auto& s) { s.out_half(0, m, buf); });
}

int qms_sort_noalloc(void* d_keys, size_t n, int dtype, const qms_options* opt, void* stream,
                     qms_stats* stats) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (!valid_dtype(dtype)) return QMS_EINVAL;
  const int pivot = opt ? opt->pivot : QMS_PIVOT_M3;
  if (pivot < QMS_PIVOT_M3 || pivot > QMS_PIVOT_HYBRID) return QMS_EINVAL;
  if (opt && opt->profile) return QMS_EINVAL;
  if (n > kNoallocMaxN) return QMS_EINVAL;
  if (n <= 1) return QMS_OK;
  if (d_keys == nullptr) return QMS_EINVAL;
  unsigned char* base = nullptr;
  const int rc = noalloc_scratch(&base);
  if (rc != QMS_OK) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool cnt = opt && opt->count_cmps;
  try {
    if (dtype == QMS_U64 || dtype == QMS_I64) {
      return cnt ? run_noalloc<uint64_t, true>(d_keys, n, dtype, pivot, opt, st, base, stats)
                 : run_noalloc<uint64_t, false>(d_keys, n, dtype, pivot, opt, st, base, stats);
    }
    return cnt ? run_noalloc<uint32_t, true>(d_keys, n, dtype, pivot, opt, st, base, stats)
               : run_noalloc<uint32_t, false>(d_keys, n, dtype, pivot, opt, st, base, stats);
  } catch (const Err& e) {
    return e.code;
  } catch (...) {
    return QMS_EINTERNAL;
  }
}

static int key_bytes_of(int dtype) { return (dtype == QMS_U64 || dtype == QMS_I64) ? 8 : 4; }

int qms_batched_autotune(int dtype, int with_payload, void* stream, char* report, size_t report_len) {
  if (!valid_dtype(dtype)) return QMS_EINVAL;
  if (report && report_len) report[0] = 0;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  try {
    if (key_bytes_of(dtype) == 8)
      return with_payload ? autotune_typed<uint64_t, true>(st, report, report_len)
                          : autotune_typed<uint64_t, false>(st, report, report_len);
    return with_payload ? autotune_typed<uint32_t, true>(st, report, report_len)
                        : autotune_typed<uint32_t, false>(st, report, report_len);
  } catch (const Err& e) {
    return e.code;
  } catch (...) {
    return QMS_EINTERNAL;
  }
}

int qms_batched_get_plan(int dtype, int with_payload, int* cfg, int nbins, int* tuned) {
  if (!valid_dtype(dtype) || cfg == nullptr || nbins < 1) return QMS_EINVAL;
  try {
    const BatchPlan p = plan_for(key_bytes_of(dtype), with_payload != 0);
    for (int b = 0; b < nbins; ++b) cfg[b] = b < BATCH_BINS ? p.cfg[b] : BC_QMS;
    if (tuned) *tuned = p.tuned ? 1 : 0;
    return QMS_OK;
  } catch (const Err& e) {
    return e.code;
  } catch (...) {
    return QMS_EINTERNAL;
  }
}

int qms_batched_set_plan(int dtype, int with_payload, const int* cfg, int nbins) {
  if (!valid_dtype(dtype) || cfg == nullptr || nbins != BATCH_BINS) return QMS_EINVAL;
  const int ks = key_bytes_of(dtype);
  BatchPlan p{};
  for (int b = 0; b < BATCH_BINS; ++b) {
    const int c = cfg[b];
    if (!batch_cfg_valid(c, ks, with_payload != 0)) return QMS_EINVAL;
    if (c != BC_QMS && batch_cfg_capacity(c) < (1 << b)) return QMS_EINVAL;
    p.cfg[b] = c;
  }
  p.tuned = false;
  try {
    set_plan(ks, with_payload != 0, p);
    return QMS_OK;
  } catch (const Err& e) {
    return e.code;
  } catch (...) {
    return QMS_EINTERNAL;
  }
}

int qms_batched_plan_read(const char* path, int dtype, int with_payload, int sm_count, int* cfg,
                          int nbins) {
  if (path == nullptr || !valid_dtype(dtype) || cfg == nullptr || nbins != BATCH_BINS) return QMS_EINVAL;
  BatchPlan p = default_plan(key_bytes_of(dtype), with_payload != 0);
  const bool ok = read_plan(path, key_bytes_of(dtype), with_payload != 0, sm_count, &p);
  for (int b = 0; b < BATCH_BINS; ++b) cfg[b] = p.cfg[b];
  return ok ? QMS_OK : QMS_EAGAIN;
}

int qms_batched_plan_write(const char* path, int dtype, int with_payload, int sm_count, const int* cfg,
                           const double* ns_per_key, int nbins) {
  if (path == nullptr || !valid_dtype(dtype) || cfg == nullptr || nbins != BATCH_BINS) return QMS_EINVAL;
  BatchPlan p{};
  for (int b = 0; b < BATCH_BINS; ++b) {
    if (!batch_cfg_valid(cfg[b], key_bytes_of(dtype), with_payload != 0)) return QMS_EINVAL;
    p.cfg[b] = cfg[b];
  }
  return write_plan(path, key_bytes_of(dtype), with_payload != 0, sm_count, p, ns_per_key) ? QMS_OK
                                                                                             : QMS_EINVAL;
}

const char* qms_batched_config_name(int cfg) { return batch_cfg_name(cfg); }

int qms_sort_batched(void* d_keys, uint32_t* d_vals, const uint64_t* d_offsets, size_t nseg,
                     int dtype, const qms_options* opt, void* stream, qms_stats* stats) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (!valid_dtype(dtype)) return QMS_EINVAL;
  const int pivot = opt ? opt->pivot : QMS_PIVOT_M3;
  if (pivot < QMS_PIVOT_M3 || pivot > QMS_PIVOT_HYBRID) return QMS_EINVAL;
  if (nseg == 0) return QMS_OK;
  if (d_keys == nullptr || d_offsets == nullptr || nseg >= (1ull << 32)) return QMS_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool cnt = opt && opt->count_cmps;
  qms_profile* prof = opt ? opt->profile : nullptr;
  try {
    const bool u64 = (dtype == QMS_U64 || dtype == QMS_I64);
    const bool hv = d_vals != nullptr;
#define QMS_B(K, H, C) run_batched<K, H, C>(d_keys, d_vals, d_offsets, nseg, dtype, pivot, st, prof, stats)
    if (u64) {
      if (hv) return cnt ? QMS_B(uint64_t, true, true) : QMS_B(uint64_t, true, false);
      return cnt ? QMS_B(uint64_t, false, true) : QMS_B(uint64_t, false, false);
    }
    if (hv) return cnt ? QMS_B(uint32_t, true, true) : QMS_B(uint32_t, true, false);
    return cnt ? QMS_B(uint32_t, false, true) : QMS_B(uint32_t, false, false);
#undef QMS_B
  } catch (const Err& e) {
    return e.code;
  } catch (...) {
    return QMS_EINTERNAL;
  }
}

}  // extern "C"
