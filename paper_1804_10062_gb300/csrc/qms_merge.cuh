// Grid-wide swap-merge level (Fig. 3 "merge" of arXiv 1804.10062, in its
// full-buffer form): runs of length L in region X are merged pairwise into
// region Y while Y's buffer elements move into exactly the X slots each
// output tile consumed.
//
// Small blocks (128 threads, one output tile of 128 x VM elements each) and
// many of them per SM: every thread first issues all of its global loads
// (its share of the tile's A/B slices and of the buffer tile) into
// registers, so a block has a whole tile in flight and eight blocks per SM
// keep enough bytes in flight to stream at HBM speed.  The merge runs in
// shared memory (padded layout, no bank conflicts on the merge-path probes).
#pragma once

#include "qms_device.cuh"

namespace qms {

constexpr int MBT = 128;  // threads per merge block

template <class K, bool HV>
struct MergeCfg {
  static constexpr int VM = sizeof(K) == 4 ? 16 : 8;  // outputs per thread
  static constexpr int MT = MBT * VM;                 // outputs per tile
  static constexpr int IN_K = MT + MT / (128 / static_cast<int>(sizeof(K))) + 4;  // padded
  static constexpr int IN_V = MT + MT / 32 + 4;
  static constexpr int MINB = HV ? 4 : 8;  // resident blocks per SM the kernel is built for
};

template <int MT>
struct MGeom {
  uint64_t pbase, la, lb, d0, d1;
  __device__ __forceinline__ MGeom(uint64_t m, uint64_t L, uint64_t t) {
    const uint64_t o0 = t * MT;
    const uint64_t o1 = (o0 + MT < m) ? o0 + MT : m;
    pbase = o0 & ~(2 * L - 1);  // run lengths are powers of two
    la = (m - pbase < L) ? m - pbase : L;
    const uint64_t rem = m - pbase - la;
    lb = rem < L ? rem : L;
    d0 = o0 - pbase;
    d1 = o1 - pbase;
  }
};

// Merges the tile staged in shared memory (A at logical [0, na), B at
// [na, cnt), encoded keys) and writes the cnt outputs, decoded, to gy/gyv.
// Call after a __syncthreads that made the staged tile visible.  Thread
// produces outputs [d, d + VM).
template <class K, bool HV, bool CNT>
__device__ __forceinline__ void merge_staged_out(const K* sin, K* sout, const uint32_t* svin,
                                                 uint32_t* svout, int na, int cnt, K* gy,
                                                 uint32_t* gyv, int xf, uint64_t& cmp) {
  using C = MergeCfg<K, HV>;
  constexpr int VM = C::VM;
  constexpr int PE = 128 / static_cast<int>(sizeof(K));
  constexpr int SK = MBT + MBT / PE;
  constexpr int SV = MBT + MBT / 32;
  const int tid = threadIdx.x;
  const int nb = cnt - na;
  const int ps = tid + tid / PE;
  const int pv = tid + tid / 32;
  const int d = tid * VM;
  const int pd = d + d / PE;  // padded blocked base
  const int pdv = d + d / 32;
  if (d < cnt) {
    int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (CNT) ++cmp;
      if (!(sin[sk_i<K>(na + d - 1 - mid)] < sin[sk_i<K>(mid)])) lo = mid + 1; else hi = mid;
    }
    int ai = lo, bi = na + d - lo;
    // Once both runs are exhausted (only in the last, partial tile) ai keeps
    // advancing, but never past d + VM <= MT, so every read stays inside
    // sin; such values are discarded by the bound checks.
    K ka = sin[sk_i<K>(ai)];
    K kb = sin[sk_i<K>(bi)];
#pragma unroll
    for (int j = 0; j < VM; ++j) {
      const bool a_ok = ai < na, b_ok = bi < cnt;
      if (CNT && a_ok && b_ok) ++cmp;
      const bool tb = b_ok && (!a_ok || kb < ka);
      if (d + j < cnt) {
        sout[pd + j] = tb ? kb : ka;
        if (HV) svout[pdv + j] = svin[sv_i(tb ? bi : ai)];
      }
      ai += tb ? 0 : 1;
      bi += tb ? 1 : 0;
      const K nk = sin[sk_i<K>(tb ? bi : ai)];
      ka = tb ? ka : nk;
      kb = tb ? nk : kb;
    }
  }
  __syncthreads();
  with_xf<K>(xf, [&](auto xc) {
#pragma unroll
    for (int j = 0; j < VM; ++j) {
      const int i = j * MBT + tid;
      if (i < cnt) {
        gy[i] = dec_key(sout[ps + j * SK], xc);
        if (HV) gyv[i] = svout[pv + j * SV];
      }
    }
  });
}

// One output tile per block.  Element i of the tile (i = j*MBT + thread) is
// loaded from the A/B slices and from the buffer tile by the same thread,
// which then stores its buffer value into that X slot: the tile's consumed
// slots receive exactly its buffer elements.
//
// The buffer tile does not depend on the split step, so it is loaded first;
// with `wait` the block then waits for the split step's grid (launched with
// a programmatic dependency, the merge starts while the split still runs).
//
// Shared-memory indices carry one padding element per 128 bytes.  For the
// striped element i = j*MBT + thread that is j*(MBT + MBT/PE) + pad(thread),
// and for the blocked element d + j (d = thread*VM, a multiple of VM, and
// PE a multiple of 2*VM) it is pad(d) + j: both a per-thread base plus a
// compile-time offset.
template <class K, bool HV, bool CNT>
__device__ __forceinline__ void merge_level_tile(K* keys, uint32_t* vals, uint64_t X, uint64_t Y,
                                                 uint64_t m, uint64_t L, const uint64_t* splits,
                                                 int xf, Desc* desc, uint64_t t, bool wait) {
  using C = MergeCfg<K, HV>;
  constexpr int MT = C::MT;
  constexpr int VM = C::VM;
  constexpr int PE = 128 / static_cast<int>(sizeof(K));  // keys per padded row
  static_assert(PE % (2 * VM) == 0 || VM % PE == 0, "blocked rows must not straddle padding");
  constexpr int SK = MBT + MBT / PE;  // padded stride of one striped row of keys
  constexpr int SV = MBT + MBT / 32;
  __shared__ K sin[C::IN_K];
  __shared__ K sout[C::IN_K];
  __shared__ uint32_t svin[HV ? C::IN_V : 1];
  __shared__ uint32_t svout[HV ? C::IN_V : 1];
  const MGeom<MT> gm(m, L, t);
  K* gy = keys + Y + t * MT;
  uint32_t* gyv = HV ? vals + Y + t * MT : nullptr;
  uint64_t cmp = 0;
  const int tid = threadIdx.x;
  const int cnt = static_cast<int>(gm.d1 - gm.d0);
  K x[VM], y[VM];
  uint32_t xv[VM], yv[VM];
#pragma unroll
  for (int j = 0; j < VM; ++j) {
    const int i = j * MBT + tid;
    if (i < cnt) {
      y[j] = gy[i];
      if (HV) yv[j] = gyv[i];
    }
  }
  if (wait) {
    grid_dep_wait();
    grid_dep_trigger();
  }
  const uint64_t a_lo = splits[t];
  const uint64_t a_hi = (gm.d1 == gm.la + gm.lb) ? gm.la : splits[t + 1];
  const int na = static_cast<int>(a_hi - a_lo);
  const uint64_t b_lo = gm.d0 - a_lo;
  // element i < na comes from A[a_lo + i], element i >= na from B[b_lo + i - na]
  K* ga = keys + X + gm.pbase + a_lo;
  K* gb = keys + X + gm.pbase + gm.la + b_lo - na;
  uint32_t* gav = HV ? vals + X + gm.pbase + a_lo : nullptr;
  uint32_t* gbv = HV ? vals + X + gm.pbase + gm.la + b_lo - na : nullptr;
  const int ps = tid + tid / PE;  // padded striped base
  const int pv = tid + tid / 32;
#pragma unroll
  for (int j = 0; j < VM; ++j) {
    const int i = j * MBT + tid;
    if (i < cnt) {
      x[j] = (i < na ? ga : gb)[i];
      if (HV) xv[j] = (i < na ? gav : gbv)[i];
    }
  }
  with_xf<K>(xf, [&](auto xc) {
#pragma unroll
    for (int j = 0; j < VM; ++j) {
      const int i = j * MBT + tid;
      if (i < cnt) {
        sin[ps + j * SK] = enc_key(x[j], xc);
        (i < na ? ga : gb)[i] = y[j];
        if (HV) {
          svin[pv + j * SV] = xv[j];
          (i < na ? gav : gbv)[i] = yv[j];
        }
      }
    }
  });
  __syncthreads();
  merge_staged_out<K, HV, CNT>(sin, sout, svin, svout, na, cnt, gy, gyv, xf, cmp);
  if (CNT) flush_count(cmp, &desc->cmp);
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(MBT, MergeCfg<K, HV>::MINB)
    k_merge_level3(K* keys, uint32_t* vals, uint64_t X, uint64_t Y, uint64_t m, uint64_t L,
                   const uint64_t* splits, int xf, Desc* desc) {
  merge_level_tile<K, HV, CNT>(keys, vals, X, Y, m, L, splits, xf, desc, blockIdx.x, true);
}

// One lane's merge-path search for diagonal d over A and B (global memory)
// inside [lo, hi]: three probes per step, whose six loads are issued
// together, narrow the window four-fold, so a window of w takes about
// log4(w) dependent round trips (a binary search takes log2(w)).
//
// With delta > 0 a first round tries the window [g - delta, g + delta]
// around a guess g of the answer (its two probes' loads issued together):
// the window shrinks to it when the guess is good, else to one side of it.
template <class K, bool CNT>
__device__ __forceinline__ uint64_t merge_path_lane4(const K* A, const K* B, uint64_t d,
                                                     uint64_t lo, uint64_t hi, int xf,
                                                     uint64_t& cmp, uint64_t g = 0,
                                                     uint64_t delta = 0) {
  // P(m) = !(B[d-1-m] < A[m]) holds below the answer and fails from it on.
  if (delta > 0 && hi > lo && hi - lo > 4 * delta) {
    g = g < lo ? lo : (g >= hi ? hi - 1 : g);
    const uint64_t m1 = g > lo + delta ? g - delta : lo;
    const uint64_t m2 = g + delta < hi ? g + delta : hi - 1;
    const bool p1 = !(enc_key(B[d - 1 - m1], xf) < enc_key(A[m1], xf));
    const bool p2 = !(enc_key(B[d - 1 - m2], xf) < enc_key(A[m2], xf));
    if (CNT) cmp += 2;
    if (!p1) {
      hi = m1;
    } else if (p2) {
      lo = m2 + 1;
    } else {
      lo = m1 + 1;
      hi = m2;
    }
  }
  while (hi - lo >= 4) {
    const uint64_t q = (hi - lo) / 4;
    const uint64_t m1 = lo + q, m2 = m1 + q, m3 = m2 + q;  // all < hi
    const bool p1 = !(enc_key(B[d - 1 - m1], xf) < enc_key(A[m1], xf));
    const bool p2 = !(enc_key(B[d - 1 - m2], xf) < enc_key(A[m2], xf));
    const bool p3 = !(enc_key(B[d - 1 - m3], xf) < enc_key(A[m3], xf));
    if (CNT) cmp += 3;
    if (p3) {
      lo = m3 + 1;
    } else if (p2) {
      lo = m2 + 1;
      hi = m3;
    } else if (p1) {
      lo = m1 + 1;
      hi = m2;
    } else {
      hi = m1;
    }
  }
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (CNT) ++cmp;
    if (!(enc_key(B[d - 1 - mid], xf) < enc_key(A[mid], xf))) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Split step for tiles of MT outputs: for every tile, the number of A
// elements of its run pair preceding its first output.  Runs before any tile
// of the level moves a buffer element.  A warp serves 32 consecutive tiles:
// when they share one run pair it first finds the exact splits at both ends
// of its group (32 probes per round), then every lane binary-searches its
// own tile's split inside the window those two bound (the split moves by at
// most the diagonal's advance); otherwise each lane searches its tile's full
// window.
template <class K, bool HV, bool CNT>
__device__ __forceinline__ void split_group(const K* keys, uint64_t X, uint64_t m, uint64_t L,
                                            int xf, uint64_t* splits, uint64_t w, uint64_t& cmp) {
  using C = MergeCfg<K, HV>;
  constexpr int MT = C::MT;
  const uint64_t ntiles = (m + MT - 1) / MT;
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t t0 = w * 32;
  if (t0 >= ntiles) return;
  const bool grouped = 2 * L >= 32ull * MT;  // pairs hold whole groups
  uint64_t a0 = 0, a1 = 0, d0 = 0, d1 = 0;
  if (grouped) {
    // both ends of the group at once, one per half-warp
    const MGeom<MT> g0(m, L, t0);
    const K* A = keys + X + g0.pbase;
    d0 = g0.d0;
    const uint64_t te = (t0 + 32 < ntiles) ? t0 + 32 : ntiles;
    const uint64_t oe = (te * MT < m) ? te * MT : m;
    d1 = oe - g0.pbase;
    const uint64_t r = merge_path_halfwarp<K, CNT>(A, g0.la, A + g0.la, g0.lb, lane < 16 ? d0 : d1,
                                                   xf, cmp);
    a0 = __shfl_sync(0xffffffffu, r, 0);
    a1 = __shfl_sync(0xffffffffu, r, 16);
  }
  const uint64_t t = t0 + lane;
  if (t < ntiles) {
    const MGeom<MT> g(m, L, t);
    const K* A = keys + X + g.pbase;
    const K* B = A + g.la;
    const uint64_t d = g.d0;
    uint64_t lo = d > g.lb ? d - g.lb : 0, hi = d < g.la ? d : g.la;
    // guess of the answer: the split at the same fraction of the group's
    // advance as at its ends, else the runs' proportion
    uint64_t guess = static_cast<uint64_t>(static_cast<double>(d) * g.la /
                                           static_cast<double>(g.la + g.lb));
    uint64_t delta = 4 * static_cast<uint64_t>(sqrtf(static_cast<float>(d))) + 64;
    if (grouped) {
      const uint64_t lo2 = (a1 > d1 - d) ? a1 - (d1 - d) : 0;
      const uint64_t hi2 = a0 + (d - d0);
      const uint64_t l3 = a0 > lo2 ? a0 : lo2, h3 = a1 < hi2 ? a1 : hi2;
      lo = lo > l3 ? lo : l3;
      hi = hi < h3 ? hi : h3;
      guess = a0 + (a1 - a0) * (d - d0) / (d1 - d0);
      delta = 256;
    }
    splits[t] = merge_path_lane4<K, CNT>(A, B, d, lo, hi, xf, cmp, guess, delta);
  }
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(256) k_merge_split3(const K* keys, uint64_t X, uint64_t m,
                                                      uint64_t L, int xf, uint64_t* splits,
                                                      Desc* desc) {
  grid_dep_wait();     // the runs of the level are complete
  grid_dep_trigger();  // the merge may start and load its buffer tiles
  uint64_t cmp = 0;
  split_group<K, HV, CNT>(keys, X, m, L, xf, splits,
                          (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5, cmp);
  if (CNT) flush_count(cmp, &desc->cmp);
}

// ---------------------------------------------------------------------------
// Overlapped final merge of Fig. 3 "out" (rounds that Mergesort the larger
// side with a buffer of half its size).
//
// A = keys[Ab, Ab + la) (the sorted second half, in the buffer region) and
// B = keys[Ob + la, Ob + la + lb) (the sorted first half, at the tail of the
// target) merge into keys[Ob, Ob + m), m = la + lb.  The la slots
// keys[Ob, Ob + la) hold buffer elements at the start; at the end they are
// in A's slots.  Output tile t covers target positions [t*MT, t*MT + MT).
//
// Slot Ob + p with p >= la holds B[p - la] until that element is consumed,
// and B[j] is output at a position <= la + j.  So a tile's window holds only
// buffer elements and its own B elements once every earlier tile that
// consumed a B element of the window has finished.  Such a tile moves its
// buffer elements into its own consumed A slots and into its consumed B
// slots beyond its window (those lie in later windows, whose tiles wait for
// it).  The counts match exactly: the window holds cnt - (own B elements in
// the window) buffer elements, and the tile frees na A slots plus
// nb - (own B elements in the window) B slots beyond the window.
//
// Tiles are taken in increasing order from a ticket, and a tile waits only
// for earlier tiles, which are already running: the waits cannot deadlock.
// Every wait is bounded; on expiry the tile records the error in the round
// descriptor, which makes all further waits give up, and goes on (the sort
// then reports the error).

// Split step: for every output tile the number of A elements before its
// first output (a warp per 32 tiles, exact anchors at the group's ends, then
// one binary search per lane inside the window they bound).  Also clears the
// tiles' completion flags and the ticket.
template <class K, bool HV, bool CNT>
__device__ __forceinline__ void ovl_split_group(const K* keys, uint64_t Ab, uint64_t la, uint64_t Ob,
                                                uint64_t lb, int xf, uint64_t* splits,
                                                unsigned* flags, uint64_t w, uint64_t& cmp) {
  constexpr int MT = MergeCfg<K, HV>::MT;
  const uint64_t m = la + lb;
  const uint64_t ntiles = (m + MT - 1) / MT;
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t t0 = w * 32;
  if (t0 >= ntiles) return;
  const K* A = keys + Ab;
  const K* B = keys + Ob + la;
  const uint64_t d0 = t0 * MT;
  const uint64_t te = (t0 + 32 < ntiles) ? t0 + 32 : ntiles;
  const uint64_t d1 = (te * MT < m) ? te * MT : m;
  const uint64_t r = merge_path_halfwarp<K, CNT>(A, la, B, lb, lane < 16 ? d0 : d1, xf, cmp);
  const uint64_t a0 = __shfl_sync(0xffffffffu, r, 0);
  const uint64_t a1 = __shfl_sync(0xffffffffu, r, 16);
  const uint64_t t = t0 + lane;
  if (t < ntiles) {
    const uint64_t d = t * MT;
    uint64_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    const uint64_t lo2 = (a1 > d1 - d) ? a1 - (d1 - d) : 0;
    const uint64_t hi2 = a0 + (d - d0);
    lo = lo > a0 ? lo : a0;
    lo = lo > lo2 ? lo : lo2;
    hi = hi < a1 ? hi : a1;
    hi = hi < hi2 ? hi : hi2;
    splits[t] = merge_path_lane4<K, CNT>(A, B, d, lo, hi, xf, cmp);
    flags[t] = 0;
  }
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(256) k_ovl_split(const K* keys, uint64_t Ab, uint64_t la,
                                                   uint64_t Ob, uint64_t lb, int xf,
                                                   uint64_t* splits, unsigned* flags, Desc* desc) {
  uint64_t cmp = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) desc->oticket = 0;
  const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t ngroups = (la + lb + MergeCfg<K, HV>::MT * 32ull - 1) / (MergeCfg<K, HV>::MT * 32ull);
  for (uint64_t w = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; w < ngroups;
       w += nw)
    ovl_split_group<K, HV, CNT>(keys, Ab, la, Ob, lb, xf, splits, flags, w, cmp);
  if (CNT) flush_count(cmp, &desc->cmp);
}

// Wait ranges: tile t of the overlapped merge must wait for the tiles
// [dep_lo[t], dep_hi[t]), the earlier tiles that consumed B elements lying
// in its window.  Window positions p >= la hold B[p - la]; B[j0, j1) are the
// ones consumed before tile t (j < b_lo(t) = t*MT - splits[t]), and the
// tiles holding B[j0] and B[j1 - 1] bound the range (b_lo is nondecreasing
// in the tile).  One thread per tile.
template <int MT>
__device__ __forceinline__ void ovl_deps_tile(uint64_t la, uint64_t lb, const uint64_t* splits,
                                              uint32_t* dep_lo, uint32_t* dep_hi, uint64_t t) {
  const uint64_t m = la + lb;
  const uint64_t o0 = t * MT, o1 = (o0 + MT < m) ? o0 + MT : m;
  const uint64_t b_lo = o0 - splits[t];
  uint32_t lo_t = 0, hi_t = 0;
  if (o1 > la) {
    const uint64_t j0 = (o0 > la ? o0 : la) - la;
    const uint64_t j1 = (o1 - la < b_lo) ? o1 - la : b_lo;
    if (j0 < j1) {
      // last tile u < t with u*MT - splits[u] <= j (tile 0 qualifies)
      auto holder = [&](uint64_t j) {
        uint64_t lo = 0, hi = t;
        while (hi - lo > 1) {
          const uint64_t mid = (lo + hi) >> 1;
          if (mid * MT - splits[mid] <= j) lo = mid; else hi = mid;
        }
        return lo;
      };
      lo_t = static_cast<uint32_t>(holder(j0));
      hi_t = static_cast<uint32_t>(holder(j1 - 1) + 1);
    }
  }
  dep_lo[t] = lo_t;
  dep_hi[t] = hi_t;
}

template <class K, bool HV>
__global__ void __launch_bounds__(256) k_ovl_deps(uint64_t la, uint64_t lb, const uint64_t* splits,
                                                  uint32_t* dep_lo, uint32_t* dep_hi) {
  constexpr int MT = MergeCfg<K, HV>::MT;
  const uint64_t ntiles = (la + lb + MT - 1) / MT;
  for (uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; t < ntiles;
       t += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    ovl_deps_tile<MT>(la, lb, splits, dep_lo, dep_hi, t);
}

constexpr unsigned kOvlSpinLimit = 1u << 20;  // default polls of one flag (about a second)
constexpr unsigned kErrOvlWait = 8u;          // Desc::err bit: a wait ran out

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until flags[u] != 0 for every u in [u0, u1) (the block's threads
// share the flags); false if a wait ran out (more than `limit` polls of one
// flag).  The first wait that runs out sets kErrOvlWait in *err, and every
// wait, current or later, that sees the bit gives up at once: one stuck tile
// costs one wait, not one per tile.
__device__ __forceinline__ bool wait_flags(const unsigned* flags, uint64_t u0, uint64_t u1,
                                           unsigned* err, unsigned limit) {
  bool ok = (ld_acquire_u32(err) & kErrOvlWait) == 0;
  for (uint64_t u = u0 + threadIdx.x; u < u1 && ok; u += blockDim.x) {
    unsigned it = 0;
    while (ld_acquire_u32(flags + u) == 0) {
      if ((++it & 255u) == 0 && (ld_acquire_u32(err) & kErrOvlWait) != 0) {
        ok = false;
        break;
      }
      if (it > limit) {
        atomicOr(err, kErrOvlWait);
        ok = false;
        break;
      }
      __nanosleep(100);
    }
  }
  return __syncthreads_and(ok) != 0;
}

// One output tile of the overlapped merge; returns false if a wait ran out.
//
// Element i of the tile (i = j*MBT + thread) is A[a_lo + i] for i < na and
// B[b_lo + i - na] otherwise.  The first W B elements lie inside the window
// (their slots get outputs); every other element's slot receives one of the
// window's G = cnt - W buffer elements: the g-th, with g = i for i < na and
// g = i - W beyond, where the window's buffer elements are numbered in
// position order around the W own slots.  The thread that loads element i
// also moves that buffer element into its slot, so the tile needs no
// barrier between reading its elements and overwriting their slots.
template <class K, bool HV, bool CNT>
__device__ __forceinline__ bool ovl_merge_tile(K* keys, uint32_t* vals, uint64_t Ab, uint64_t la,
                                               uint64_t Ob, uint64_t lb, const uint64_t* splits,
                                               const uint32_t* dep_lo, const uint32_t* dep_hi,
                                               unsigned* flags, unsigned* err, int xf, uint64_t t,
                                               K* sin, K* sout, uint32_t* svin, uint32_t* svout,
                                               uint64_t& cmp, unsigned limit, bool withhold) {
  using C = MergeCfg<K, HV>;
  constexpr int VM = C::VM, MT = C::MT;
  constexpr int PE = 128 / static_cast<int>(sizeof(K));
  constexpr int SK = MBT + MBT / PE;
  constexpr int SV = MBT + MBT / 32;
  const int tid = threadIdx.x;
  const uint64_t m = la + lb;
  const uint64_t o0 = t * MT, o1 = (o0 + MT < m) ? o0 + MT : m;
  const int cnt = static_cast<int>(o1 - o0);
  const uint64_t a_lo = splits[t], a_hi = (o1 == m) ? la : splits[t + 1];
  const uint64_t b_lo = o0 - a_lo, b_hi = o1 - a_hi;
  const int na = static_cast<int>(a_hi - a_lo);
  const uint64_t Bs = Ob + la;  // B[j] lives at keys[Bs + j] until consumed
  // Own B slots, target-relative: [la + b_lo, la + b_hi); la + b_lo >= o0
  // (an element is output no later than its slot).  Window-relative, the own
  // slots inside the window are [w_lo, w_lo + W).
  const uint64_t own_lo = la + b_lo, own_hi = la + b_hi;
  const int w_lo = static_cast<int>((own_lo < o1 ? own_lo : o1) - o0);
  const int W = static_cast<int>((own_hi < o1 ? own_hi : o1) - o0) - w_lo;
  // 1. Wait for the earlier tiles that consumed B elements of the window.
  bool ok = true;
  {
    const uint64_t u0 = dep_lo[t], u1 = dep_hi[t];
    if (u0 < u1) ok = wait_flags(flags, u0, u1, err, limit);
  }
  // 2. Load the tile's elements and the buffer elements bound for their
  //    slots together.
  K* ga = keys + Ab + a_lo;
  K* gb = keys + Bs + b_lo - na;
  uint32_t* gav = HV ? vals + Ab + a_lo : nullptr;
  uint32_t* gbv = HV ? vals + Bs + b_lo - na : nullptr;
  const K* win = keys + Ob + o0;
  const uint32_t* winv = HV ? vals + Ob + o0 : nullptr;
  const int ps = tid + tid / PE;
  const int pv = tid + tid / 32;
  K x[VM], gk[VM];
  uint32_t xv[VM], gv[VM];
#pragma unroll
  for (int j = 0; j < VM; ++j) {
    const int i = j * MBT + tid;
    if (i < cnt) {
      x[j] = (i < na ? ga : gb)[i];
      if (HV) xv[j] = (i < na ? gav : gbv)[i];
      if (i < na || i >= na + W) {
        const int g = i < na ? i : i - W;
        const int src = g < w_lo ? g : g + W;
        gk[j] = __ldcg(win + src);
        if (HV) gv[j] = __ldcg(winv + src);
      }
    }
  }
  with_xf<K>(xf, [&](auto xc) {
#pragma unroll
    for (int j = 0; j < VM; ++j) {
      const int i = j * MBT + tid;
      if (i < cnt) {
        sin[ps + j * SK] = enc_key(x[j], xc);
        if (HV) svin[pv + j * SV] = xv[j];
        if (i < na || i >= na + W) {
          (i < na ? ga : gb)[i] = gk[j];
          if (HV) (i < na ? gav : gbv)[i] = gv[j];
        }
      }
    }
  });
  __syncthreads();
  // 3. Merge and write the window (its buffer elements are all read).
  merge_staged_out<K, HV, CNT>(sin, sout, svin, svout, na, cnt, keys + Ob + o0,
                               HV ? vals + Ob + o0 : nullptr, xf, cmp);
  // 4. Publish.  A tile that moved buffer elements into later windows makes
  //    them visible before its flag; any other tile has nothing a later tile
  //    reads and only sets the flag.  (withhold: a test hook that never
  //    publishes tile 0, so that the waits on it run out.)
  if (withhold && t == 0) {
    // nothing is published
  } else if (static_cast<uint64_t>(W) < b_hi - b_lo) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release_u32(flags + t, 1u);
    }
  } else if (tid == 0) {
    st_release_u32(flags + t, 1u);
  }
  return ok;
}

template <class K, bool HV, bool CNT>
__device__ __forceinline__ void ovl_merge_loop(K* keys, uint32_t* vals, uint64_t Ab, uint64_t la,
                                               uint64_t Ob, uint64_t lb, const uint64_t* splits,
                                               const uint32_t* dep_lo, const uint32_t* dep_hi,
                                               unsigned* flags, int xf, Desc* desc, unsigned limit,
                                               int withhold) {
  using C = MergeCfg<K, HV>;
  __shared__ K sin[C::IN_K];
  __shared__ K sout[C::IN_K];
  __shared__ uint32_t svin[HV ? C::IN_V : 1];
  __shared__ uint32_t svout[HV ? C::IN_V : 1];
  __shared__ unsigned long long ticket;
  const uint64_t ntiles = (la + lb + C::MT - 1) / C::MT;
  uint64_t cmp = 0;
  bool ok = true;
  // Tickets are taken one tile ahead: the atomic's latency overlaps the
  // current tile.  A block finishes every tile it took, and waits still
  // point only to smaller tiles, so this keeps the waits deadlock-free.
  // With a grid of at least ntiles blocks each block takes one ticket.
  const bool one = gridDim.x >= ntiles;
  if (threadIdx.x == 0) ticket = atomicAdd(&desc->oticket, 1ull);
  __syncthreads();
  uint64_t t = ticket;
  while (t < ntiles) {
    __syncthreads();  // every thread has read the ticket
    if (!one && threadIdx.x == 0) ticket = atomicAdd(&desc->oticket, 1ull);
    ok = ovl_merge_tile<K, HV, CNT>(keys, vals, Ab, la, Ob, lb, splits, dep_lo, dep_hi, flags,
                                    &desc->err, xf, t, sin, sout, svin, svout, cmp, limit,
                                    withhold != 0) && ok;
    if (one) break;
    __syncthreads();
    t = ticket;
  }
  if (!ok && threadIdx.x == 0) atomicOr(&desc->err, kErrOvlWait);
  if (CNT) flush_count(cmp, &desc->cmp);
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(MBT, MergeCfg<K, HV>::MINB)
    k_ovl_merge(K* keys, uint32_t* vals, uint64_t Ab, uint64_t la, uint64_t Ob, uint64_t lb,
                const uint64_t* splits, const uint32_t* dep_lo, const uint32_t* dep_hi,
                unsigned* flags, int xf, Desc* desc, unsigned limit, int withhold) {
  ovl_merge_loop<K, HV, CNT>(keys, vals, Ab, la, Ob, lb, splits, dep_lo, dep_hi, flags, xf, desc,
                             limit, withhold);
}

}  // namespace qms
