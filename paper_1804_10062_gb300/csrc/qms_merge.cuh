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

// One output tile per block.  Element i of the tile (i = j*MBT + thread) is
// loaded from the A/B slices and from the buffer tile by the same thread,
// which then stores its buffer value into that X slot: the tile's consumed
// slots receive exactly its buffer elements.
//
// Shared-memory indices carry one padding element per 128 bytes.  For the
// striped element i = j*MBT + thread that is j*(MBT + MBT/PE) + pad(thread),
// and for the blocked element d + j (d = thread*VM, a multiple of VM, and
// PE a multiple of 2*VM) it is pad(d) + j: both a per-thread base plus a
// compile-time offset.
template <class K, bool HV, bool CNT>
__device__ __forceinline__ void merge_level_tile_impl(K* keys, uint32_t* vals,
                                                      const MGeom<MergeCfg<K, HV>::MT>& gm,
                                                      uint64_t a_lo, uint64_t a_hi, K* gy,
                                                      uint32_t* gyv, uint64_t X, int xf, Desc* desc,
                                                      K* sin, K* sout, uint32_t* svin,
                                                      uint32_t* svout) {
  using C = MergeCfg<K, HV>;
  constexpr int VM = C::VM, MT = C::MT;
  constexpr int PE = 128 / static_cast<int>(sizeof(K));  // keys per padded row
  static_assert(PE % (2 * VM) == 0 || VM % PE == 0, "blocked rows must not straddle padding");
  constexpr int SK = MBT + MBT / PE;  // padded stride of one striped row of keys
  constexpr int SV = MBT + MBT / 32;
  uint64_t cmp = 0;
  const int tid = threadIdx.x;
  const int cnt = static_cast<int>(gm.d1 - gm.d0);
  const int na = static_cast<int>(a_hi - a_lo), nb = cnt - na;
  const uint64_t b_lo = gm.d0 - a_lo;
  // element i < na comes from A[a_lo + i], element i >= na from B[b_lo + i - na]
  K* ga = keys + X + gm.pbase + a_lo;
  K* gb = keys + X + gm.pbase + gm.la + b_lo - na;
  uint32_t* gav = HV ? vals + X + gm.pbase + a_lo : nullptr;
  uint32_t* gbv = HV ? vals + X + gm.pbase + gm.la + b_lo - na : nullptr;
  const int ps = tid + tid / PE;  // padded striped base
  const int pv = tid + tid / 32;
  K x[VM], y[VM];
  uint32_t xv[VM], yv[VM];
#pragma unroll
  for (int j = 0; j < VM; ++j) {
    const int i = j * MBT + tid;
    if (i < cnt) {
      K* src = (i < na ? ga : gb) + i;
      x[j] = *src;
      y[j] = gy[i];
      if (HV) {
        xv[j] = (i < na ? gav : gbv)[i];
        yv[j] = gyv[i];
      }
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
  // Staged layout: A at logical [0, na), B at [na, cnt).  Thread produces
  // outputs [d, d + VM).
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
  if (CNT) flush_count(cmp, &desc->cmp);
}

template <class K, bool HV, bool CNT>
__device__ __forceinline__ void merge_level_tile(K* keys, uint32_t* vals, uint64_t X, uint64_t Y,
                                                 uint64_t m, uint64_t L, const uint64_t* splits,
                                                 int xf, Desc* desc, uint64_t t) {
  using C = MergeCfg<K, HV>;
  constexpr int MT = C::MT;
  const MGeom<MT> gm(m, L, t);
  const uint64_t a_lo = splits[t];
  const uint64_t a_hi = (gm.d1 == gm.la + gm.lb) ? gm.la : splits[t + 1];
  K* gy = keys + Y + t * MT;
  uint32_t* gyv = HV ? vals + Y + t * MT : nullptr;
  __shared__ K sin[C::IN_K];
  __shared__ K sout[C::IN_K];
  __shared__ uint32_t svin[HV ? C::IN_V : 1];
  __shared__ uint32_t svout[HV ? C::IN_V : 1];
  merge_level_tile_impl<K, HV, CNT>(keys, vals, gm, a_lo, a_hi, gy, gyv, X, xf, desc, sin, sout,
                                    svin, svout);
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(MBT, MergeCfg<K, HV>::MINB)
    k_merge_level3(K* keys, uint32_t* vals, uint64_t X, uint64_t Y, uint64_t m, uint64_t L,
                   const uint64_t* splits, int xf, Desc* desc) {
  merge_level_tile<K, HV, CNT>(keys, vals, X, Y, m, L, splits, xf, desc, blockIdx.x);
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
    const MGeom<MT> g0(m, L, t0);
    const K* A = keys + X + g0.pbase;
    d0 = g0.d0;
    a0 = (d0 == 0) ? 0 : merge_path_warp<K, CNT>(A, g0.la, A + g0.la, g0.lb, d0, xf, cmp);
    const uint64_t te = (t0 + 32 < ntiles) ? t0 + 32 : ntiles;
    const uint64_t oe = (te * MT < m) ? te * MT : m;
    d1 = oe - g0.pbase;
    a1 = (d1 >= g0.la + g0.lb) ? g0.la : merge_path_warp<K, CNT>(A, g0.la, A + g0.la, g0.lb, d1, xf, cmp);
  }
  const uint64_t t = t0 + lane;
  if (t < ntiles) {
    const MGeom<MT> g(m, L, t);
    const K* A = keys + X + g.pbase;
    const K* B = A + g.la;
    const uint64_t d = g.d0;
    uint64_t lo = d > g.lb ? d - g.lb : 0, hi = d < g.la ? d : g.la;
    if (grouped) {
      const uint64_t lo2 = (a1 > d1 - d) ? a1 - (d1 - d) : 0;
      const uint64_t hi2 = a0 + (d - d0);
      const uint64_t l3 = a0 > lo2 ? a0 : lo2, h3 = a1 < hi2 ? a1 : hi2;
      lo = lo > l3 ? lo : l3;
      hi = hi < h3 ? hi : h3;
    }
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (CNT) ++cmp;
      if (!(enc_key(B[d - 1 - mid], xf) < enc_key(A[mid], xf))) lo = mid + 1; else hi = mid;
    }
    splits[t] = lo;
  }
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(256) k_merge_split3(const K* keys, uint64_t X, uint64_t m,
                                                      uint64_t L, int xf, uint64_t* splits,
                                                      Desc* desc) {
  uint64_t cmp = 0;
  split_group<K, HV, CNT>(keys, X, m, L, xf, splits,
                          (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5, cmp);
  if (CNT) flush_count(cmp, &desc->cmp);
}

}  // namespace qms
