// CTA-scoped QuickMergesort: one thread block sorts one segment of up to
// CTA_MAX_TILES tiles entirely by itself (the batched form).  The steps are
// those of the grid path (arXiv 1804.10062, Sec. 2 and Fig. 3: pivot,
// in-place partition, Mergesort of one side with the other side as swap
// buffer, continue on the other side), built from the same tile routines of
// qms_device.cuh; the per-tile counters that the grid path keeps in global
// memory live in shared memory here, and phases are separated by
// __syncthreads instead of kernel boundaries.  Segments are small enough to
// stay in L2 while their block works on them.
#pragma once

#include "qms_kernels.cuh"

namespace qms {

constexpr int CTA_MAX_TILES = 64;  // segments up to 64 * 8192 keys
#ifndef QMS_CTA_MINB
#define QMS_CTA_MINB 2  // blocks per SM the block-per-segment kernel is built for
#endif

// Out-of-line copies of the tile routines for the block-scoped path: the
// whole QuickMergesort of a segment lives in one kernel, and separate
// register allocation per routine keeps it from spilling.
template <class K, bool HV, bool CNT>
__device__ __noinline__ uint32_t part_local_tile_call(TileSmem<K, HV> s, K* g, uint32_t* gv, int cnt,
                                                      K piv, bool le, int xf, uint64_t& cmp) {
  return part_local_tile<K, HV, CNT>(s, g, gv, cnt, piv, le, xf, cmp);
}
// Leaves of the block-scoped path: 512 threads of CtaLeaf::VL keys, so
// 4-byte keys without payloads sort 16384-key leaves (one merge level and
// about one round fewer per segment than 8192-key leaves); the tile shares
// the block's shared memory with the 8192-key partition and merge tiles.
template <class K, bool HV>
struct CtaLeaf {
  static constexpr int VL = (sizeof(K) == 4 && !HV) ? 2 * V : V;
  static constexpr int TL = NT * VL;
};
template <class K, bool HV>
__host__ __device__ constexpr size_t cta_smem_bytes() {
  return tile_smem_bytes<K, HV, NT, CtaLeaf<K, HV>::VL>() > tile_smem_bytes<K, HV>()
             ? tile_smem_bytes<K, HV, NT, CtaLeaf<K, HV>::VL>()
             : tile_smem_bytes<K, HV>();
}

template <class K, bool HV, bool CNT>
__device__ __noinline__ void leaf_sort_tile_call(unsigned char* smem, K* g, uint32_t* gv, K* buf,
                                                 uint32_t* bufv, int cnt, int xf, uint64_t& cmp) {
  constexpr int VL = CtaLeaf<K, HV>::VL;
  leaf_sort_tile<K, HV, CNT, NT, VL>(TileSmem<K, HV, NT, VL>::carve(smem), g, gv, buf, bufv, cnt, xf, cmp);
}
template <class K, bool HV, bool CNT>
__device__ __noinline__ void merge_tile_call(TileSmem<K, HV> s, K* keys, uint32_t* vals, uint64_t X,
                                             uint64_t Y, uint64_t m, uint64_t L, uint64_t tile,
                                             const uint64_t* splits, int xf, uint64_t& cmp) {
  merge_tile<K, HV, CNT>(s, keys, vals, X, Y, m, L, tile, splits, xf, cmp);
}

struct CtaState {
  uint32_t counts[CTA_MAX_TILES];
  uint64_t pml[CTA_MAX_TILES + 1];
  uint64_t pmr[CTA_MAX_TILES + 1];
  uint64_t splits[CTA_MAX_TILES + 1];
  uint64_t L, mis, piv, pos, sel_prefix, sel_mask, sel_rank, sel_eq;
  uint64_t bytes;  // algorithmic bytes moved (thread 0 accumulates)
  uint32_t hist[256];
  uint32_t tie, err, seg;
};

// In-place partition of [lo, hi) around piv (le: "<=" pass).  Returns L.
template <class K, bool HV, bool CNT>
__device__ __noinline__ uint64_t cta_partition(TileSmem<K, HV> s, CtaState& cs, K* keys, uint32_t* vals,
                                  uint64_t lo, uint64_t hi, K piv, bool le, int xf, uint64_t& cmp) {
  const uint64_t n = hi - lo;
  const uint32_t nt = static_cast<uint32_t>((n + TILE - 1) / TILE);
  for (uint32_t t = 0; t < nt; ++t) {
    const uint64_t off = static_cast<uint64_t>(t) * TILE;
    const int cnt = static_cast<int>((n - off) < static_cast<uint64_t>(TILE) ? (n - off) : TILE);
    const uint32_t c = part_local_tile_call<K, HV, CNT>(s, keys + lo + off, HV ? vals + lo + off : nullptr,
                                                   cnt, piv, le, xf, cmp);
    if (threadIdx.x == 0) cs.counts[t] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t L = 0;
    for (uint32_t t = 0; t < nt; ++t) L += cs.counts[t];
    const uint64_t sb = lo + L;
    cs.pml[0] = 0;
    cs.pmr[0] = 0;
    for (uint32_t t = 0; t < nt; ++t) {
      const uint64_t ts = lo + static_cast<uint64_t>(t) * TILE;
      const uint64_t te = (ts + TILE < hi) ? ts + TILE : hi;
      const uint64_t c = ts + cs.counts[t];
      const uint64_t lend = te < sb ? te : sb;
      const uint64_t rbeg = ts > sb ? ts : sb;
      cs.pml[t + 1] = cs.pml[t] + (lend > c ? lend - c : 0);
      cs.pmr[t + 1] = cs.pmr[t] + (c > rbeg ? c - rbeg : 0);
    }
    cs.L = L;
    cs.mis = cs.pml[nt];
    if (cs.pml[nt] != cs.pmr[nt]) cs.err |= 1u;
    cs.bytes += 2 * n * (sizeof(K) + (HV ? 4 : 0)) + 4 * cs.mis * (sizeof(K) + (HV ? 4 : 0));
  }
  __syncthreads();
  const uint64_t L = cs.L, mis = cs.err ? 0 : cs.mis;
  for (uint64_t j0 = static_cast<uint64_t>(threadIdx.x) * EXV; j0 < mis;
       j0 += static_cast<uint64_t>(NT) * EXV) {
    exchange_ranks<K, HV>(keys, vals, lo, lo + L, cs.counts, cs.pml, cs.pmr, nt, j0, mis);
  }
  __syncthreads();
  return L;
}

// Mergesort of P[0, m) with the disjoint buffer Bb[0, m) (full-buffer form).
template <class K, bool HV, bool CNT>
__device__ __noinline__ void cta_mergesort(TileSmem<K, HV> s, unsigned char* smem, CtaState& cs, K* keys,
                                           uint32_t* vals, uint64_t P, uint64_t m, uint64_t Bb, int xf,
                                           uint64_t& cmp) {
  constexpr uint64_t ES = sizeof(K) + (HV ? 4 : 0);
  constexpr uint64_t TL = CtaLeaf<K, HV>::TL;
  if (m <= 1) return;
  if (m <= TL) {
    leaf_sort_tile_call<K, HV, CNT>(smem, keys + P, HV ? vals + P : nullptr, nullptr, nullptr,
                               static_cast<int>(m), xf, cmp);
    if (threadIdx.x == 0) cs.bytes += 2 * m * ES;
    __syncthreads();
    return;
  }
  const uint32_t leaves = static_cast<uint32_t>((m + TL - 1) / TL);
  int levels = 0;
  while ((1u << levels) < leaves) ++levels;
  const bool to_buf = (levels & 1) != 0;
  for (uint32_t t = 0; t < leaves; ++t) {
    const uint64_t off = static_cast<uint64_t>(t) * TL;
    const int cnt = static_cast<int>((m - off) < TL ? (m - off) : TL);
    leaf_sort_tile_call<K, HV, CNT>(smem, keys + P + off, HV ? vals + P + off : nullptr,
                               to_buf ? keys + Bb + off : nullptr,
                               (HV && to_buf) ? vals + Bb + off : nullptr, cnt, xf, cmp);
  }
  uint64_t X = to_buf ? Bb : P, Y = to_buf ? P : Bb;
  const uint32_t mtiles = static_cast<uint32_t>((m + TILE - 1) / TILE);  // merge tiles of 8192 outputs
  for (int l = 0; l < levels; ++l) {
    const uint64_t L = TL << l;
    __syncthreads();
    for (uint32_t t = threadIdx.x >> 5; t < mtiles; t += NWARP)
      merge_split_warp<K, CNT>(keys, X, m, L, t, xf, cs.splits, cmp);
    __syncthreads();
    for (uint32_t t = 0; t < mtiles; ++t)
      merge_tile_call<K, HV, CNT>(s, keys, vals, X, Y, m, L, t, cs.splits, xf, cmp);
    const uint64_t x = X;
    X = Y;
    Y = x;
  }
  if (threadIdx.x == 0) cs.bytes += (to_buf ? 4 : 2) * m * ES + 4 * m * ES * levels;
  __syncthreads();
}

template <class K, bool HV>
__device__ __forceinline__ void swap_elems(K* keys, uint32_t* vals, uint64_t a, uint64_t b) {
  if (a == b) return;
  const K x = keys[a];
  keys[a] = keys[b];
  keys[b] = x;
  if (HV) {
    const uint32_t y = vals[a];
    vals[a] = vals[b];
    vals[b] = y;
  }
}

// Median-of-3 pivot (thread 0): parks the pivot at e - 1.
template <class K, bool HV, bool CNT>
__device__ __noinline__ void cta_pivot_m3(CtaState& cs, K* keys, uint32_t* vals, uint64_t b, uint64_t e, int xf,
                             uint64_t& cmp) {
  if (threadIdx.x == 0) {
    const uint64_t n = e - b;
    uint64_t p0 = b, p1 = b + n / 2, p2 = e - 1;
    K u0 = enc_key(keys[p0], xf), u1 = enc_key(keys[p1], xf), u2 = enc_key(keys[p2], xf);
    if (u1 < u0) { K t = u0; u0 = u1; u1 = t; uint64_t q = p0; p0 = p1; p1 = q; }
    if (u2 < u1) {
      K t = u1; u1 = u2; u2 = t; uint64_t q = p1; p1 = p2; p2 = q;
      if (u1 < u0) { t = u0; u0 = u1; u1 = t; q = p0; p0 = p1; p1 = q; }
    }
    if (CNT) cmp += 5;
    cs.tie = (!(u0 < u1) || !(u1 < u2)) ? 1u : 0u;
    cs.piv = static_cast<uint64_t>(u1);
    swap_elems<K, HV>(keys, vals, p1, e - 1);
  }
  __syncthreads();
}

// Median-of-sqrt(n) pivot: the block sorts a sample of k (largest odd <=
// ceil(sqrt n), at most TILE - 1) keys at b + i*floor(n/k), takes its median
// and parks a sample element with that key at e - 1.
template <class K, bool HV, bool CNT>
__device__ __noinline__ void cta_pivot_sqrtn(TileSmem<K, HV> s, CtaState& cs, K* keys, uint32_t* vals, uint64_t b,
                                uint64_t e, int xf, uint64_t& cmp) {
  const uint64_t n = e - b;
  uint64_t c = 1;
  while (c * c < n) ++c;
  uint64_t k = (c & 1) ? c : c - 1;
  if (k > static_cast<uint64_t>(TILE - 1)) k = TILE - 1;
  const uint64_t step = n / k;
  const int ks = static_cast<int>(k);
  const int P = threads_for(ks);
  __syncthreads();
  for (int i = threadIdx.x; i < P * V; i += NT) {
    s.k[sk_i<K>(i)] = (i < ks) ? enc_key(keys[b + static_cast<uint64_t>(i) * step], xf) : key_max<K>();
    if (HV) s.v[sv_i(i)] = 0;
  }
  block_sort_tile<K, HV, CNT>(s, cmp, P);
  if (threadIdx.x == 0) {
    const int h = ks / 2;
    const K med = s.k[sk_i<K>(h)];
    cs.tie = (ks >= 3 && (!(s.k[sk_i<K>(h - 1)] < med) || !(med < s.k[sk_i<K>(h + 1)]))) ? 1u : 0u;
    cs.piv = static_cast<uint64_t>(med);
    cs.pos = ~0ull;
  }
  __syncthreads();
  const K med = static_cast<K>(cs.piv);
  for (int i = threadIdx.x; i < ks; i += NT) {
    if (enc_key(keys[b + static_cast<uint64_t>(i) * step], xf) == med)
      atomicMin(reinterpret_cast<unsigned long long*>(&cs.pos), static_cast<unsigned long long>(i));
  }
  __syncthreads();
  if (threadIdx.x == 0) swap_elems<K, HV>(keys, vals, b + cs.pos * step, e - 1);
  __syncthreads();
}

// MoM pivot (Sec. 4): medians of the floor(n/3) triples moved to the middle
// slot of each triple, exact median of those medians by radix selection in
// shared memory, then parked at e - 1.
template <class K, bool HV, bool CNT>
__device__ __noinline__ void cta_pivot_mom(CtaState& cs, K* keys, uint32_t* vals, uint64_t b, uint64_t e, int xf,
                              uint64_t& cmp) {
  const uint64_t t = (e - b) / 3;
  for (uint64_t i = threadIdx.x; i < t; i += NT) {
    const uint64_t q = b + 3 * i;
    const K x0 = keys[q], x1 = keys[q + 1], x2 = keys[q + 2];
    const K u0 = enc_key(x0, xf), u1 = enc_key(x1, xf), u2 = enc_key(x2, xf);
    int mi;
    if (u1 < u0) {
      mi = (u2 < u1) ? 1 : ((u2 < u0) ? 2 : 0);
    } else {
      mi = (u2 < u1) ? ((u2 < u0) ? 0 : 2) : 1;
    }
    if (CNT) cmp += 3;
    if (mi != 1) swap_elems<K, HV>(keys, vals, q + 1, q + mi);
  }
  if (threadIdx.x == 0) {
    cs.sel_prefix = 0;
    cs.sel_mask = 0;
    cs.sel_rank = t / 2;
    cs.pos = ~0ull;
  }
  __syncthreads();
  for (int shift = static_cast<int>(sizeof(K) * 8) - 8; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += NT) cs.hist[i] = 0;
    __syncthreads();
    const K pre = static_cast<K>(cs.sel_prefix), msk = static_cast<K>(cs.sel_mask);
    for (uint64_t i = threadIdx.x; i < t; i += NT) {
      const K u = enc_key(keys[b + 3 * i + 1], xf);
      if (((u ^ pre) & msk) == 0) atomicAdd(&cs.hist[static_cast<unsigned>(u >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t r = cs.sel_rank, acc = 0;
      int bin = 255;
      for (int i = 0; i < 256; ++i) {
        if (r < acc + cs.hist[i]) { bin = i; break; }
        acc += cs.hist[i];
      }
      cs.sel_eq = cs.hist[bin];
      cs.sel_prefix |= static_cast<uint64_t>(bin) << shift;
      cs.sel_mask |= 255ull << shift;
      cs.sel_rank = r - acc;
    }
    __syncthreads();
  }
  const K v = static_cast<K>(cs.sel_prefix);
  for (uint64_t i = threadIdx.x; i < t; i += NT) {
    if (enc_key(keys[b + 3 * i + 1], xf) == v)
      atomicMin(reinterpret_cast<unsigned long long*>(&cs.pos), static_cast<unsigned long long>(i));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (cs.pos < t) {
      swap_elems<K, HV>(keys, vals, b + 3 * cs.pos + 1, e - 1);
      cs.piv = cs.sel_prefix;
      cs.tie = cs.sel_eq > 1 ? 1u : 0u;
    } else {
      cs.err |= 2u;
    }
  }
  __syncthreads();
}

// QuickMergesort of keys[b, e) by one block (pivot: QMS_PIVOT_* code).
template <class K, bool HV, bool CNT>
__device__ void cta_qms(TileSmem<K, HV> s, unsigned char* smem, CtaState& cs, K* keys, uint32_t* vals,
                        uint64_t b, uint64_t e, int pivot, int xf, uint64_t& cmp) {
  bool mom_next = false;
  while (e - b > static_cast<uint64_t>(CtaLeaf<K, HV>::TL)) {
    if (cs.err) return;
    const uint64_t nn = e - b;
    const bool mom = pivot == 2 || (pivot == 3 && mom_next);
    if (mom) {
      cta_pivot_mom<K, HV, CNT>(cs, keys, vals, b, e, xf, cmp);
    } else if (pivot == 1) {
      cta_pivot_sqrtn<K, HV, CNT>(s, cs, keys, vals, b, e, xf, cmp);
    } else {
      cta_pivot_m3<K, HV, CNT>(cs, keys, vals, b, e, xf, cmp);
    }
    if (cs.err) return;
    const K piv = static_cast<K>(cs.piv);
    const bool tie = cs.tie != 0;
    const uint64_t L = cta_partition<K, HV, CNT>(s, cs, keys, vals, b, e - 1, piv, false, xf, cmp);
    const uint64_t k = b + L;
    if (threadIdx.x == 0) swap_elems<K, HV>(keys, vals, k, e - 1);
    __syncthreads();
    uint64_t eq = 0;
    if (tie && k + 1 < e) eq = cta_partition<K, HV, CNT>(s, cs, keys, vals, k + 1, e, piv, true, xf, cmp);
    if (pivot == 3) {
      const uint64_t d = nn / 16, rlo = k - b, rhi = k + eq - b;
      mom_next = !mom && (rhi < d || rlo > nn - 1 - d);
    }
    const uint64_t rb = k + 1 + eq;
    const uint64_t nl = k - b, nr = e - rb;
    const bool left = (eq == 0) ? (k < b + nn / 2) : (nl <= nr);
    if (left) {
      cta_mergesort<K, HV, CNT>(s, smem, cs, keys, vals, b, nl, rb, xf, cmp);
      b = rb;
    } else {
      cta_mergesort<K, HV, CNT>(s, smem, cs, keys, vals, rb, nr, b, xf, cmp);
      e = k;
    }
  }
  if (e - b > 1) {
    leaf_sort_tile_call<K, HV, CNT>(smem, keys + b, HV ? vals + b : nullptr, nullptr, nullptr,
                               static_cast<int>(e - b), xf, cmp);
    if (threadIdx.x == 0) cs.bytes += 2 * (e - b) * (sizeof(K) + (HV ? 4 : 0));
  }
  __syncthreads();
}

// Batched form: a persistent grid; each block repeatedly takes the next
// segment (in the host's longest-first order) from an atomic ticket and sorts
// it alone.
template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(NT, QMS_CTA_MINB) k_batched(K* keys, uint32_t* vals, const uint64_t* offsets,
                                                const uint32_t* order, uint32_t nseg,
                                                unsigned int* ticket, int pivot, int xf,
                                                Desc* desc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaState cs;
  const auto s = TileSmem<K, HV>::carve(smem);
  uint64_t cmp = 0;
  if (threadIdx.x == 0) {
    cs.err = 0;
    cs.bytes = 0;
  }
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) cs.seg = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t t = cs.seg;
    if (t >= nseg || cs.err) break;
    const uint32_t sg = order[t];
    cta_qms<K, HV, CNT>(s, smem, cs, keys, vals, offsets[sg], offsets[sg + 1], pivot, xf, cmp);
  }
  if (CNT) flush_count(cmp, &desc->cmp);
  if (threadIdx.x == 0) {
    if (cs.err) atomicOr(&desc->err, cs.err);
    atomicAdd(&desc->bytes, static_cast<unsigned long long>(cs.bytes));
  }
}

// Served form: the segments are separate arrays (one per request), listed by
// pointer, length and key transform.
struct SegDesc {
  void* keys;
  unsigned long long n;
  int xf;
  int pad;
};

template <class K, bool CNT>
__global__ void __launch_bounds__(NT, QMS_CTA_MINB) k_batched_ptrs(const SegDesc* segs, uint32_t nseg,
                                                     unsigned int* ticket, int pivot, Desc* desc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaState cs;
  const auto s = TileSmem<K, false>::carve(smem);
  uint64_t cmp = 0;
  if (threadIdx.x == 0) {
    cs.err = 0;
    cs.bytes = 0;
  }
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) cs.seg = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t t = cs.seg;
    if (t >= nseg || cs.err) break;
    const SegDesc sd = segs[t];
    cta_qms<K, false, CNT>(s, smem, cs, static_cast<K*>(sd.keys), nullptr, 0, sd.n, pivot, sd.xf, cmp);
  }
  if (CNT) flush_count(cmp, &desc->cmp);
  if (threadIdx.x == 0) {
    if (cs.err) atomicOr(&desc->err, cs.err);
    atomicAdd(&desc->bytes, static_cast<unsigned long long>(cs.bytes));
  }
}

}  // namespace qms
