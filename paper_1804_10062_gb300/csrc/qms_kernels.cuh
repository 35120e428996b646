// Global kernels of the GB300 QuickMergesort path.  Each kernel is one step
// of a QuickMergesort round (arXiv 1804.10062, Sec. 2 and the Fig. 3
// listing): pivot selection, in-place partition (local partition, scan,
// exchange, pivot placement), Mergesort leaves (base case X) and swap-merge
// levels.  Round state that the device computes (pivot, left count, ...)
// lives in a small device descriptor so that kernels can be queued without
// the host knowing it.
#pragma once

#include "qms_device.cuh"

namespace qms {

// Device-side round descriptor (one per sort call; O(1) words).
struct Desc {
  unsigned long long cmp;         // comparisons (counting build only)
  unsigned long long L;           // left elements of the last partition pass
  unsigned long long mis;         // misplaced pairs of the last partition pass
  unsigned long long pivot;       // order key of the pivot
  unsigned long long sel_prefix;  // radix select state (MoM)
  unsigned long long sel_mask;
  unsigned long long sel_rank;
  unsigned long long sel_eq;
  unsigned long long pos;
  unsigned long long bytes;       // algorithmic bytes reported by the batched form
  unsigned long long oticket;     // next tile of the overlapped merge
  unsigned int mdone;             // blocks of the current merge level that finished
  unsigned int tie;  // pivot sample saw a tie: run the second (<=) pass
  unsigned int err;  // nonzero: an internal consistency check failed
  unsigned int hist[256];
  unsigned long long csum[2 * 1024];  // per-chunk misplaced sums of the partition scan
};

// Side choice of a round on [b, e) whose pivot block is [k, k + 1 + eq).
//   SIDE_LARGER_*: Mergesort the larger side with a buffer of half its size
//     taken from the front of the other side (Sec. 2 allows either side when
//     the other one can hold the buffer; Fig. 1 takes the larger one), used
//     when that side is longer than one tile and the buffer fits.
//   SIDE_LEFT / SIDE_RIGHT: Fig. 3's rule, a full-size buffer: the left side
//     iff the pivot lies left of the integer midpoint; after a three-way
//     split, the smaller side.
enum : int { SIDE_LEFT = 0, SIDE_RIGHT = 1, SIDE_LARGER_LEFT = 2, SIDE_LARGER_RIGHT = 3 };
__host__ __device__ inline int choose_side(uint64_t b, uint64_t e, uint64_t k, uint64_t eq,
                                           bool fig3) {
  const uint64_t nn = e - b, rb = k + 1 + eq, nl = k - b, nr = e - rb;
  if (!fig3) {
    const uint64_t big = nl > nr ? nl : nr, small = nl > nr ? nr : nl;
    if (big > static_cast<uint64_t>(TILE) && big - big / 2 <= small)
      return nl >= nr ? SIDE_LARGER_LEFT : SIDE_LARGER_RIGHT;
  }
  const bool left = (eq == 0) ? (k < b + nn / 2) : (nl <= nr);
  return left ? SIDE_LEFT : SIDE_RIGHT;
}

// The partition scan works on chunks of scan_chunk(ntiles) tiles, at most
// 1024 chunks.
__host__ __device__ inline uint64_t scan_chunk(uint64_t ntiles) {
  const uint64_t c = (ntiles + 1023) / 1024;
  return c < 2048 ? 2048 : c;
}

// ---------------------------------------------------------------------------
// Base case / Mergesort leaves: sort tiles of P[0, m); with to_buf the
// sorted tiles go to the buffer region and the buffer's contents move into P.

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(LeafCfg<K, HV>::LT, LeafCfg<K, HV>::MINB) k_leaf_sort(K* keys, uint32_t* vals, uint64_t P,
                                                                  uint64_t m, uint64_t Bb, int to_buf,
                                                                  int xf, Desc* desc) {
  grid_dep_wait();
  grid_dep_trigger();
  constexpr int LT = LeafCfg<K, HV>::LT, TL = LeafCfg<K, HV>::TILE_L, VL = LeafCfg<K, HV>::VL;
  extern __shared__ __align__(16) unsigned char smem[];
  const auto s = TileSmem<K, HV, LT, VL>::carve(smem);
  uint64_t cmp = 0;
  const uint64_t ntiles = (m + TL - 1) / TL;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t off = t * TL;
    const int cnt = static_cast<int>((m - off) < static_cast<uint64_t>(TL) ? (m - off) : TL);
    K* g = keys + P + off;
    uint32_t* gv = HV ? vals + P + off : nullptr;
    K* b = to_buf ? keys + Bb + off : nullptr;
    uint32_t* bv = (HV && to_buf) ? vals + Bb + off : nullptr;
    leaf_sort_tile<K, HV, CNT, LT, VL>(s, g, gv, b, bv, cnt, xf, cmp);
  }
  if (CNT) flush_count(cmp, &desc->cmp);
}

// ---------------------------------------------------------------------------
// Pivot selection.  Each pivot kernel parks the chosen pivot element at
// position e - 1 and records its order key and whether the sample held a
// tie (duplicate guard: a tie selects the second, "<=", partition pass).

// Median-of-3 at b, b + floor(n/2), e - 1 (proof of Thm. 1).
template <class K, bool HV, bool CNT>
__global__ void k_pivot_m3(K* keys, uint32_t* vals, uint64_t b, uint64_t e, int xf, Desc* desc) {
  grid_dep_wait();
  grid_dep_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint64_t n = e - b;
  uint64_t p0 = b, p1 = b + n / 2, p2 = e - 1;
  K u0 = enc_key(keys[p0], xf), u1 = enc_key(keys[p1], xf), u2 = enc_key(keys[p2], xf);
  // sort3 on (key, position) pairs
  if (u1 < u0) { K t = u0; u0 = u1; u1 = t; uint64_t q = p0; p0 = p1; p1 = q; }
  unsigned c = 2;
  if (u2 < u1) {
    K t = u1; u1 = u2; u2 = t; uint64_t q = p1; p1 = p2; p2 = q;
    ++c;
    if (u1 < u0) { t = u0; u0 = u1; u1 = t; q = p0; p0 = p1; p1 = q; }
  }
  const bool tie = !(u0 < u1) || !(u1 < u2);
  const uint64_t pm = p1, last = e - 1;
  if (pm != last) {
    const K a = keys[pm]; keys[pm] = keys[last]; keys[last] = a;
    if (HV) { const uint32_t x = vals[pm]; vals[pm] = vals[last]; vals[last] = x; }
  }
  desc->pivot = static_cast<unsigned long long>(u1);
  desc->tie = tie ? 1u : 0u;
  desc->L = 0;  // the round's partition counts from zero
  if (CNT) desc->cmp += c + 2;
}

// The median-of-sqrt(n) sample is sorted by one block of SAMPLE_T threads
// with V keys each, so it may hold SAMPLE_MAX = SAMPLE_T * V - 1 keys: about
// sqrt(n) up to n = 2^28.
constexpr int SAMPLE_T = 2 * NT;
constexpr int SAMPLE_MAX = SAMPLE_T * V - 1;

// Median of a sample of ks (odd, <= SAMPLE_MAX) elements at b + i*step
// (median-of-sqrt(n), Sec. 2 / Thm. 2).  One block sorts the sample with the
// base-case sort, carrying the sample index as payload.
template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(SAMPLE_T) k_pivot_sample(K* keys, uint32_t* vals, uint64_t b, uint64_t e,
                                                           int ks, uint64_t step, int xf, Desc* desc) {
  grid_dep_wait();
  grid_dep_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  const auto s = TileSmem<K, true, SAMPLE_T, V>::carve(smem);
  uint64_t cmp = 0;
  for (int i = threadIdx.x; i < SAMPLE_T * V; i += SAMPLE_T) {
    s.k[sk_i<K>(i)] = (i < ks) ? enc_key(keys[b + static_cast<uint64_t>(i) * step], xf) : key_max<K>();
    s.v[sv_i(i)] = static_cast<uint32_t>(i);
  }
  block_sort_tile<K, true, CNT, SAMPLE_T, V>(s, cmp);
  if (CNT) flush_count(cmp, &desc->cmp);
  if (threadIdx.x == 0) {
    const int h = ks / 2;
    const K med = s.k[sk_i<K>(h)];
    const uint64_t pm = b + static_cast<uint64_t>(s.v[sv_i(h)]) * step, last = e - 1;
    bool tie = false;
    if (ks >= 3) tie = !(s.k[sk_i<K>(h - 1)] < med) || !(med < s.k[sk_i<K>(h + 1)]);
    if (pm != last) {
      const K a = keys[pm]; keys[pm] = keys[last]; keys[last] = a;
      if (HV) { const uint32_t x = vals[pm]; vals[pm] = vals[last]; vals[last] = x; }
    }
    desc->pivot = static_cast<unsigned long long>(med);
    desc->tie = tie ? 1u : 0u;
    desc->L = 0;
    if (CNT) desc->cmp += 2;
  }
}

// MoM step 1 (Sec. 4): the median of each triple (3i, 3i+1, 3i+2), i < t,
// is moved to the middle slot 3i+1 of its triple.
template <class K, bool HV, bool CNT>
__global__ void k_mom_triples(K* keys, uint32_t* vals, uint64_t b, uint64_t t, int xf, Desc* desc) {
  uint64_t cmp = 0;
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < t;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint64_t q = b + 3 * i;
    const K x0 = keys[q], x1 = keys[q + 1], x2 = keys[q + 2];
    const K u0 = enc_key(x0, xf), u1 = enc_key(x1, xf), u2 = enc_key(x2, xf);
    int mi;
    if (u1 < u0) {                     // u1 < u0
      mi = (u2 < u1) ? 1 : ((u2 < u0) ? 2 : 0);
    } else {                           // u0 <= u1
      mi = (u2 < u1) ? ((u2 < u0) ? 0 : 2) : 1;
    }
    if (CNT) cmp += 3;
    if (mi != 1) {
      const uint64_t p = q + mi;
      keys[q + 1] = (mi == 0) ? x0 : x2;
      keys[p] = x1;
      if (HV) { const uint32_t a = vals[p]; vals[p] = vals[q + 1]; vals[q + 1] = a; }
    }
  }
  if (CNT) flush_count(cmp, &desc->cmp);
}

// MoM step 2: exact radix selection of the median of the medians (8 bits a
// pass, most significant first).
template <class K>
__global__ void k_sel_hist(const K* keys, uint64_t b, uint64_t t, int xf, int shift, Desc* desc) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const K pre = static_cast<K>(desc->sel_prefix), msk = static_cast<K>(desc->sel_mask);
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < t;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const K u = enc_key(keys[b + 3 * i + 1], xf);
    if (((u ^ pre) & msk) == 0) atomicAdd(&h[static_cast<unsigned>(u >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&desc->hist[i], h[i]);
}

static __global__ void k_sel_pick(int shift, Desc* desc) {
  if (threadIdx.x != 0) return;
  unsigned long long r = desc->sel_rank, acc = 0;
  int bin = 255;
  for (int i = 0; i < 256; ++i) {
    const unsigned long long c = desc->hist[i];
    if (r < acc + c) { bin = i; break; }
    acc += c;
  }
  desc->sel_eq = desc->hist[bin];
  desc->sel_prefix |= static_cast<unsigned long long>(bin) << shift;
  desc->sel_mask |= 255ull << shift;
  desc->sel_rank = r - acc;
  for (int i = 0; i < 256; ++i) desc->hist[i] = 0;
}

// MoM step 3: locate a median equal to the selected value and park it.
template <class K>
__global__ void k_mom_locate(const K* keys, uint64_t b, uint64_t t, int xf, Desc* desc) {
  const K v = static_cast<K>(desc->sel_prefix);
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < t;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    if (enc_key(keys[b + 3 * i + 1], xf) == v) atomicMin(&desc->pos, static_cast<unsigned long long>(i));
  }
}

template <class K, bool HV>
__global__ void k_mom_place(K* keys, uint32_t* vals, uint64_t b, uint64_t e, uint64_t t, Desc* desc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (desc->pos >= t) {  // no median carried the selected key: report, touch nothing
    desc->err |= 2u;
    return;
  }
  const uint64_t pm = b + 3 * desc->pos + 1, last = e - 1;
  if (pm != last) {
    const K a = keys[pm]; keys[pm] = keys[last]; keys[last] = a;
    if (HV) { const uint32_t x = vals[pm]; vals[pm] = vals[last]; vals[last] = x; }
  }
  desc->pivot = desc->sel_prefix;
  desc->tie = desc->sel_eq > 1 ? 1u : 0u;
  desc->L = 0;
}

// ---------------------------------------------------------------------------
// In-place partition of [lo, hi) around desc->pivot (Sec. 2; every element is
// compared with the pivot once).

// Step 1: local partition of every partition tile (PT keys, PNT threads),
// left count per tile.
template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(PNT, (part_minb<K, HV>())) k_part_local(K* keys, uint32_t* vals, uint64_t lo, uint64_t hi,
                                                    int le, int xf, Desc* desc, uint32_t* counts) {
  grid_dep_wait();
  grid_dep_trigger();
  __shared__ K sk[pk_len<K>()];
  __shared__ uint32_t sv[HV ? pv_len() : 1];
  __shared__ uint32_t scr[PNWARP + 1];
  uint64_t cmp = 0;
  const K piv = static_cast<K>(desc->pivot);
  const uint64_t n = hi - lo, ntiles = (n + PT - 1) / PT;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t off = t * PT;
    const int cnt = static_cast<int>((n - off) < static_cast<uint64_t>(PT) ? (n - off) : PT);
    __syncthreads();
    K* const g = keys + lo + off;
    uint32_t* const gv = HV ? vals + lo + off : nullptr;
    const uint32_t c =
        cnt == PT ? part_local_small<K, HV, CNT, true>(g, gv, cnt, piv, le != 0, xf, sk, sv, scr, cmp)
                  : part_local_small<K, HV, CNT>(g, gv, cnt, piv, le != 0, xf, sk, sv, scr, cmp);
    if (threadIdx.x == 0) {
      counts[t] = c;
      atomicAdd(&desc->L, static_cast<unsigned long long>(c));
    }
  }
  if (CNT) flush_count(cmp, &desc->cmp);
}

// Block-wide exclusive scan of 64-bit values (scratch: NWARP + 1 u64).
__device__ __forceinline__ uint64_t block_excl_scan_u64(uint64_t x, uint64_t* scratch,
                                                        uint64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) scratch[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint64_t s = lane < NWARP ? scratch[lane] : 0ull;
    uint64_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    if (lane < NWARP) scratch[lane] = si - s;
    if (lane == 31) scratch[NWARP] = si;
  }
  __syncthreads();
  const uint64_t r = scratch[w] + inc - x;
  *total = scratch[NWARP];
  __syncthreads();
  return r;
}

// Step 2: with L (the number of left keys, summed by step 1) known, the
// misplaced run lengths of every tile and their exclusive prefix sums pml /
// pmr (ntiles + 1 entries).  Two parallel passes over chunks of tiles: the
// sums of each chunk, then each chunk's prefixes.

__device__ __forceinline__ void tile_mis(uint64_t lo, uint64_t hi, uint64_t sb, uint32_t t, uint32_t c,
                                         uint64_t* ml, uint64_t* mr) {
  const uint64_t ts = lo + static_cast<uint64_t>(t) * PT;
  const uint64_t te = (ts + PT < hi) ? ts + PT : hi;
  const uint64_t cs = ts + c;
  const uint64_t lend = te < sb ? te : sb;
  const uint64_t rbeg = ts > sb ? ts : sb;
  *ml = lend > cs ? lend - cs : 0;
  *mr = cs > rbeg ? cs - rbeg : 0;
}

__device__ __forceinline__ void scan_chunks_body(uint64_t lo, uint64_t hi, const uint32_t* counts,
                                                 Desc* desc) {
  __shared__ uint64_t scr[NWARP + 1];
  const uint32_t ntiles = static_cast<uint32_t>((hi - lo + PT - 1) / PT);
  const uint64_t ch = scan_chunk(ntiles);
  const uint64_t sb = lo + desc->L;
  const uint64_t t0 = blockIdx.x * ch;
  const uint64_t t1 = (t0 + ch < ntiles) ? t0 + ch : ntiles;
  uint64_t sl = 0, sr = 0;
  for (uint64_t t = t0 + threadIdx.x; t < t1; t += NT) {
    uint64_t ml, mr;
    tile_mis(lo, hi, sb, static_cast<uint32_t>(t), counts[t], &ml, &mr);
    sl += ml;
    sr += mr;
  }
  uint64_t tl, tr;
  (void)block_excl_scan_u64(sl, scr, &tl);
  (void)block_excl_scan_u64(sr, scr, &tr);
  if (threadIdx.x == 0) {
    desc->csum[2 * blockIdx.x] = tl;
    desc->csum[2 * blockIdx.x + 1] = tr;
  }
}

__device__ __forceinline__ void scan_prefix_body(uint64_t lo, uint64_t hi, const uint32_t* counts,
                                                 uint64_t* pml, uint64_t* pmr, uint32_t* wtl,
                                                 uint32_t* wtr, Desc* desc) {
  __shared__ uint64_t scr[NWARP + 1];
  const uint32_t ntiles = static_cast<uint32_t>((hi - lo + PT - 1) / PT);
  const uint64_t ch = scan_chunk(ntiles);
  const uint32_t nchunks = static_cast<uint32_t>((ntiles + ch - 1) / ch);
  const uint64_t sb = lo + desc->L;
  // prefix of the chunk sums before this chunk (and the totals)
  uint64_t bl = 0, br = 0, al = 0, ar = 0;
  for (uint32_t c = threadIdx.x; c < nchunks; c += NT) {
    const uint64_t l = desc->csum[2 * c], r = desc->csum[2 * c + 1];
    if (c < blockIdx.x) {
      bl += l;
      br += r;
    }
    al += l;
    ar += r;
  }
  uint64_t base_l, base_r, tot_l, tot_r;
  (void)block_excl_scan_u64(bl, scr, &base_l);
  (void)block_excl_scan_u64(br, scr, &base_r);
  (void)block_excl_scan_u64(al, scr, &tot_l);
  (void)block_excl_scan_u64(ar, scr, &tot_r);
  // this chunk: each thread a contiguous run of tiles
  const uint64_t t0 = blockIdx.x * ch;
  const uint64_t t1 = (t0 + ch < ntiles) ? t0 + ch : ntiles;
  const uint64_t per = (t1 - t0 + NT - 1) / NT;
  const uint64_t u0 = t0 + threadIdx.x * per;
  const uint64_t u1 = (u0 + per < t1) ? u0 + per : t1;
  uint64_t sl = 0, sr = 0;
  for (uint64_t t = u0; t < u1; ++t) {
    uint64_t ml, mr;
    tile_mis(lo, hi, sb, static_cast<uint32_t>(t), counts[t], &ml, &mr);
    sl += ml;
    sr += mr;
  }
  uint64_t dummy;
  uint64_t pl = base_l + block_excl_scan_u64(sl, scr, &dummy);
  uint64_t pr = base_r + block_excl_scan_u64(sr, scr, &dummy);
  for (uint64_t t = u0; t < u1; ++t) {
    pml[t] = pl;
    pmr[t] = pr;
    uint64_t ml, mr;
    tile_mis(lo, hi, sb, static_cast<uint32_t>(t), counts[t], &ml, &mr);
    // exchange warps whose first left / right rank falls in this tile
    for (uint64_t w = (pl + EXJ - 1) / EXJ; w * EXJ < pl + ml; ++w) wtl[w] = static_cast<uint32_t>(t);
    for (uint64_t w = (pr + EXJ - 1) / EXJ; w * EXJ < pr + mr; ++w) wtr[w] = static_cast<uint32_t>(t);
    pl += ml;
    pr += mr;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    pml[ntiles] = tot_l;
    pmr[ntiles] = tot_r;
    desc->mis = tot_l;
    if (tot_l != tot_r) desc->err |= 1u;
  }
}

static __global__ void __launch_bounds__(NT) k_part_chunks(uint64_t lo, uint64_t hi,
                                                           const uint32_t* counts, Desc* desc) {
  grid_dep_wait();
  grid_dep_trigger();
  scan_chunks_body(lo, hi, counts, desc);
}

static __global__ void __launch_bounds__(NT) k_part_prefix(uint64_t lo, uint64_t hi,
                                                           const uint32_t* counts, uint64_t* pml,
                                                           uint64_t* pmr, uint32_t* wtl,
                                                           uint32_t* wtr, Desc* desc) {
  grid_dep_wait();
  grid_dep_trigger();
  scan_prefix_body(lo, hi, counts, pml, pmr, wtl, wtr, desc);
}

// Step 3: exchange the misplaced elements by rank (one warp per chunk of
// EXJ ranks).
// P: uint32_t positions for ranges shorter than 2^32 keys, else uint64_t.
// For 4-byte keys without payloads the kernel is built for five blocks per
// SM (95 registers, no spills; 126 registers and four blocks before).
template <class K, bool HV, class P>
__global__ void __launch_bounds__(EXB, (sizeof(K) == 4 && !HV) ? 5 : 1) k_part_exchange(K* keys, uint32_t* vals, uint64_t lo,
                                                       const uint32_t* counts, const uint64_t* pml,
                                                       const uint64_t* pmr, const uint32_t* wtl,
                                                       const uint32_t* wtr, const Desc* desc) {
  grid_dep_wait();
  grid_dep_trigger();
  const uint64_t mis = desc->mis;
  const uint64_t s = lo + desc->L;
  const uint64_t w0 = (blockIdx.x * static_cast<uint64_t>(EXB) + threadIdx.x) >> 5;
  const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * EXB) >> 5;
  for (uint64_t jw = w0 * EXJ; jw < mis; jw += nw * EXJ)
    exchange_warp<K, HV, P>(keys, vals, lo, s, counts, pml, pmr, wtl, wtr, jw, mis);
}

// Step 4: the pivot parked at position `parked` moves to its final index
// lo + L.
template <class K, bool HV>
__global__ void k_place_pivot(K* keys, uint32_t* vals, uint64_t lo, uint64_t parked, Desc* desc) {
  grid_dep_wait();
  grid_dep_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint64_t k = lo + desc->L;
  if (k != parked) {
    const K a = keys[k]; keys[k] = keys[parked]; keys[parked] = a;
    if (HV) { const uint32_t x = vals[k]; vals[k] = vals[parked]; vals[parked] = x; }
  }
}

}  // namespace qms
