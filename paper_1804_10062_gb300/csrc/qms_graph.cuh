// Device-driven QuickMergesort: the whole round loop of Fig. 3 (arXiv
// 1804.10062, "sort") runs inside one CUDA graph with conditional nodes, so
// the host never waits between rounds.
//
//   WHILE (range longer than one tile):
//     begin   - pivot rule of the round; median-of-3 done here
//     [sample / median-of-medians pivot kernels, present for those rules]
//     partition pass 1 (local, scan, exchange) around the pivot
//     mid     - place the pivot; IF a sample tie: partition pass 2 ("<=")
//     side    - Fig. 3 side choice, Mergesort part and buffer, level count
//     leaves  - base case X on the part (in place or swapped into the buffer)
//     WHILE (levels left): split, swap-merge (its last block ends the level)
//     end     - continue on the other side
//   final leaf sort of the last range.
//
// All round state lives in DState (device memory); work kernels run a fixed
// grid and stride over the counts they read from it, control kernels are a
// single thread and set the conditions with cudaGraphSetConditional.
#pragma once

#include "qms_kernels.cuh"
#include "qms_merge.cuh"

namespace qms {

struct DState {
  // written by the host for every launch
  void* keys;
  uint32_t* vals;
  unsigned long long n;
  int xf;
  int pivot;  // QMS_PIVOT_* of the call
  Desc* desc;
  uint32_t* counts;
  unsigned long long* pml;
  unsigned long long* pmr;
  unsigned long long* splits;
  unsigned* flags;  // overlapped-merge tile flags
  uint32_t* wtl;
  uint32_t* wtr;
  int fig3;  // always Fig. 3's side rule
  unsigned spin_limit;  // polls of one flag before a bounded wait gives up
  int withhold;         // test hook: the overlapped merge never publishes tile 0
  // driver state
  unsigned long long b, e;          // remaining range
  unsigned long long lo, hi, parked;  // current partition pass
  unsigned long long k, eq;         // pivot block of the round
  unsigned long long P0, M0, B0;    // the round's Mergesort: part, size, buffer
  unsigned long long P, Bb, m;      // current phase: part, size, buffer
  unsigned long long X, Y, L;       // current merge level
  unsigned long long rounds, mom_rounds;
  unsigned long long launches;  // kernels of the graph that ran (all nodes count)
  unsigned int le, levels, to_buf, mom_next, rule, active, pass2, pad;
  unsigned int half, phase;  // larger side with a half buffer: phases 0 and 1
  // Work nodes whose grid the control kernels size to the round's work
  // (device-updatable kernel nodes); null when the graph was built with
  // fixed grids.  cap: the fixed grid the node was built with.
  cudaGraphDeviceNode_t dn[14];
  unsigned int cap[14];
  unsigned int dyn;
};

enum : int { DN_PART1 = 0, DN_EXCH1 = 1, DN_PART2 = 2, DN_EXCH2 = 3, DN_LEAF = 4, DN_SPLIT = 5,
             DN_MERGE = 6, DN_CHUNK1 = 7, DN_PREF1 = 8, DN_CHUNK2 = 9, DN_PREF2 = 10,
             DN_OSPLIT = 11, DN_OMERGE = 12, DN_ODEPS = 13, DN_COUNT = 14 };

// Loads a call's state (its parameters travel with the launch, so the host
// copy may be reused at once).
__global__ static void k_g_load_state(DState* S, DState v) { *S = v; }

// Sets a work node's grid to cover `units` blocks (at least 1, at most its
// built-in grid).
__device__ __forceinline__ void size_node(DState& s, int i, unsigned long long units) {
  if (!s.dyn) return;
  unsigned long long g = units < 1 ? 1 : units;
  if (g > s.cap[i]) g = s.cap[i];
  cudaGraphKernelNodeSetGridDim(s.dn[i], dim3(static_cast<unsigned>(g)));
}

constexpr int RULE_M3 = 0, RULE_SQRTN = 1, RULE_MOM = 2, RULE_HYBRID = 3;

__device__ __forceinline__ void count_launch(DState* S) {
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&S->launches, 1ull);
}

template <class K, bool HV>
__device__ __forceinline__ void swap_at(DState& s, uint64_t a, uint64_t b) {
  if (a == b) return;
  K* keys = static_cast<K*>(s.keys);
  const K x = keys[a];
  keys[a] = keys[b];
  keys[b] = x;
  if (HV) {
    const uint32_t y = s.vals[a];
    s.vals[a] = s.vals[b];
    s.vals[b] = y;
  }
}

template <class K, bool HV, bool CNT>
__global__ void k_g_begin(DState* S, cudaGraphConditionalHandle h_round) {
  count_launch(S);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DState& s = *S;
  if (s.e - s.b <= static_cast<unsigned long long>(LeafCfg<K, HV>::TILE_L)) {
    s.active = 0;
    cudaGraphSetConditional(h_round, 0);
    return;
  }
  s.active = 1;
  ++s.rounds;
  const uint64_t b = s.b, e = s.e, n = e - b;
  const int rule = (s.pivot == RULE_MOM || (s.pivot == RULE_HYBRID && s.mom_next))
                       ? RULE_MOM
                       : (s.pivot == RULE_SQRTN ? RULE_SQRTN : RULE_M3);
  s.rule = rule;
  s.lo = b;
  s.hi = e - 1;
  s.parked = e - 1;
  s.le = 0;
  s.pass2 = 0;
  {
    const uint64_t nt = (n - 1 + PT - 1) / PT;
    const uint64_t ch = scan_chunk(nt);
    size_node(s, DN_PART1, nt);
    size_node(s, DN_CHUNK1, (nt + ch - 1) / ch);
    size_node(s, DN_PREF1, (nt + ch - 1) / ch);
  }
  Desc* d = s.desc;
  d->L = 0;
  if (rule == RULE_MOM) {
    ++s.mom_rounds;
    d->sel_prefix = 0;
    d->sel_mask = 0;
    d->sel_rank = (n / 3) / 2;
    d->pos = ~0ull;
  } else if (rule == RULE_M3) {
    K* keys = static_cast<K*>(s.keys);
    uint64_t p0 = b, p1 = b + n / 2, p2 = e - 1;
    K u0 = enc_key(keys[p0], s.xf), u1 = enc_key(keys[p1], s.xf), u2 = enc_key(keys[p2], s.xf);
    if (u1 < u0) { K t = u0; u0 = u1; u1 = t; uint64_t q = p0; p0 = p1; p1 = q; }
    unsigned c = 2;
    if (u2 < u1) {
      K t = u1; u1 = u2; u2 = t; uint64_t q = p1; p1 = p2; p2 = q;
      ++c;
      if (u1 < u0) { t = u0; u0 = u1; u1 = t; q = p0; p0 = p1; p1 = q; }
    }
    d->tie = (!(u0 < u1) || !(u1 < u2)) ? 1u : 0u;
    d->pivot = static_cast<unsigned long long>(u1);
    if (CNT) d->cmp += c + 2;
    swap_at<K, HV>(s, p1, e - 1);
  }
}

// Median-of-sqrt(n) sample pivot (one block).
template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(SAMPLE_T) k_g_pivot_sample(DState* S) {
  count_launch(S);
  DState& s = *S;
  if (!s.active || s.rule != RULE_SQRTN) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const auto sm = TileSmem<K, true, SAMPLE_T, V>::carve(smem);
  uint64_t cmp = 0;
  const uint64_t b = s.b, e = s.e, n = e - b;
  uint64_t c = 1;
  while (c * c < n) ++c;
  uint64_t kk = (c & 1) ? c : c - 1;
  if (kk > static_cast<uint64_t>(SAMPLE_MAX)) kk = SAMPLE_MAX;
  const int ks = static_cast<int>(kk);
  const uint64_t step = n / kk;
  K* keys = static_cast<K*>(s.keys);
  for (int i = threadIdx.x; i < SAMPLE_T * V; i += SAMPLE_T) {
    sm.k[sk_i<K>(i)] = (i < ks) ? enc_key(keys[b + static_cast<uint64_t>(i) * step], s.xf) : key_max<K>();
    sm.v[sv_i(i)] = static_cast<uint32_t>(i);
  }
  block_sort_tile<K, true, CNT, SAMPLE_T, V>(sm, cmp);
  if (CNT) flush_count(cmp, &s.desc->cmp);
  if (threadIdx.x == 0) {
    const int h = ks / 2;
    const K med = sm.k[sk_i<K>(h)];
    const uint64_t pm = b + static_cast<uint64_t>(sm.v[sv_i(h)]) * step;
    bool tie = false;
    if (ks >= 3) tie = !(sm.k[sk_i<K>(h - 1)] < med) || !(med < sm.k[sk_i<K>(h + 1)]);
    swap_at<K, HV>(s, pm, e - 1);
    s.desc->pivot = static_cast<unsigned long long>(med);
    s.desc->tie = tie ? 1u : 0u;
    if (CNT) s.desc->cmp += 2;
  }
}

// Median-of-medians pivot (Sec. 4): triple medians, radix select, place.
template <class K, bool HV, bool CNT>
__global__ void k_g_mom_triples(DState* S) {
  count_launch(S);
  DState& s = *S;
  if (!s.active || s.rule != RULE_MOM) return;
  uint64_t cmp = 0;
  const uint64_t b = s.b, t = (s.e - s.b) / 3;
  K* keys = static_cast<K*>(s.keys);
  const int xf = s.xf;
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < t;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
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
    if (mi != 1) {
      const uint64_t p = q + mi;
      keys[q + 1] = (mi == 0) ? x0 : x2;
      keys[p] = x1;
      if (HV) { const uint32_t a = s.vals[p]; s.vals[p] = s.vals[q + 1]; s.vals[q + 1] = a; }
    }
  }
  if (CNT) flush_count(cmp, &s.desc->cmp);
}

template <class K>
__global__ void k_g_sel_hist(DState* S, int shift) {
  count_launch(S);
  DState& s = *S;
  if (!s.active || s.rule != RULE_MOM) return;
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  Desc* d = s.desc;
  const K pre = static_cast<K>(d->sel_prefix), msk = static_cast<K>(d->sel_mask);
  const uint64_t b = s.b, t = (s.e - s.b) / 3;
  const K* keys = static_cast<const K*>(s.keys);
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < t;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const K u = enc_key(keys[b + 3 * i + 1], s.xf);
    if (((u ^ pre) & msk) == 0) atomicAdd(&h[static_cast<unsigned>(u >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&d->hist[i], h[i]);
}

__global__ static void k_g_sel_pick(DState* S, int shift) {
  count_launch(S);
  DState& s = *S;
  if (threadIdx.x != 0 || !s.active || s.rule != RULE_MOM) return;
  Desc* d = s.desc;
  unsigned long long r = d->sel_rank, acc = 0;
  int bin = 255;
  for (int i = 0; i < 256; ++i) {
    const unsigned long long c = d->hist[i];
    if (r < acc + c) { bin = i; break; }
    acc += c;
  }
  d->sel_eq = d->hist[bin];
  d->sel_prefix |= static_cast<unsigned long long>(bin) << shift;
  d->sel_mask |= 255ull << shift;
  d->sel_rank = r - acc;
  for (int i = 0; i < 256; ++i) d->hist[i] = 0;
}

template <class K>
__global__ void k_g_mom_locate(DState* S) {
  count_launch(S);
  DState& s = *S;
  if (!s.active || s.rule != RULE_MOM) return;
  const K v = static_cast<K>(s.desc->sel_prefix);
  const uint64_t b = s.b, t = (s.e - s.b) / 3;
  const K* keys = static_cast<const K*>(s.keys);
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < t;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    if (enc_key(keys[b + 3 * i + 1], s.xf) == v) atomicMin(&s.desc->pos, static_cast<unsigned long long>(i));
  }
}

template <class K, bool HV>
__global__ void k_g_mom_place(DState* S) {
  count_launch(S);
  DState& s = *S;
  if (threadIdx.x != 0 || !s.active || s.rule != RULE_MOM) return;
  Desc* d = s.desc;
  const uint64_t t = (s.e - s.b) / 3;
  if (d->pos >= t) {
    d->err |= 2u;
    s.active = 0;
    return;
  }
  swap_at<K, HV>(s, s.b + 3 * d->pos + 1, s.e - 1);
  d->pivot = d->sel_prefix;
  d->tie = d->sel_eq > 1 ? 1u : 0u;
}

// Partition pass over [lo, hi) (mode le), grid striding over partition tiles.
template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(PNT, (part_minb<K, HV>())) k_g_part_local(DState* S) {
  count_launch(S);
  DState& s = *S;
  if (!s.active) return;
  __shared__ K sk[pk_len<K>()];
  __shared__ uint32_t sv[HV ? pv_len() : 1];
  __shared__ uint32_t scr[PNWARP + 1];
  uint64_t cmp = 0;
  const K piv = static_cast<K>(s.desc->pivot);
  const uint64_t lo = s.lo, n = s.hi - s.lo, ntiles = (n + PT - 1) / PT;
  K* keys = static_cast<K*>(s.keys);
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t off = t * PT;
    const int cnt = static_cast<int>((n - off) < static_cast<uint64_t>(PT) ? (n - off) : PT);
    __syncthreads();
    K* const g = keys + lo + off;
    uint32_t* const gv = HV ? s.vals + lo + off : nullptr;
    const uint32_t c =
        cnt == PT ? part_local_small<K, HV, CNT, true>(g, gv, cnt, piv, s.le != 0, s.xf, sk, sv, scr, cmp)
                  : part_local_small<K, HV, CNT>(g, gv, cnt, piv, s.le != 0, s.xf, sk, sv, scr, cmp);
    if (threadIdx.x == 0) {
      s.counts[t] = c;
      atomicAdd(&s.desc->L, static_cast<unsigned long long>(c));
    }
  }
  if (CNT) flush_count(cmp, &s.desc->cmp);
}

__global__ static void __launch_bounds__(NT) k_g_part_chunks(DState* S) {
  count_launch(S);
  DState& s = *S;
  if (!s.active) return;
  scan_chunks_body(s.lo, s.hi, s.counts, s.desc);
}

__global__ static void __launch_bounds__(NT) k_g_part_prefix(DState* S) {
  count_launch(S);
  DState& s = *S;
  if (!s.active) return;
  scan_prefix_body(s.lo, s.hi, s.counts, reinterpret_cast<uint64_t*>(s.pml),
                   reinterpret_cast<uint64_t*>(s.pmr), s.wtl, s.wtr, s.desc);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (s.desc->err) s.active = 0;
    const unsigned long long per = static_cast<unsigned long long>(EXB) * EXW;
    size_node(s, s.pass2 ? DN_EXCH2 : DN_EXCH1, (s.desc->mis + per - 1) / per);
  }
}

// P: uint32_t positions (graphs for arrays shorter than 2^32 keys), else uint64_t.
template <class K, bool HV, class P>
__global__ void __launch_bounds__(EXB) k_g_part_exchange(DState* S) {
  count_launch(S);
  const DState& s = *S;
  if (!s.active) return;
  // the state, read once (the stores to the keys could alias it otherwise)
  K* const keys = static_cast<K*>(s.keys);
  uint32_t* const vals = s.vals;
  const uint32_t* const counts = s.counts;
  const uint64_t* const pml = reinterpret_cast<const uint64_t*>(s.pml);
  const uint64_t* const pmr = reinterpret_cast<const uint64_t*>(s.pmr);
  const uint32_t* const wtl = s.wtl;
  const uint32_t* const wtr = s.wtr;
  const uint64_t mis = s.desc->mis, lo = s.lo;
  const uint64_t sb = lo + s.desc->L;
  const uint64_t w0 = (blockIdx.x * static_cast<uint64_t>(EXB) + threadIdx.x) >> 5;
  const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * EXB) >> 5;
  for (uint64_t jw = w0 * EXJ; jw < mis; jw += nw * EXJ)
    exchange_warp<K, HV, P>(keys, vals, lo, sb, counts, pml, pmr, wtl, wtr, jw, mis);
}

template <class K, bool HV>
__global__ void k_g_mid(DState* S, cudaGraphConditionalHandle h_pass2) {
  count_launch(S);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DState& s = *S;
  s.pass2 = 0;
  if (s.active) {
    const uint64_t k = s.lo + s.desc->L;
    swap_at<K, HV>(s, k, s.parked);
    s.k = k;
    if (s.desc->tie && k + 1 < s.e) {
      s.lo = k + 1;
      s.hi = s.e;
      s.le = 1;
      s.parked = ~0ull;
      s.pass2 = 1;
      s.desc->L = 0;
      const uint64_t nt = (s.hi - s.lo + PT - 1) / PT;
      const uint64_t ch = scan_chunk(nt);
      size_node(s, DN_PART2, nt);
      size_node(s, DN_CHUNK2, (nt + ch - 1) / ch);
      size_node(s, DN_PREF2, (nt + ch - 1) / ch);
    }
  }
  cudaGraphSetConditional(h_pass2, s.pass2);
}

// Sets up Mergesort phase ph of the round: the part, its buffer, the
// number of levels and where the leaves go, so that the sorted part ends in
// its own range (Fig. 3 rule, one phase) or in its target (half-buffer
// rounds: phase 0 sorts the second half into the buffer, phase 1 the first
// half into the tail of the part).
template <class K, bool HV>
__device__ __forceinline__ void setup_phase(DState& s, unsigned ph, cudaGraphConditionalHandle h_level) {
  bool into_buf = false;
  if (!s.half) {
    s.P = s.P0;
    s.m = s.M0;
    s.Bb = s.B0;
  } else {
    const unsigned long long q = s.M0 / 2, r = s.M0 - q;
    into_buf = true;
    if (ph == 0) {
      s.P = s.P0 + q;
      s.m = r;
      s.Bb = s.B0;
    } else {
      s.P = s.P0;
      s.m = q;
      s.Bb = s.P0 + r;
    }
  }
  s.phase = ph;
  constexpr uint64_t TL = LeafCfg<K, HV>::TILE_L;
  const uint64_t leaves = (s.m + TL - 1) / TL;
  unsigned levels = 0;
  while ((1ull << levels) < leaves) ++levels;
  s.levels = levels;
  s.to_buf = ((levels & 1u) != 0) != into_buf ? 1u : 0u;
  s.X = s.to_buf ? s.Bb : s.P;
  s.Y = s.to_buf ? s.P : s.Bb;
  s.L = TL;
  size_node(s, DN_LEAF, leaves);
  const unsigned long long mt = MergeCfg<K, HV>::MT;
  const unsigned long long mtiles = (s.m + mt - 1) / mt;
  size_node(s, DN_SPLIT, (mtiles + 255) / 256);
  size_node(s, DN_MERGE, mtiles);
  cudaGraphSetConditional(h_level, s.levels > 0 ? 1u : 0u);
}

// HALF: the graph holds the phase loop and the overlapped merge (handles
// h_phase and h_ovl); without it every round takes Fig. 3's rule.
template <class K, bool HV, bool HALF>
__global__ void k_g_side(DState* S, cudaGraphConditionalHandle h_level,
                         cudaGraphConditionalHandle h_phase, cudaGraphConditionalHandle h_ovl) {
  count_launch(S);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DState& s = *S;
  s.levels = 0;
  s.m = 0;
  s.M0 = 0;
  s.half = 0;
  if (s.active) {
    const uint64_t b = s.b, e = s.e, nn = e - b, k = s.k;
    const uint64_t eq = s.pass2 ? s.desc->L : 0;
    s.eq = eq;
    if (s.pivot == RULE_HYBRID) {
      const uint64_t d = nn / 16, rlo = k - b, rhi = k + eq - b;
      s.mom_next = (s.rule != RULE_MOM && (rhi < d || rlo > nn - 1 - d)) ? 1u : 0u;
    }
    const uint64_t rb = k + 1 + eq;
    const uint64_t nl = k - b, nr = e - rb;
    const int side = choose_side(b, e, k, eq, !HALF || s.fig3 != 0);
    s.half = (side == SIDE_LARGER_LEFT || side == SIDE_LARGER_RIGHT) ? 1u : 0u;
    if (side == SIDE_LEFT || side == SIDE_LARGER_LEFT) {
      s.P0 = b;
      s.M0 = nl;
      s.B0 = rb;
      s.b = rb;
    } else {
      s.P0 = rb;
      s.M0 = nr;
      s.B0 = b;
      s.e = k;
    }
    setup_phase<K, HV>(s, 0, h_level);
    if (s.half) {
      const unsigned long long mt = MergeCfg<K, HV>::MT;
      const unsigned long long mtiles = (s.M0 + mt - 1) / mt;
      size_node(s, DN_OSPLIT, (mtiles + 255) / 256);
      size_node(s, DN_ODEPS, (mtiles + 255) / 256);
      size_node(s, DN_OMERGE, mtiles);
    }
  } else {
    cudaGraphSetConditional(h_level, 0u);
  }
  if (HALF) {
    cudaGraphSetConditional(h_phase, s.active ? 1u : 0u);
    cudaGraphSetConditional(h_ovl, s.active && s.half ? 1u : 0u);
  }
}

// After a Mergesort phase: the next phase of a half-buffer round, or done.
template <class K, bool HV>
__global__ void k_g_phase_end(DState* S, cudaGraphConditionalHandle h_phase,
                              cudaGraphConditionalHandle h_level) {
  count_launch(S);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DState& s = *S;
  if (s.active && s.half && s.phase == 0 && !s.desc->err) {
    setup_phase<K, HV>(s, 1, h_level);
    cudaGraphSetConditional(h_phase, 1u);
  } else {
    cudaGraphSetConditional(h_phase, 0u);
  }
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(256) k_g_ovl_split(DState* S) {
  count_launch(S);
  const DState& s = *S;
  if (!s.active) return;
  const uint64_t q = s.M0 / 2, r = s.M0 - q;
  uint64_t cmp = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) s.desc->oticket = 0;
  const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t ngroups = (s.M0 + MergeCfg<K, HV>::MT * 32ull - 1) / (MergeCfg<K, HV>::MT * 32ull);
  for (uint64_t w = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; w < ngroups;
       w += nw)
    ovl_split_group<K, HV, CNT>(static_cast<const K*>(s.keys), s.B0, r, s.P0, q, s.xf,
                                reinterpret_cast<uint64_t*>(s.splits), s.flags, w, cmp);
  if (CNT) flush_count(cmp, &s.desc->cmp);
}

// The wait ranges live in the exchange start tables, which the partition
// alone uses.
template <class K, bool HV>
__global__ void __launch_bounds__(256) k_g_ovl_deps(DState* S) {
  count_launch(S);
  const DState& s = *S;
  if (!s.active) return;
  constexpr int MT = MergeCfg<K, HV>::MT;
  const uint64_t q = s.M0 / 2, r = s.M0 - q;
  const uint64_t ntiles = (s.M0 + MT - 1) / MT;
  for (uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; t < ntiles;
       t += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    ovl_deps_tile<MT>(r, q, reinterpret_cast<const uint64_t*>(s.splits), s.wtl, s.wtr, t);
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(MBT, MergeCfg<K, HV>::MINB) k_g_ovl_merge(DState* S) {
  count_launch(S);
  const DState& s = *S;
  if (!s.active) return;
  const uint64_t q = s.M0 / 2, r = s.M0 - q;
  ovl_merge_loop<K, HV, CNT>(static_cast<K*>(s.keys), s.vals, s.B0, r, s.P0, q,
                             reinterpret_cast<const uint64_t*>(s.splits), s.wtl, s.wtr, s.flags,
                             s.xf, s.desc, s.spin_limit, s.withhold);
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(LeafCfg<K, HV>::LT, LeafCfg<K, HV>::MINB) k_g_leaf(DState* S) {
  constexpr int LT = LeafCfg<K, HV>::LT, TL = LeafCfg<K, HV>::TILE_L, VL = LeafCfg<K, HV>::VL;
  count_launch(S);
  DState& s = *S;
  if (!s.active || s.m <= 1) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const auto sm = TileSmem<K, HV, LT, VL>::carve(smem);
  uint64_t cmp = 0;
  const uint64_t m = s.m, P = s.P, Bb = s.Bb;
  const bool to_buf = s.to_buf != 0;
  K* keys = static_cast<K*>(s.keys);
  const uint64_t ntiles = (m + TL - 1) / TL;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t off = t * TL;
    const int cnt = static_cast<int>((m - off) < static_cast<uint64_t>(TL) ? (m - off) : TL);
    leaf_sort_tile<K, HV, CNT, LT, VL>(sm, keys + P + off, HV ? s.vals + P + off : nullptr,
                                   to_buf ? keys + Bb + off : nullptr,
                                   (HV && to_buf) ? s.vals + Bb + off : nullptr, cnt, s.xf, cmp);
  }
  if (CNT) flush_count(cmp, &s.desc->cmp);
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(256) k_g_split(DState* S) {
  grid_dep_wait();
  grid_dep_trigger();  // the merge node may start and load its buffer tiles
  count_launch(S);
  const DState& s = *S;
  uint64_t cmp = 0;
  const uint64_t ngroups = (s.m + MergeCfg<K, HV>::MT * 32ull - 1) / (MergeCfg<K, HV>::MT * 32ull);
  const uint64_t nw = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t w = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; w < ngroups;
       w += nw)
    split_group<K, HV, CNT>(static_cast<const K*>(s.keys), s.X, s.m, s.L, s.xf,
                            reinterpret_cast<uint64_t*>(s.splits), w, cmp);
  if (CNT) flush_count(cmp, &s.desc->cmp);
}

// One swap-merge level of the level loop.  The last block to finish ends
// the level: doubles the run length, swaps the regions and sets the loop's
// condition (all other blocks have read the level's state by then).
template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(MBT, MergeCfg<K, HV>::MINB)
    k_g_merge(DState* S, cudaGraphConditionalHandle h_level) {
  count_launch(S);
  DState& s = *S;
  using C = MergeCfg<K, HV>;
  const uint64_t m = s.m, L = s.L, X = s.X, Y = s.Y;
  const uint64_t ntiles = (m + C::MT - 1) / C::MT;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    merge_level_tile<K, HV, CNT>(static_cast<K*>(s.keys), s.vals, X, Y, m, L,
                                 reinterpret_cast<const uint64_t*>(s.splits), s.xf, s.desc, t,
                                 t == blockIdx.x);
  }
  grid_dep_wait();  // (blocks without a tile) the split step has finished
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&s.desc->mdone, 1u) == gridDim.x - 1) {
      s.desc->mdone = 0;
      s.L = L * 2;
      s.X = Y;
      s.Y = X;
      --s.levels;
      cudaGraphSetConditional(h_level, s.levels > 0 ? 1u : 0u);
    }
  }
}

// Enters the round loop only if the array is longer than one leaf tile
// (else the graph goes straight to the final leaf sort).
template <class K, bool HV>
__global__ void k_g_start(DState* S, cudaGraphConditionalHandle h_round) {
  count_launch(S);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const DState& s = *S;
  cudaGraphSetConditional(
      h_round, s.e - s.b > static_cast<unsigned long long>(LeafCfg<K, HV>::TILE_L) ? 1u : 0u);
}

template <class K, bool HV>
__global__ void k_g_end(DState* S, cudaGraphConditionalHandle h_round) {
  count_launch(S);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DState& s = *S;
  const bool more =
      s.active && s.e - s.b > static_cast<unsigned long long>(LeafCfg<K, HV>::TILE_L) && !s.desc->err;
  cudaGraphSetConditional(h_round, more ? 1u : 0u);
}

template <class K, bool HV, bool CNT>
__global__ void __launch_bounds__(LeafCfg<K, HV>::LT) k_g_final(DState* S) {
  constexpr int LT = LeafCfg<K, HV>::LT, VL = LeafCfg<K, HV>::VL;
  count_launch(S);
  DState& s = *S;
  if (s.desc->err || s.e - s.b <= 1) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const auto sm = TileSmem<K, HV, LT, VL>::carve(smem);
  uint64_t cmp = 0;
  const uint64_t b = s.b;
  K* keys = static_cast<K*>(s.keys);
  leaf_sort_tile<K, HV, CNT, LT, VL>(sm, keys + b, HV ? s.vals + b : nullptr, nullptr, nullptr,
                                 static_cast<int>(s.e - b), s.xf, cmp);
  if (CNT) flush_count(cmp, &s.desc->cmp);
}

}  // namespace qms
