// Device primitives of the GB300 QuickMergesort path (sm_103a).
//
// Paper: Edelkamp & Weiss, "QuickMergesort: Practically Efficient
// Constant-Factor Optimal Sorting", arXiv 1804.10062.
//
// Every routine here is CTA-scoped: one thread block works on one tile, and
// the kernels in qms_kernels.cuh either spread tiles over a grid or loop over
// them inside one block.  Keys are moved in their raw bit pattern and
// compared as unsigned "order keys" (a bijection computed in registers):
//   uint32 / uint64 : identity
//   int64           : flip the sign bit
//   float32         : IEEE totalOrder bits (negative: all bits flipped;
//                     non-negative: sign bit set), so -0 < +0.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace qms {

constexpr int NT = 512;          // threads per block
constexpr int V = 16;            // items per thread
constexpr int TILE = NT * V;     // keys per tile (leaf, partition, merge)
constexpr int NWARP = NT / 32;

enum : int { XF_NONE = 0, XF_F32 = 1, XF_I64 = 2 };

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with a programmatic
// dependency on the one before it in its stream (or graph) may start while
// that one still runs.  grid_dep_wait() returns once the earlier grid has
// finished and its writes are visible (at once when there is no such
// dependency); grid_dep_trigger() lets the next kernel start once every
// block of this one has called it.  Kernels call wait before trigger, so a
// kernel that starts early never overlaps the one two steps back.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Order keys

__device__ __forceinline__ uint32_t enc_key(uint32_t b, int xf) {
  if (xf == XF_F32) return b ^ (static_cast<uint32_t>(static_cast<int32_t>(b) >> 31) | 0x80000000u);
  return b;
}
__device__ __forceinline__ uint32_t dec_key(uint32_t u, int xf) {
  if (xf == XF_F32) return u ^ (((u >> 31) - 1u) | 0x80000000u);
  return u;
}
__device__ __forceinline__ uint64_t enc_key(uint64_t b, int xf) {
  return xf == XF_I64 ? (b ^ 0x8000000000000000ull) : b;
}
__device__ __forceinline__ uint64_t dec_key(uint64_t u, int xf) {
  return xf == XF_I64 ? (u ^ 0x8000000000000000ull) : u;
}

// The same transforms with the kind fixed at compile time, and with_xf,
// which calls f with the kind of a launch as such a constant: one uniform
// branch per call instead of a test per element.
template <int X>
using XfC = std::integral_constant<int, X>;
template <int X>
__device__ __forceinline__ uint32_t enc_key(uint32_t b, XfC<X>) {
  return X == XF_F32 ? enc_key(b, XF_F32) : b;
}
template <int X>
__device__ __forceinline__ uint32_t dec_key(uint32_t u, XfC<X>) {
  return X == XF_F32 ? dec_key(u, XF_F32) : u;
}
template <int X>
__device__ __forceinline__ uint64_t enc_key(uint64_t b, XfC<X>) {
  return X == XF_I64 ? (b ^ 0x8000000000000000ull) : b;
}
template <int X>
__device__ __forceinline__ uint64_t dec_key(uint64_t u, XfC<X>) {
  return X == XF_I64 ? (u ^ 0x8000000000000000ull) : u;
}
template <class K, class F>
__device__ __forceinline__ void with_xf(int xf, F&& f) {
  if (xf == XF_NONE)
    f(XfC<XF_NONE>{});
  else
    f(XfC<sizeof(K) == 4 ? XF_F32 : XF_I64>{});
}

template <class K>
__device__ __forceinline__ K key_max() {
  return static_cast<K>(~static_cast<K>(0));
}

// Shared-memory index with one padding element per 128 bytes, so that the
// blocked (thread-contiguous) accesses of the sort do not conflict on banks.
template <class K>
__device__ __forceinline__ int sk_i(int i) {
  return i + i / (128 / static_cast<int>(sizeof(K)));
}
__device__ __forceinline__ int sv_i(int i) { return i + (i >> 5); }

// Shared-memory tiles hold LT * VV keys: LT = NT threads of VV = V keys
// (8192 keys) everywhere but in the Mergesort leaves (LeafCfg).
template <class K, int LT = NT, int VV = V>
__host__ __device__ constexpr int sk_len() {
  return LT * VV + LT * VV / (128 / static_cast<int>(sizeof(K))) + 4;
}
template <int LT = NT, int VV = V>
__host__ __device__ constexpr int sv_len() { return LT * VV + LT * VV / 32 + 4; }

// Scratch words used by block scans and small per-block tables.
constexpr int SCRATCH_WORDS = 64;

template <class K, bool HV, int LT = NT, int VV = V>
__host__ __device__ constexpr size_t tile_smem_bytes() {
  return static_cast<size_t>(sk_len<K, LT, VV>()) * sizeof(K) +
         (HV ? static_cast<size_t>(sv_len<LT, VV>()) * 4 : 0) + SCRATCH_WORDS * 8;
}

template <class K, bool HV, int LT = NT, int VV = V>
struct TileSmem {
  K* k;
  uint32_t* v;
  uint32_t* scratch;  // SCRATCH_WORDS * 2 uint32 words
  __device__ __forceinline__ static TileSmem carve(unsigned char* base) {
    TileSmem s;
    s.k = reinterpret_cast<K*>(base);
    size_t off = static_cast<size_t>(sk_len<K, LT, VV>()) * sizeof(K);
    s.v = HV ? reinterpret_cast<uint32_t*>(base + off) : nullptr;
    if (HV) off += static_cast<size_t>(sv_len<LT, VV>()) * 4;
    s.scratch = reinterpret_cast<uint32_t*>(base + off);
    return s;
  }
};

// Mergesort leaves: LT threads of VL keys each.
//   - 4-byte keys without payloads: 16384-key leaves of 512 threads x 32
//     keys, two blocks per SM.  Each thread's 32 keys are sorted by a
//     network in registers, so a leaf needs 9 shared-memory merge rounds
//     instead of 10, and every merge-path search serves 32 outputs.
//   - 8-byte keys without payloads: 16384-key leaves of 1024 threads x 16
//     keys (about 53 registers), one block of 139 KB shared memory per SM.
//   - With payloads: 8192-key leaves of 512 threads x 16, two blocks per SM
//     (64 registers; for 8-byte keys a few spills, still faster than one
//     block per SM).
// 16384-key leaves save one HBM merge level per Mergesort against 8192.
#ifndef QMS_LEAF_U32
#define QMS_LEAF_U32 0  // 0: 512 x 32 keys; 1: 1024 x 32 (32768-key leaves); 2: 1024 x 16
#endif
template <class K, bool HV>
struct LeafCfg {
  static constexpr bool W32 = sizeof(K) == 4 && !HV;
  static constexpr int LT = HV ? NT : (W32 && QMS_LEAF_U32 == 0 ? NT : 2 * NT);
  static constexpr int VL = W32 && QMS_LEAF_U32 != 2 ? 2 * V : V;
  static constexpr int TILE_L = LT * VL;
  static constexpr int MINB = (W32 && QMS_LEAF_U32 == 1) ? 1 : ((W32 || HV) ? 2 : 1);  // blocks per SM built for
};

// ---------------------------------------------------------------------------
// Block-wide scans (NT threads)

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive scan of x over the block; *total receives the block sum.
// scratch needs NWARP + 1 words.  Contains __syncthreads.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* scratch,
                                                    uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(x);
  if (lane == 31) scratch[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t s = lane < NWARP ? scratch[lane] : 0u;
    const uint32_t si = warp_incl_scan(s);
    if (lane < NWARP) scratch[lane] = si - s;
    if (lane == 31) scratch[NWARP] = si;
  }
  __syncthreads();
  const uint32_t r = scratch[w] + inc - x;
  *total = scratch[NWARP];
  __syncthreads();
  return r;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Adds a per-thread comparison count to a global counter (one atomic per warp).
__device__ __forceinline__ void flush_count(uint64_t c, unsigned long long* dst) {
  c = warp_sum_u64(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(dst, static_cast<unsigned long long>(c));
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, one element each): many
// copies stay in flight per thread without occupying registers.

__device__ __forceinline__ void cp_async_elem(uint32_t* smem, const uint32_t* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(uint64_t* smem, const uint64_t* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// Tile load / store (striped: item j of thread t is element j*NT + t)

template <class K, bool HV, int LT = NT, int VV = V>
__device__ __forceinline__ void load_tile_enc(TileSmem<K, HV, LT, VV> s, const K* g, const uint32_t* gv,
                                              int cnt, int xf) {
#pragma unroll 8
  for (int j = 0; j < VV; ++j) {
    const int i = j * LT + threadIdx.x;
    s.k[sk_i<K>(i)] = (i < cnt) ? enc_key(g[i], xf) : key_max<K>();
    if (HV) s.v[sv_i(i)] = (i < cnt) ? gv[i] : 0xffffffffu;
  }
}

template <class K, bool HV, int LT = NT, int VV = V>
__device__ __forceinline__ void store_tile_dec(TileSmem<K, HV, LT, VV> s, K* g, uint32_t* gv, int cnt,
                                               int xf) {
#pragma unroll
  for (int j = 0; j < VV; ++j) {
    const int i = j * LT + threadIdx.x;
    if (i < cnt) {
      g[i] = dec_key(s.k[sk_i<K>(i)], xf);
      if (HV) gv[i] = s.v[sv_i(i)];
    }
  }
}

// Copies cnt elements src -> dst (global to global, no overlap), striped.
// cnt <= LT * VV: each thread issues its loads in batches of VV/4 before the
// matching stores (four round trips, few registers).
template <class K, bool HV, int LT = NT, int VV = V>
__device__ __forceinline__ void copy_elems(K* dst, uint32_t* dv, const K* src, const uint32_t* sv,
                                           int cnt) {
  constexpr int B = VV / 4;
#pragma unroll
  for (int jb = 0; jb < VV; jb += B) {
    K t[B];
    uint32_t tv[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int i = (jb + j) * LT + threadIdx.x;
      if (i < cnt) {
        t[j] = src[i];
        if (HV) tv[j] = sv[i];
      }
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int i = (jb + j) * LT + threadIdx.x;
      if (i < cnt) {
        dst[i] = t[j];
        if (HV) dv[i] = tv[j];
      }
    }
  }
}


// ---------------------------------------------------------------------------
// Merge path (stable: on equal keys the A element goes first)

// Number of A elements among the first d outputs of merging sorted runs
// A = s[a0, a0+la) and B = s[b0, b0+lb) held in shared memory.
template <class K, bool CNT>
__device__ __forceinline__ int merge_path_smem(const K* sk, int a0, int la, int b0, int lb, int d,
                                               uint64_t& cmp) {
  int lo = d > lb ? d - lb : 0;
  int hi = d < la ? d : la;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (CNT) ++cmp;
    if (!(sk[sk_i<K>(b0 + d - 1 - mid)] < sk[sk_i<K>(a0 + mid)])) {
      lo = mid + 1;
    } else {
      hi = mid;
    }
  }
  return lo;
}

// Serial stable merge of V outputs starting at A index ai / B index bi.
// Keys land in k[], the source indices (for payloads) in src[].  Branch
// free: one shared-memory load per output, of the element that replaces the
// one just taken.  A load past a run's end stays inside the tile's array and
// is never used (the bound checks decide first).
template <class K, bool CNT>
__device__ __forceinline__ void serial_merge(const K* sk, int ai, int ae, int bi, int be, K (&k)[V],
                                             int (&src)[V], uint64_t& cmp) {
  K ka = sk[sk_i<K>(ai)];
  K kb = sk[sk_i<K>(bi)];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const bool a_ok = ai < ae, b_ok = bi < be;
    if (CNT && a_ok && b_ok) ++cmp;
    const bool tb = b_ok && (!a_ok || kb < ka);
    k[j] = tb ? kb : ka;
    src[j] = tb ? bi : ai;
    ai += tb ? 0 : 1;
    bi += tb ? 1 : 0;
    const K nk = sk[sk_i<K>(tb ? bi : ai)];
    ka = tb ? ka : nk;
    kb = tb ? nk : kb;
  }
}

// The same merge, with the payloads read along (no source indices kept).
template <class K, bool HV, bool CNT, int VV = V>
__device__ __forceinline__ void serial_merge_kv(const K* sk, const uint32_t* sv, int ai, int ae,
                                                int bi, int be, K (&k)[VV], uint32_t (&v)[VV],
                                                uint64_t& cmp) {
  K ka = sk[sk_i<K>(ai)];
  K kb = sk[sk_i<K>(bi)];
#pragma unroll
  for (int j = 0; j < VV; ++j) {
    const bool a_ok = ai < ae, b_ok = bi < be;
    if (CNT && a_ok && b_ok) ++cmp;
    const bool tb = b_ok && (!a_ok || kb < ka);
    k[j] = tb ? kb : ka;
    if (HV) v[j] = sv[sv_i(tb ? bi : ai)];
    ai += tb ? 0 : 1;
    bi += tb ? 1 : 0;
    const K nk = sk[sk_i<K>(tb ? bi : ai)];
    ka = tb ? ka : nk;
    kb = tb ? nk : kb;
  }
}

// Batcher's merge-exchange network (Knuth, TAOCP 5.2.2, Algorithm M) for
// N = 2^t inputs, as a compile-time comparator list.
struct NetPair {
  int a, b;
};
template <int N>
struct MergeExchangeNet {
  NetPair c[N * N];
  int len;
  constexpr MergeExchangeNet() : c{}, len(0) {
    int t = 0;
    while ((1 << t) < N) ++t;
    for (int p = 1 << (t - 1); p > 0; p >>= 1) {
      int q = 1 << (t - 1), r = 0, d = p;
      for (;;) {
        for (int i = 0; i + d < N; ++i)
          if ((i & p) == r) c[len++] = NetPair{i, i + d};
        if (q == p) break;
        d = q - p;
        q >>= 1;
        r = p;
      }
    }
  }
};
template <int N>
inline constexpr MergeExchangeNet<N> kNet{};

// Sorts the VV register items of one thread with the network (comparator I
// onwards).
template <class K, bool HV, int VV = V, int I = 0>
__device__ __forceinline__ void net_sort(K (&k)[VV], uint32_t (&v)[VV]) {
  if constexpr (I < kNet<VV>.len) {
    constexpr int a = kNet<VV>.c[I].a, b = kNet<VV>.c[I].b;
    if (!HV && sizeof(K) == 4) {
      const K lo = min(k[a], k[b]);
      k[b] = max(k[a], k[b]);
      k[a] = lo;
    } else {
      const bool sw = k[b] < k[a];
      const K lo = sw ? k[b] : k[a];
      const K hi = sw ? k[a] : k[b];
      k[a] = lo;
      k[b] = hi;
      if (HV) {
        const uint32_t x = sw ? v[b] : v[a];
        const uint32_t y = sw ? v[a] : v[b];
        v[a] = x;
        v[b] = y;
      }
    }
    net_sort<K, HV, VV, I + 1>(k, v);
  }
}

// Barrier among the threads that share a merge pair of `threads` threads
// (a power of two) in a tile sort of LT threads: the warp while the pair
// fits in one, half of a 2*NT-thread block (named barriers 1 and 2) while it
// fits there, else the block.  Every thread of the block calls it.
template <int LT>
__device__ __forceinline__ void tile_sync(int threads) {
  if (threads <= 32) {
    __syncwarp();
  } else if (LT == 2 * NT && threads <= NT) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + static_cast<int>(threadIdx.x) / NT), "r"(NT) : "memory");
  } else {
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Base case X: sort of one full tile in shared memory.  A sorting network
// on the V items each thread holds in registers (Batcher's merge exchange,
// 63 comparators for V = 16), then log2(NT) rounds of merge-path merges in
// shared memory.

// Keys without payloads: the runs of every round alternate between
// ascending and descending order, so each pair of runs to merge lies in
// shared memory as one bitonic sequence (A ascending, then B descending).
// From its merge-path split a thread repeatedly takes the smaller of the two
// ends of its remaining range: that range stays bitonic, so its minimum is
// at one end, and the two ends never pass each other before the thread's VV
// outputs are out, so the loop needs no bound checks.  Equal keys are equal
// bit patterns here, so which of two equal keys goes first does not matter.
// Thread lt (< P) of the P threads holding data sorts sk[0, P * VV);
// sync(t) is a barrier among the groups of t threads that share a run pair
// (every thread of the caller's group calls it).
template <class K, bool CNT, int VV, class Sync>
__device__ __forceinline__ void tile_sort_keys(K* sk, int lt, int P, Sync&& sync, uint64_t& cmp) {
  static_assert((128 / static_cast<int>(sizeof(K))) % VV == 0,
                "a thread's VV keys must share one padded row");
  K k[VV];
  if (lt < P) {
    const int base = sk_i<K>(lt * VV);
#pragma unroll
    for (int j = 0; j < VV; ++j) k[j] = sk[base + j];
    uint32_t none[VV];
    net_sort<K, false, VV>(k, none);
    if (CNT) cmp += kNet<VV>.len;
    // the odd thread of each first-round pair stores its keys descending
    const bool desc = (lt & 1) && P > 1;
    const int b2 = desc ? base + VV - 1 : base;
    const int step = desc ? -1 : 1;
#pragma unroll
    for (int j = 0; j < VV; ++j) sk[b2 + j * step] = k[j];
  }
  sync(2);
  for (int sp = 1; sp < P; sp <<= 1) {
    const int L = sp * VV;
    const int g = lt / (2 * sp), r = lt - g * 2 * sp;
    const int a0 = g * 2 * L;
    const int d = r * VV;
    if (lt < P) {
      // A = sk[a0, a0 + L) ascending; B[q] = sk[a0 + 2L - 1 - q].
      int lo = d > L ? d - L : 0, hi = d < L ? d : L;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (CNT) ++cmp;
        if (!(sk[sk_i<K>(a0 + 2 * L - d + mid)] < sk[sk_i<K>(a0 + mid)])) lo = mid + 1; else hi = mid;
      }
      int i = a0 + lo;                    // next A key
      int j = a0 + 2 * L - 1 - (d - lo);  // next B key
      K ka = sk[sk_i<K>(i)];
      K kb = sk[sk_i<K>(j)];
#pragma unroll
      for (int t = 0; t < VV; ++t) {
        if (CNT) ++cmp;
        const bool tb = kb < ka;
        k[t] = tb ? kb : ka;
        if (t + 1 < VV) {  // after the last output the range may be empty
          i += tb ? 0 : 1;
          j -= tb ? 1 : 0;
          const K nk = sk[sk_i<K>(tb ? j : i)];
          ka = tb ? ka : nk;
          kb = tb ? nk : kb;
        }
      }
    }
    sync(2 * sp);  // the pair's reads are done before its writes
    if (lt < P) {
      // The merged run is the next round's B (stored descending) when its
      // index is odd and a next round exists: k[t] goes to a0 + d + t, or
      // to a0 + 2L - 1 - d - t.
      const bool desc = (g & 1) && 4 * sp <= P;
      const int base = desc ? sk_i<K>(a0 + 2 * L - 1 - d) : sk_i<K>(a0 + d);
      const int step = desc ? -1 : 1;
#pragma unroll
      for (int t = 0; t < VV; ++t) sk[base + t * step] = k[t];
    }
    if (2 * sp < P) sync(4 * sp);  // the next round's pairs see the writes
  }
}

template <class K, bool HV, bool CNT, int LT = NT, int VV = V>
__device__ void block_sort_tile(TileSmem<K, HV, LT, VV> s, uint64_t& cmp, int P = LT) {
  // P (a power of two <= LT): threads holding data; items beyond the data
  // are padding keys, so the first P*VV items end up sorted.
  if constexpr (!HV) {
    __syncthreads();
    tile_sort_keys<K, CNT, VV>(s.k, static_cast<int>(threadIdx.x), P,
                               [](int t) { tile_sync<LT>(t); }, cmp);
    __syncthreads();  // the whole sorted tile is visible to the block
    return;
  }
  const int tid = threadIdx.x;
  K k[VV];
  uint32_t v[VV];
  __syncthreads();
  if (tid < P) {  // each thread reads, sorts and writes back its own VV keys
#pragma unroll
    for (int j = 0; j < VV; ++j) {
      k[j] = s.k[sk_i<K>(tid * VV + j)];
      if (HV) v[j] = s.v[sv_i(tid * VV + j)];
    }
    net_sort<K, HV, VV>(k, v);
    if (CNT) cmp += kNet<VV>.len;
#pragma unroll
    for (int j = 0; j < VV; ++j) {
      s.k[sk_i<K>(tid * VV + j)] = k[j];
      if (HV) s.v[sv_i(tid * VV + j)] = v[j];
    }
  }
  tile_sync<LT>(2);
  for (int sp = 1; sp < P; sp <<= 1) {
    const int L = sp * VV;
    const int g = tid / (2 * sp), r = tid - g * 2 * sp;
    const int a0 = g * 2 * L, b0 = a0 + L;
    const int d = r * VV;
    if (tid < P) {
      const int ia = merge_path_smem<K, CNT>(s.k, a0, L, b0, L, d, cmp);
      serial_merge_kv<K, HV, CNT, VV>(s.k, s.v, a0 + ia, a0 + L, b0 + d - ia, b0 + L, k, v, cmp);
    }
    tile_sync<LT>(2 * sp);  // the pair's reads are done before its writes
    if (tid < P) {
#pragma unroll
      for (int j = 0; j < VV; ++j) {
        s.k[sk_i<K>(a0 + d + j)] = k[j];
        if (HV) s.v[sv_i(a0 + d + j)] = v[j];
      }
    }
    if (2 * sp < P) tile_sync<LT>(4 * sp);  // the next round's pairs see the writes
  }
  __syncthreads();  // the whole sorted tile is visible to the block
}

// Smallest power of two P with P * VV >= cnt.
template <int VV = V>
__device__ __forceinline__ int threads_for(int cnt) {
  int P = 1;
  while (P * VV < cnt) P <<= 1;
  return P;
}

// Sorts the tile g[0, cnt) (cnt <= TILE).  If buf != nullptr the sorted keys
// are written to buf[0, cnt) and buf's old contents move to g[0, cnt) (the
// Mergesort leaf "X then swap into the target", Fig. 3 msort); otherwise the
// tile is sorted in place.
template <class K, bool HV, bool CNT, int LT = NT, int VV = V>
__device__ __forceinline__ void leaf_sort_tile(TileSmem<K, HV, LT, VV> s, K* g, uint32_t* gv, K* buf, uint32_t* bufv,
                               int cnt, int xf, uint64_t& cmp) {
  const int P = threads_for<VV>(cnt);
  __syncthreads();
  if (P == LT) {
    load_tile_enc<K, HV, LT, VV>(s, g, gv, cnt, xf);
  } else {
    for (int i = threadIdx.x; i < P * VV; i += LT) {
      s.k[sk_i<K>(i)] = (i < cnt) ? enc_key(g[i], xf) : key_max<K>();
      if (HV) s.v[sv_i(i)] = (i < cnt) ? gv[i] : 0xffffffffu;
    }
  }
  __syncthreads();
  if (buf != nullptr) copy_elems<K, HV, LT, VV>(g, gv, buf, bufv, cnt);
  block_sort_tile<K, HV, CNT, LT, VV>(s, cmp, P);
  if (buf != nullptr) {
    store_tile_dec<K, HV, LT, VV>(s, buf, bufv, cnt, xf);
  } else {
    store_tile_dec<K, HV, LT, VV>(s, g, gv, cnt, xf);
  }
}

// ---------------------------------------------------------------------------
// Swap-merge of one output tile.
//
// X holds sorted runs of length L (the last one may be shorter) over m
// elements; Y holds m buffer elements.  Output tile t covers Y[o0, o1) of the
// merged runs of length 2L.  The block finds its merge-path window in X
// (cooperative search in global memory), stages the A and B slices in shared
// memory, moves the buffer elements Y[o0, o1) into exactly the X slots it
// consumed, then writes the merged tile to Y.  Tiles consume disjoint X slots
// and write disjoint Y slots, so a whole level runs without inter-block
// synchronisation, and buffer elements are permuted, never overwritten.

// Warp-cooperative merge-path search over runs A[0, la) and B[0, lb) in
// global memory for diagonal d: returns the number of A elements among the
// first d outputs.  Each round the 32 lanes probe evenly spaced candidates,
// so the window shrinks 32-fold per round.
template <class K, bool CNT>
__device__ uint64_t merge_path_warp(const K* A, uint64_t la, const K* B, uint64_t lb, uint64_t d,
                                    int xf, uint64_t& cmp) {
  const unsigned lane = threadIdx.x & 31u;
  uint64_t lo = d > lb ? d - lb : 0;
  uint64_t hi = d < la ? d : la;
  // The answer lies in [lo, hi]; P(m) = (A[m] <= B[d-1-m]) holds for every m
  // below the answer and fails from the answer on.
  while (hi > lo) {
    const uint64_t span = hi - lo;
    const uint64_t step = span <= 32u ? 1 : (span + 31u) / 32u;
    const uint64_t m = lo + static_cast<uint64_t>(lane) * step;
    bool p = false;
    if (m < hi) {
      if (CNT) ++cmp;
      p = !(enc_key(B[d - 1 - m], xf) < enc_key(A[m], xf));
    }
    const int c = __popc(__ballot_sync(0xffffffffu, p));
    if (step == 1) {
      lo += static_cast<uint64_t>(c);
      break;
    }
    if (c == 0) break;  // P(lo) fails: the answer is lo
    const uint64_t nhi = lo + static_cast<uint64_t>(c) * step;
    lo = lo + static_cast<uint64_t>(c - 1) * step + 1;
    if (nhi < hi) hi = nhi;
  }
  return lo;
}

// The same search for two diagonals at once: each half-warp (16 lanes, 16
// probes per round) searches its own d over its own runs.  Every lane
// returns its half's answer.
template <class K, bool CNT>
__device__ uint64_t merge_path_halfwarp(const K* A, uint64_t la, const K* B, uint64_t lb,
                                        uint64_t d, int xf, uint64_t& cmp) {
  const unsigned lane = threadIdx.x & 31u, g = lane & 15u, half = lane >> 4;
  uint64_t lo = d > lb ? d - lb : 0;
  uint64_t hi = d < la ? d : la;
  {
    // First a round that tries the window of +-delta around the answer's
    // guess d * la / (la + lb), delta = 4 sqrt(d) + 64 (on random keys the
    // answer strays from the guess by about sqrt(d) / 2): when the guess is
    // good the 16-probe rounds start from that window, else from one side.
    const uint64_t delta = 4 * static_cast<uint64_t>(sqrtf(static_cast<float>(d))) + 64;
    const bool use = hi > lo && hi - lo > 64 * delta;
    bool p = false;
    uint64_t m1 = 0, m2 = 0;
    if (use) {
      uint64_t gs = static_cast<uint64_t>(static_cast<double>(d) * la / static_cast<double>(la + lb));
      gs = gs < lo ? lo : (gs >= hi ? hi - 1 : gs);
      m1 = gs > lo + delta ? gs - delta : lo;
      m2 = gs + delta < hi ? gs + delta : hi - 1;
      const uint64_t m = g == 0 ? m1 : m2;
      if (g < 2) {
        if (CNT) ++cmp;
        p = !(enc_key(B[d - 1 - m], xf) < enc_key(A[m], xf));
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, p) >> (half * 16u);
    if (use) {
      if (!(bal & 1u)) {
        hi = m1;
      } else if (bal & 2u) {
        lo = m2 + 1;
      } else {
        lo = m1 + 1;
        hi = m2;
      }
    }
  }
  bool done = !(hi > lo);
  while (__any_sync(0xffffffffu, !done)) {
    uint64_t step = 1;
    bool p = false;
    if (!done) {
      const uint64_t span = hi - lo;
      step = span <= 16u ? 1 : (span + 15u) / 16u;
      const uint64_t m = lo + static_cast<uint64_t>(g) * step;
      if (m < hi) {
        if (CNT) ++cmp;
        p = !(enc_key(B[d - 1 - m], xf) < enc_key(A[m], xf));
      }
    }
    const int c = __popc((__ballot_sync(0xffffffffu, p) >> (half * 16u)) & 0xffffu);
    if (!done) {
      if (step == 1) {
        lo += static_cast<uint64_t>(c);
        done = true;
      } else if (c == 0) {
        done = true;  // P(lo) fails: the answer is lo
      } else {
        const uint64_t nhi = lo + static_cast<uint64_t>(c) * step;
        lo = lo + static_cast<uint64_t>(c - 1) * step + 1;
        if (nhi < hi) hi = nhi;
        done = !(hi > lo);
      }
    }
  }
  return lo;
}

// Geometry of output tile t of a level: its run pair and diagonals.
struct MergeGeom {
  uint64_t pbase, la, lb, d0, d1;
  __device__ __forceinline__ MergeGeom(uint64_t m, uint64_t L, uint64_t t) {
    const uint64_t o0 = t * TILE;
    const uint64_t o1 = (o0 + TILE < m) ? o0 + TILE : m;
    pbase = o0 & ~(2 * L - 1);  // run lengths are powers of two
    la = (m - pbase < L) ? m - pbase : L;
    const uint64_t rem = m - pbase - la;
    lb = rem < L ? rem : L;
    d0 = o0 - pbase;
    d1 = o1 - pbase;
  }
};

// Split step of a swap-merge level: for every output tile t, the number of
// A elements of its run pair that precede the tile's first output.  Runs
// before any tile of the level moves a buffer element, so every search sees
// the unmodified runs.  One warp per tile.
template <class K, bool CNT>
__device__ void merge_split_warp(const K* keys, uint64_t X, uint64_t m, uint64_t L, uint64_t t,
                                 int xf, uint64_t* splits, uint64_t& cmp) {
  const MergeGeom g(m, L, t);
  const K* A = keys + X + g.pbase;
  const uint64_t a = (g.d0 == 0) ? 0 : merge_path_warp<K, CNT>(A, g.la, A + g.la, g.lb, g.d0, xf, cmp);
  if ((threadIdx.x & 31u) == 0) splits[t] = a;
}

// Where output tile t of a level reads and writes: its A and B slices in X
// (windows from the split step), its buffer tile in Y.
template <class K>
struct TileGeo {
  K* sa;
  K* sb;
  uint32_t* sav;
  uint32_t* sbv;
  K* yk;
  uint32_t* yv;
  int cnt, na;
};

template <class K, bool HV>
__device__ __forceinline__ TileGeo<K> tile_geo(K* keys, uint32_t* vals, uint64_t X, uint64_t Y,
                                               uint64_t m, uint64_t L, uint64_t tile,
                                               const uint64_t* splits) {
  const MergeGeom gm(m, L, tile);
  const uint64_t o0 = tile * TILE;
  const uint64_t la = gm.la;
  const uint64_t a_lo = splits[tile];
  const uint64_t a_hi = (gm.d1 == la + gm.lb) ? la : splits[tile + 1];
  const uint64_t b_lo = gm.d0 - a_lo;
  TileGeo<K> g;
  g.sa = keys + X + gm.pbase + a_lo;
  g.sb = keys + X + gm.pbase + la + b_lo;
  g.sav = HV ? vals + X + gm.pbase + a_lo : nullptr;
  g.sbv = HV ? vals + X + gm.pbase + la + b_lo : nullptr;
  g.yk = keys + Y + o0;
  g.yv = HV ? vals + Y + o0 : nullptr;
  g.cnt = static_cast<int>(gm.d1 - gm.d0);
  g.na = static_cast<int>(a_hi - a_lo);
  return g;
}

// Issues the asynchronous copies of the tile's A slice then B slice into
// shared memory (element i is copied by thread i mod NT).
template <class K, bool HV>
__device__ __forceinline__ void stage_tile(TileSmem<K, HV> s, const TileGeo<K>& g) {
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = j * NT + threadIdx.x;
    if (i < g.cnt) {
      const bool fa = i < g.na;
      cp_async_elem(&s.k[sk_i<K>(i)], fa ? g.sa + i : g.sb + (i - g.na));
      if (HV) cp_async_elem(&s.v[sv_i(i)], fa ? g.sav + i : g.sbv + (i - g.na));
    }
  }
}

// Loads the tile's buffer elements Y[o0, o1) into registers.
template <class K, bool HV>
__device__ __forceinline__ void load_y(const TileGeo<K>& g, K (&y)[V], uint32_t (&yv)[V]) {
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = j * NT + threadIdx.x;
    if (i < g.cnt) {
      y[j] = g.yk[i];
      if (HV) yv[j] = g.yv[i];
    }
  }
}

// After this thread's copies have landed: its buffer elements go into the X
// slots it copied from (so the tile's consumed slots receive exactly its
// buffer tile), and its staged keys become order keys.
template <class K, bool HV>
__device__ __forceinline__ void put_y(TileSmem<K, HV> s, const TileGeo<K>& g, const K (&y)[V],
                                      const uint32_t (&yv)[V], int xf) {
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = j * NT + threadIdx.x;
    if (i < g.cnt) {
      const bool fa = i < g.na;
      *(fa ? g.sa + i : g.sb + (i - g.na)) = y[j];
      if (HV) *(fa ? g.sav + i : g.sbv + (i - g.na)) = yv[j];
      if (xf != XF_NONE) s.k[sk_i<K>(i)] = enc_key(s.k[sk_i<K>(i)], xf);
    }
  }
}

// Merges the staged slices (thread t produces outputs [tV, tV + V)) and
// writes the merged tile to Y.  Starts after a __syncthreads that made the
// staged keys visible.
template <class K, bool HV, bool CNT>
__device__ __forceinline__ void merge_staged(TileSmem<K, HV> s, const TileGeo<K>& g, int xf,
                                             uint64_t& cmp) {
  K k[V];
  uint32_t v[V];
  int src[V];
  const int cnt = g.cnt, na = g.na, nb = cnt - na;
  const int d = threadIdx.x * V;
  const bool active = d < cnt;
  if (active) {
    const int ia = merge_path_smem<K, CNT>(s.k, 0, na, na, nb, d, cmp);
    serial_merge<K, CNT>(s.k, ia, na, na + d - ia, na + nb, k, src, cmp);
    if (HV) {
#pragma unroll
      for (int j = 0; j < V; ++j) v[j] = s.v[sv_i(src[j] < cnt ? src[j] : 0)];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int j = 0; j < V; ++j) {
      if (d + j < cnt) {
        s.k[sk_i<K>(d + j)] = k[j];
        if (HV) s.v[sv_i(d + j)] = v[j];
      }
    }
  }
  __syncthreads();
  store_tile_dec<K, HV>(s, g.yk, g.yv, cnt, xf);
}

// One output tile of a swap-merge level, unpipelined (block-scoped path).
template <class K, bool HV, bool CNT>
__device__ __forceinline__ void merge_tile(TileSmem<K, HV> s, K* keys, uint32_t* vals, uint64_t X,
                                           uint64_t Y, uint64_t m, uint64_t L, uint64_t tile,
                                           const uint64_t* splits, int xf, uint64_t& cmp) {
  const TileGeo<K> g = tile_geo<K, HV>(keys, vals, X, Y, m, L, tile, splits);
  __syncthreads();
  stage_tile<K, HV>(s, g);
  K y[V];
  uint32_t yv[V];
  load_y<K, HV>(g, y, yv);
  cp_async_wait_all();
  put_y<K, HV>(s, g, y, yv, xf);
  __syncthreads();
  merge_staged<K, HV, CNT>(s, g, xf, cmp);
}

// ---------------------------------------------------------------------------
// Partition, step 1: local partition of one tile g[0, cnt) around the order
// key piv (left = key < piv, or key <= piv when le).  Left elements are
// gathered at the front of the tile; returns their number.

template <class K, bool HV, bool CNT>
__device__ __forceinline__ uint32_t part_local_tile(TileSmem<K, HV> s, K* g, uint32_t* gv, int cnt, K piv, bool le,
                                    int xf, uint64_t& cmp) {
  K x[V];
  uint32_t y[V];
  uint32_t flags = 0, lc = 0, nc = 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = j * NT + threadIdx.x;
    if (i < cnt) {
      x[j] = g[i];
      if (HV) y[j] = gv[i];
      const K u = enc_key(x[j], xf);
      const bool l = le ? !(piv < u) : (u < piv);
      flags |= static_cast<uint32_t>(l) << j;
      lc += l;
      ++nc;
    }
  }
  if (CNT) cmp += nc;
  uint32_t tot;
  const uint32_t ex = block_excl_scan(lc | ((nc - lc) << 16), s.scratch, &tot);
  const uint32_t c = tot & 0xffffu;
  if (c == 0 || c == static_cast<uint32_t>(cnt)) return c;  // tile already partitioned
  uint32_t offL = ex & 0xffffu, offR = c + (ex >> 16);
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = j * NT + threadIdx.x;
    if (i < cnt) {
      const uint32_t dst = ((flags >> j) & 1u) ? offL++ : offR++;
      s.k[sk_i<K>(dst)] = x[j];
      if (HV) s.v[sv_i(dst)] = y[j];
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int j = 0; j < V; ++j) {
    const int i = j * NT + threadIdx.x;
    if (i < cnt) {
      g[i] = s.k[sk_i<K>(i)];
      if (HV) gv[i] = s.v[sv_i(i)];
    }
  }
  return c;
}

// Partition, step 3: exchange misplaced elements by rank.  After step 1,
// tile t = [ts, te) holds its c_t left elements first.  With s = lo + L the
// final boundary, tile t's right elements inside [lo, s) form one run
// starting at ts + c_t, and its left elements inside [s, hi) one run
// starting at max(ts, s).  pml / pmr are the exclusive prefix sums of those
// run lengths over tiles; the j-th misplaced right element is swapped with
// the j-th misplaced left element.

__device__ __forceinline__ uint32_t upper_bound_u64(const uint64_t* p, uint32_t n, uint64_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (p[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

constexpr int EXV = 4;  // ranks per thread in the exchange

template <class K, bool HV>
__device__ __forceinline__ void exchange_ranks(K* keys, uint32_t* vals, uint64_t lo, uint64_t s,
                                               const uint32_t* counts, const uint64_t* pml,
                                               const uint64_t* pmr, uint32_t ntiles, uint64_t j0,
                                               uint64_t mis) {
  uint32_t tl = upper_bound_u64(pml, ntiles + 1, j0) - 1;
  uint32_t tr = upper_bound_u64(pmr, ntiles + 1, j0) - 1;
#pragma unroll
  for (int q = 0; q < EXV; ++q) {
    const uint64_t j = j0 + q;
    if (j >= mis) break;
    while (pml[tl + 1] <= j) ++tl;
    while (pmr[tr + 1] <= j) ++tr;
    const uint64_t lts = lo + static_cast<uint64_t>(tl) * TILE;
    const uint64_t lpos = lts + counts[tl] + (j - pml[tl]);
    const uint64_t rts = lo + static_cast<uint64_t>(tr) * TILE;
    const uint64_t rpos = (rts > s ? rts : s) + (j - pmr[tr]);
    const K a = keys[lpos];
    keys[lpos] = keys[rpos];
    keys[rpos] = a;
    if (HV) {
      const uint32_t b = vals[lpos];
      vals[lpos] = vals[rpos];
      vals[rpos] = b;
    }
  }
}

// ---------------------------------------------------------------------------
// Grid-wide partition with small blocks: partition tiles of PT = 2048 keys,
// one per 128-thread block, so that many blocks per SM keep loads in flight.

constexpr int PNT = 128;        // threads per partition block
// Resident blocks per SM the local-partition kernels are built for (4-byte
// keys without payloads: 48 registers, 10 blocks).
template <class K, bool HV>
constexpr int part_minb() {
  return sizeof(K) == 4 ? (HV ? 5 : 10) : (HV ? 4 : 6);
}
constexpr int PT = PNT * V;     // keys per partition tile
constexpr int PNWARP = PNT / 32;

template <class K>
__host__ __device__ constexpr int pk_len() {
  return PT + PT / (128 / static_cast<int>(sizeof(K))) + 4;
}
__host__ __device__ constexpr int pv_len() { return PT + PT / 32 + 4; }

// Exclusive scan over the PNT threads of a partition block (scratch: PNWARP + 1).
__device__ __forceinline__ uint32_t pblock_excl_scan(uint32_t x, uint32_t* scratch, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(x);
  if (lane == 31) scratch[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t s = lane < PNWARP ? scratch[lane] : 0u;
    const uint32_t si = warp_incl_scan(s);
    if (lane < PNWARP) scratch[lane] = si - s;
    if (lane == 31) scratch[PNWARP] = si;
  }
  __syncthreads();
  const uint32_t r = scratch[w] + inc - x;
  *total = scratch[PNWARP];
  __syncthreads();
  return r;
}

// Local partition of one partition tile g[0, cnt) (cnt <= PT): left keys
// (key < piv, or key <= piv when le) gathered at the front; returns their
// number.  Shared: sk (pk_len), sv (pv_len), scratch (PNWARP + 1 words).
// FULL: cnt == PT (every tile but a range's last), no per-element bound
// checks.
template <class K, bool HV, bool CNT, bool FULL = false>
__device__ __forceinline__ uint32_t part_local_small(K* g, uint32_t* gv, int cnt, K piv, bool le,
                                                     int xf, K* sk, uint32_t* sv, uint32_t* scratch,
                                                     uint64_t& cmp) {
  K x[V];
  uint32_t y[V];
  uint32_t flags = 0, lc = 0, nc = 0;
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = j * PNT + threadIdx.x;
    if (FULL || i < cnt) {
      x[j] = g[i];
      if (HV) y[j] = gv[i];
    }
  }
  with_xf<K>(xf, [&](auto xc) {
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int i = j * PNT + threadIdx.x;
      if (FULL || i < cnt) {
        const K u = enc_key(x[j], xc);
        const bool l = le ? !(piv < u) : (u < piv);
        flags |= static_cast<uint32_t>(l) << j;
        lc += l;
        if (!FULL) ++nc;
      }
    }
  });
  if (FULL) nc = V;
  if (CNT) cmp += nc;
  uint32_t tot;
  const uint32_t ex = pblock_excl_scan(lc | ((nc - lc) << 16), scratch, &tot);
  const uint32_t c = tot & 0xffffu;
  if (c == 0 || c == static_cast<uint32_t>(cnt)) return c;  // already partitioned
  uint32_t offL = ex & 0xffffu, offR = c + (ex >> 16);
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = j * PNT + threadIdx.x;
    if (FULL || i < cnt) {
      const uint32_t dst = ((flags >> j) & 1u) ? offL++ : offR++;
      sk[sk_i<K>(dst)] = x[j];
      if (HV) sv[sv_i(dst)] = y[j];
    }
  }
  __syncthreads();
  // element j * PNT + t sits at padded index j * (PNT + PNT / PE) + pad(t)
  constexpr int PE = 128 / static_cast<int>(sizeof(K));
  const int pt = static_cast<int>(threadIdx.x) + static_cast<int>(threadIdx.x) / PE;
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const int i = j * PNT + threadIdx.x;
    if (FULL || i < cnt) {
      g[i] = sk[pt + j * (PNT + PNT / PE)];
      if (HV) gv[i] = sv[sv_i(i)];
    }
  }
  return c;
}

// Exchange of misplaced keys (step 3 of the partition, tiles of PT keys):
// warp w handles ranks [jw, jw + 32 * EXW); one lane finds the chunk's first
// tile on each side, then lane l swaps ranks jw + l + 32k (consecutive lanes,
// consecutive positions inside a run), walking its tiles forward.
constexpr int EXW = 16;                // ranks per lane
constexpr uint64_t EXJ = 32ull * EXW;  // ranks per warp
constexpr int EXB = 128;               // threads per exchange block (several blocks per SM)


// Swaps the misplaced pairs of ranks [jw, jw + EXJ) (jw a multiple of EXJ).
// wtl/wtr give, per warp, the tile holding its first left / right rank.
// Positions are kept relative to lo in type P: 32 bits whenever the range
// is shorter than 2^32 (half the registers of 64-bit positions, so more
// warps stay resident), 64 bits otherwise.
template <class K, bool HV, class P = uint32_t>
__device__ __forceinline__ void exchange_warp(K* keys, uint32_t* vals, uint64_t lo, uint64_t s,
                                              const uint32_t* counts, const uint64_t* pml,
                                              const uint64_t* pmr, const uint32_t* wtl,
                                              const uint32_t* wtr, uint64_t jw, uint64_t mis) {
  const unsigned lane = threadIdx.x & 31u;
  K* kb = keys + lo;
  uint32_t* vb = HV ? vals + lo : nullptr;
  const P sr = static_cast<P>(s - lo);
  uint32_t tl = wtl[jw / EXJ], tr = wtr[jw / EXJ];
  // Positions first (walking the tiles with their bounds kept in registers),
  // then all loads, then all stores: a lane keeps 2 * EXW loads in flight.
  uint64_t l_lo = pml[tl], l_hi = pml[tl + 1];
  P l_base = static_cast<P>(tl) * PT + counts[tl];
  uint64_t r_lo = pmr[tr], r_hi = pmr[tr + 1];
  P r_base = static_cast<P>(tr) * PT;
  if (r_base < sr) r_base = sr;
  // this lane's ranks jw + lane + 32 q exist for q < nq
  const uint64_t left = mis - jw;
  const uint64_t nq64 = left > lane ? (left - lane + 31) / 32 : 0;
  const int nq = nq64 < static_cast<uint64_t>(EXW) ? static_cast<int>(nq64) : EXW;
  P lp[EXW], rp[EXW];
#pragma unroll
  for (int q = 0; q < EXW; ++q) {
    const uint64_t j = jw + lane + 32u * q;
    if (q < nq) {
      while (j >= l_hi) {
        ++tl;
        l_lo = l_hi;
        l_hi = pml[tl + 1];
        l_base = static_cast<P>(tl) * PT + counts[tl];
      }
      while (j >= r_hi) {
        ++tr;
        r_lo = r_hi;
        r_hi = pmr[tr + 1];
        r_base = static_cast<P>(tr) * PT;
        if (r_base < sr) r_base = sr;
      }
      lp[q] = l_base + static_cast<P>(j - l_lo);
      rp[q] = r_base + static_cast<P>(j - r_lo);
    }
  }
  K a[EXW], b[EXW];
  uint32_t va[EXW], vb2[EXW];
#pragma unroll
  for (int q = 0; q < EXW; ++q) {
    if (q < nq) {
      a[q] = kb[lp[q]];
      b[q] = kb[rp[q]];
      if (HV) {
        va[q] = vb[lp[q]];
        vb2[q] = vb[rp[q]];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < EXW; ++q) {
    if (q < nq) {
      kb[lp[q]] = b[q];
      kb[rp[q]] = a[q];
      if (HV) {
        vb[lp[q]] = vb2[q];
        vb[rp[q]] = va[q];
      }
    }
  }
}

}  // namespace qms
