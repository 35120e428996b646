// Batched form, short segments: thread groups of GT threads (GT a power of
// two, 32 = one warp, up to one 1024-thread block) each sort one segment of
// at most GT * VV keys by themselves, entirely in shared memory.  A segment
// that short is finished by QuickMergesort's base case (the driver loop of
// Fig. 3, arXiv 1804.10062, never partitions a range of one leaf tile or
// less): a sorting network on the VV keys each thread holds, then
// merge-path rounds in shared memory.  Several groups share a block, so a
// warp-sized segment occupies one warp, not a whole block.  Which group
// size serves which length is chosen per length bin by the autotuner
// (qms_batched_autotune).
#pragma once

#include <cooperative_groups.h>

#include "qms_kernels.cuh"

namespace qms {

// Threads of a block of groups of GT threads: NT, or one group of GT > NT.
__host__ __device__ constexpr int group_block_threads(int GT) { return GT > NT ? GT : NT; }

// Barrier of the GT threads of group g of a block: the warp for GT = 32,
// named barrier 1 + g otherwise (at most 8 groups of at least 64 threads in
// a 512-thread block, so ids 1..8; id 0 is __syncthreads).
template <int GT>
__device__ __forceinline__ void group_sync(int g) {
  if (GT <= 32) {
    __syncwarp();
  } else if (GT >= NT) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(GT) : "memory");
  }
}

template <class K, bool HV, int GT, int VV>
__host__ __device__ constexpr size_t group_smem_bytes() {
  return (static_cast<size_t>(sk_len<K, GT, VV>()) * sizeof(K) +
          (HV ? static_cast<size_t>(sv_len<GT, VV>()) * 4 : 0) + 15) / 16 * 16;
}

// Sorts g[0, cnt), cnt <= GT * VV, by the group whose thread lt this is;
// sk / sv: the group's shared-memory tile.  Every thread of the group calls
// it with the same cnt.
template <class K, bool HV, bool CNT, int GT, int VV>
__device__ __forceinline__ void group_sort_seg(K* g, uint32_t* gv, int cnt, K* sk, uint32_t* sv,
                                               int lt, int grp, int xf, uint64_t& cmp) {
  int P = 1;
  while (P * VV < cnt) P <<= 1;  // threads holding data
  for (int i = lt; i < P * VV; i += GT) {
    sk[sk_i<K>(i)] = (i < cnt) ? enc_key(g[i], xf) : key_max<K>();
    if (HV) sv[sv_i(i)] = (i < cnt) ? gv[i] : 0xffffffffu;
  }
  group_sync<GT>(grp);
  if constexpr (!HV) {
    // run pairs of at most 32 threads lie within one warp
    tile_sort_keys<K, CNT, VV>(
        sk, lt, P,
        [grp](int t) {
          if (t <= 32)
            __syncwarp();
          else
            group_sync<GT>(grp);
        },
        cmp);
    group_sync<GT>(grp);  // the last round's writes are visible
  } else {
    K k[VV];
    uint32_t v[VV];
    if (lt < P) {
#pragma unroll
      for (int j = 0; j < VV; ++j) {
        k[j] = sk[sk_i<K>(lt * VV + j)];
        if (HV) v[j] = sv[sv_i(lt * VV + j)];
      }
      net_sort<K, HV, VV>(k, v);
      if (CNT) cmp += kNet<VV>.len;
#pragma unroll
      for (int j = 0; j < VV; ++j) {
        sk[sk_i<K>(lt * VV + j)] = k[j];
        if (HV) sv[sv_i(lt * VV + j)] = v[j];
      }
    }
    group_sync<GT>(grp);
    for (int sp = 1; sp < P; sp <<= 1) {
      const int L = sp * VV;
      const int pr = lt / (2 * sp), r = lt - pr * 2 * sp;
      const int a0 = pr * 2 * L, b0 = a0 + L;
      const int d = r * VV;
      if (lt < P) {
        const int ia = merge_path_smem<K, CNT>(sk, a0, L, b0, L, d, cmp);
        serial_merge_kv<K, HV, CNT, VV>(sk, sv, a0 + ia, a0 + L, b0 + d - ia, b0 + L, k, v, cmp);
      }
      group_sync<GT>(grp);  // every read of the round is done before any write
      if (lt < P) {
#pragma unroll
        for (int j = 0; j < VV; ++j) {
          sk[sk_i<K>(a0 + d + j)] = k[j];
          if (HV) sv[sv_i(a0 + d + j)] = v[j];
        }
      }
      group_sync<GT>(grp);
    }
  }
  for (int i = lt; i < cnt; i += GT) {
    g[i] = dec_key(sk[sk_i<K>(i)], xf);
    if (HV) gv[i] = sv[sv_i(i)];
  }
  group_sync<GT>(grp);  // the tile is free for the group's next segment
}

// One launch per length bin: groups take segments order[0, nseg) from an
// atomic ticket (the host lists a bin's segments longest first).
template <class K, bool HV, bool CNT, int GT, int VV>
__global__ void __launch_bounds__(group_block_threads(GT))
    k_batched_group(K* keys, uint32_t* vals, const uint64_t* offsets, const uint32_t* order,
                    uint32_t nseg, unsigned int* ticket, int xf, Desc* desc) {
  constexpr int NG = group_block_threads(GT) / GT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t gseg[NG];
  const int grp = threadIdx.x / GT, lt = threadIdx.x % GT;
  unsigned char* base = smem + grp * group_smem_bytes<K, HV, GT, VV>();
  K* sk = reinterpret_cast<K*>(base);
  uint32_t* sv = HV ? reinterpret_cast<uint32_t*>(base + sk_len<K, GT, VV>() * sizeof(K)) : nullptr;
  uint64_t cmp = 0;
  while (true) {
    if (lt == 0) gseg[grp] = atomicAdd(ticket, 1u);
    group_sync<GT>(grp);
    const uint32_t t = gseg[grp];
    group_sync<GT>(grp);  // read by all before the next ticket overwrites it
    if (t >= nseg) break;
    const uint32_t sg = order[t];
    const uint64_t b = offsets[sg];
    const int cnt = static_cast<int>(offsets[sg + 1] - b);
    if (cnt > 1)
      group_sort_seg<K, HV, CNT, GT, VV>(keys + b, HV ? vals + b : nullptr, cnt, sk, sv, lt, grp, xf,
                                         cmp);
  }
  if (CNT) flush_count(cmp, &desc->cmp);
}

// Segments of (PH, 2 PH] keys, PH = 32768, 4-byte keys without payloads:
// a cluster of two 1024-thread blocks.  Block r sorts part r of the segment
// (its first PH keys, or the rest) in its own shared memory with the base
// case; then every thread merges 32 outputs of the whole segment, reading
// both sorted parts through distributed shared memory (block r produces
// outputs [r PH, r PH + PH)), and the block writes its outputs back.  Rank
// 0 takes the segment from the ticket.  Both blocks pass every cluster
// barrier the same number of times: they read the same ticket value and
// leave the loop together, and meet once more before either exits.
constexpr int PAIR_T = 1024;           // threads per block
constexpr int PAIR_VV = 2 * V;         // keys per thread
constexpr int PAIR_H = PAIR_T * PAIR_VV;  // keys per block (32768)

template <class K, bool CNT>
__global__ void __launch_bounds__(PAIR_T, 1)
    k_batched_pair(K* keys, const uint64_t* offsets, const uint32_t* order, uint32_t nseg,
                   unsigned int* ticket, int xf, Desc* desc) {
  static_assert(sizeof(K) == 4, "4-byte keys");
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t seg_t;
  K* sk = reinterpret_cast<K*>(smem);
  const unsigned rank = cluster.block_rank();
  const int tid = threadIdx.x;
  uint64_t cmp = 0;
  while (true) {
    if (rank == 0 && tid == 0) seg_t = atomicAdd(ticket, 1u);
    cluster.sync();
    const uint32_t t = *cluster.map_shared_rank(&seg_t, 0);
    if (t >= nseg) break;  // both blocks read the same t
    const uint32_t sg = order[t];
    const uint64_t b = offsets[sg];
    const int n = static_cast<int>(offsets[sg + 1] - b);
    const int la = n < PAIR_H ? n : PAIR_H;  // part 0
    const int lb = n - la;                   // part 1
    const int cnt = rank == 0 ? la : lb;
    K* g = keys + b + (rank == 0 ? 0 : PAIR_H);
    int P = 1;
    while (P * PAIR_VV < cnt) P <<= 1;
    for (int i = tid; i < P * PAIR_VV; i += PAIR_T) sk[sk_i<K>(i)] = i < cnt ? enc_key(g[i], xf) : key_max<K>();
    __syncthreads();
    tile_sort_keys<K, CNT, PAIR_VV>(sk, tid, P, [](int th) { tile_sync<PAIR_T>(th); }, cmp);
    cluster.sync();  // both parts sorted and visible to the cluster
    // merge outputs [d, d + VV) of the segment: A = part 0, B = part 1
    const int d = static_cast<int>(rank) * PAIR_H + tid * PAIR_VV;
    K k[PAIR_VV];
    if (d < n) {
      const K* sA = cluster.map_shared_rank(sk, 0);
      const K* sB = cluster.map_shared_rank(sk, 1);
      int lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (CNT) ++cmp;
        if (!(sB[sk_i<K>(d - 1 - mid)] < sA[sk_i<K>(mid)])) lo = mid + 1; else hi = mid;
      }
      int ai = lo, bi = d - lo;
      K ka = ai < la ? sA[sk_i<K>(ai)] : key_max<K>();
      K kb = bi < lb ? sB[sk_i<K>(bi)] : key_max<K>();
#pragma unroll
      for (int j = 0; j < PAIR_VV; ++j) {
        const bool a_ok = ai < la, b_ok = bi < lb;
        if (CNT && a_ok && b_ok) ++cmp;
        const bool tb = b_ok && (!a_ok || kb < ka);
        k[j] = tb ? kb : ka;
        if (tb) {
          ++bi;
          kb = bi < lb ? sB[sk_i<K>(bi)] : key_max<K>();
        } else {
          ++ai;
          ka = ai < la ? sA[sk_i<K>(ai)] : key_max<K>();
        }
      }
    }
    cluster.sync();  // every read of both parts is done
    if (d < n) {
      const int base = sk_i<K>(tid * PAIR_VV);
#pragma unroll
      for (int j = 0; j < PAIR_VV; ++j) sk[base + j] = k[j];
    }
    __syncthreads();
    const int outn = rank == 0 ? la : lb;
    for (int i = tid; i < outn; i += PAIR_T) g[i] = dec_key(sk[sk_i<K>(i)], xf);
    __syncthreads();  // the tile is free for the next segment
  }
  // Rank 1 has read the last ticket from rank 0's shared memory before
  // rank 0 may exit.
  cluster.sync();
  if (CNT) flush_count(cmp, &desc->cmp);
}

}  // namespace qms
