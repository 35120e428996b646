// Group kernels of the batched form (see qms_batch.cuh), in a translation
// unit of their own so that they compile beside the rest of the library.

#include "qms_batch.cuh"
#include "qms_batch.h"
#include "qms_host.h"

namespace qms {

int batch_cfg_threads(int c) {
  static const int t[BC_COUNT] = {32, 64, 128, 256, 512, 256, 512, NT, 1024, 1024};
  return (c >= 0 && c < BC_COUNT) ? t[c] : 0;
}
int batch_cfg_keys_per_thread(int c) {
  static const int v[BC_COUNT] = {V, V, V, V, V, 2 * V, 2 * V, V, 2 * V, 2 * V};
  return (c >= 0 && c < BC_COUNT) ? v[c] : 0;
}
const char* batch_cfg_name(int c) {
  static const char* n[BC_COUNT] = {"group32x16", "group64x16", "group128x16", "group256x16",
                                    "group512x16", "group256x32", "group512x32", "block_qms",
                                    "group1024x32", "pair1024x32"};
  return (c >= 0 && c < BC_COUNT) ? n[c] : "invalid";
}

namespace {

template <class K, bool HV, bool CNT, int GT, int VV>
cudaError_t launch_one(void* keys, uint32_t* vals, const uint64_t* offsets, const uint32_t* order,
                       uint32_t nseg, unsigned int* ticket, int xf, Desc* desc, cudaStream_t st) {
  constexpr int BT = group_block_threads(GT);
  constexpr size_t smem = group_smem_bytes<K, HV, GT, VV>() * (BT / GT);
  auto f = k_batched_group<K, HV, CNT, GT, VV>;
  cudaError_t e = smem_attr(reinterpret_cast<const void*>(f), smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, BT, smem)) != cudaSuccess) return e;
  const uint64_t groups = (nseg + (BT / GT) - 1) / (BT / GT);
  const uint64_t resident = static_cast<uint64_t>(sms) * (occ > 0 ? occ : 1);
  const unsigned grid = static_cast<unsigned>(groups < resident ? (groups > 0 ? groups : 1) : resident);
  f<<<grid, BT, smem, st>>>(static_cast<K*>(keys), vals, offsets, order, nseg, ticket, xf, desc);
  return cudaGetLastError();
}

// The two-block cluster configuration: as many clusters as fit the GPU at
// once (at most one per two segments' worth of work), each looping over
// segments from the ticket.
template <class K, bool CNT>
cudaError_t launch_pair(void* keys, const uint64_t* offsets, const uint32_t* order, uint32_t nseg,
                        unsigned int* ticket, int xf, Desc* desc, cudaStream_t st) {
  constexpr size_t smem = group_smem_bytes<K, false, PAIR_T, PAIR_VV>();
  auto f = k_batched_pair<K, CNT>;
  cudaError_t e = smem_attr(reinterpret_cast<const void*>(f), smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(PAIR_T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  cfg.gridDim = dim3(2);
  if ((e = cudaOccupancyMaxActiveClusters(&clusters, f, &cfg)) != cudaSuccess) return e;
  if (clusters < 1) return cudaErrorInvalidConfiguration;
  const unsigned nc = nseg < static_cast<uint32_t>(clusters) ? nseg : static_cast<unsigned>(clusters);
  cfg.gridDim = dim3(2 * nc);
  return cudaLaunchKernelEx(&cfg, f, static_cast<K*>(keys), offsets, order, nseg, ticket, xf, desc);
}

template <class K, bool HV, bool CNT>
cudaError_t launch_typed(int c, void* keys, uint32_t* vals, const uint64_t* offsets,
                         const uint32_t* order, uint32_t nseg, unsigned int* ticket, int xf,
                         Desc* desc, cudaStream_t st) {
  switch (c) {
    case BC_G32: return launch_one<K, HV, CNT, 32, V>(keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    case BC_G64: return launch_one<K, HV, CNT, 64, V>(keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    case BC_G128: return launch_one<K, HV, CNT, 128, V>(keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    case BC_G256: return launch_one<K, HV, CNT, 256, V>(keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    case BC_G512: return launch_one<K, HV, CNT, 512, V>(keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    default: break;
  }
  if constexpr (sizeof(K) == 4 && !HV) {
    if (c == BC_G256W)
      return launch_one<K, HV, CNT, 256, 2 * V>(keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    if (c == BC_G512W)
      return launch_one<K, HV, CNT, 512, 2 * V>(keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    if (c == BC_G1024W)
      return launch_one<K, HV, CNT, 1024, 2 * V>(keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    if (c == BC_PAIR) return launch_pair<K, CNT>(keys, offsets, order, nseg, ticket, xf, desc, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_group_cfg(int c, int ksize, bool hv, bool cnt, void* keys, uint32_t* vals,
                             const uint64_t* offsets, const uint32_t* order, uint32_t nseg,
                             unsigned int* ticket, int xf, Desc* desc, cudaStream_t st) {
  if (nseg == 0) return cudaSuccess;
  if (ksize == 8) {
    if (hv) return cnt ? launch_typed<uint64_t, true, true>(c, keys, vals, offsets, order, nseg, ticket, xf, desc, st)
                       : launch_typed<uint64_t, true, false>(c, keys, vals, offsets, order, nseg, ticket, xf, desc, st);
    return cnt ? launch_typed<uint64_t, false, true>(c, keys, vals, offsets, order, nseg, ticket, xf, desc, st)
               : launch_typed<uint64_t, false, false>(c, keys, vals, offsets, order, nseg, ticket, xf, desc, st);
  }
  if (hv) return cnt ? launch_typed<uint32_t, true, true>(c, keys, vals, offsets, order, nseg, ticket, xf, desc, st)
                     : launch_typed<uint32_t, true, false>(c, keys, vals, offsets, order, nseg, ticket, xf, desc, st);
  return cnt ? launch_typed<uint32_t, false, true>(c, keys, vals, offsets, order, nseg, ticket, xf, desc, st)
             : launch_typed<uint32_t, false, false>(c, keys, vals, offsets, order, nseg, ticket, xf, desc, st);
}

}  // namespace qms
