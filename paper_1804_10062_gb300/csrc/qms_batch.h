// Internal interface between the library's translation units: the batched
// form's group kernels (qms_batch.cu) and the host code that plans and
// launches them (qms_lib.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace qms {

struct Desc;

// Kernel configurations of the batched form, one per way of sorting a
// segment: a group of GT threads with VV keys each sorts a segment of at
// most GT * VV keys in shared memory (the base case), or one block runs the
// QuickMergesort rounds of a longer segment (BC_QMS).
enum BatchCfg : int {
  BC_G32 = 0,   // one warp, 16 keys per thread: segments up to 512 keys
  BC_G64,       // 64 threads x 16: up to 1024
  BC_G128,      // 128 x 16: up to 2048
  BC_G256,      // 256 x 16: up to 4096
  BC_G512,      // 512 x 16: up to 8192
  BC_G256W,     // 256 x 32: up to 8192 (4-byte keys without payloads)
  BC_G512W,     // 512 x 32: up to 16384 (4-byte keys without payloads)
  BC_QMS,       // one block per segment, QuickMergesort rounds (any length)
  BC_G1024W,    // 1024 x 32: up to 32768 (4-byte keys without payloads)
  BC_PAIR,      // a cluster of two 1024 x 32 blocks: up to 65536 (4-byte keys, no payloads)
  BC_COUNT
};

// Length bins: bin b holds the segments of (2^(b-1), 2^b] keys, b <= 16;
// longer segments always take BC_QMS (or the grid driver).
constexpr int BATCH_BINS = 17;

int batch_cfg_threads(int c);
int batch_cfg_keys_per_thread(int c);
inline int batch_cfg_capacity(int c) {
  return c == BC_QMS ? (1 << 30)
                     : batch_cfg_threads(c) * batch_cfg_keys_per_thread(c) * (c == BC_PAIR ? 2 : 1);
}
// Whether configuration c exists for keys of ksize bytes (with payloads: hv).
inline bool batch_cfg_valid(int c, int ksize, bool hv) {
  if (c < 0 || c >= BC_COUNT) return false;
  if (c == BC_G256W || c == BC_G512W || c == BC_G1024W || c == BC_PAIR) return ksize == 4 && !hv;
  return true;
}
const char* batch_cfg_name(int c);

// Launches the group kernel of configuration c (c != BC_QMS) over the
// segments order[0, nseg) of keys (offsets: nseg + 1 device offsets).
cudaError_t launch_group_cfg(int c, int ksize, bool hv, bool cnt, void* keys, uint32_t* vals,
                             const uint64_t* offsets, const uint32_t* order, uint32_t nseg,
                             unsigned int* ticket, int xf, Desc* desc, cudaStream_t st);

}  // namespace qms
