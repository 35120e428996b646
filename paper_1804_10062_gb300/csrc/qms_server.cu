// Served form of the GB300 QuickMergesort library: a request server with
// continuous batching (include/qms.h, qms_server_*).
//
// Requests (sort n keys of one dtype) arrive at any time.  Each is admitted
// against a device-memory budget (the bytes the server itself holds for it:
// a device slot for its keys unless the keys already are a device array
// sorted in place, plus the sort's O(n/8192 + 1)-word workspace) and a
// maximum number of admitted requests.  Admission is in arrival order.
// Worker threads, each with its own CUDA stream, take admitted work:
//   - a request longer than one block's limit runs alone through qms_sort
//     (the grid-wide rounds);
//   - otherwise the worker gathers every admissible short request at the head
//     of the queue with the same key width and sorts them together in one
//     persistent launch (one block per request, longest first).
// Workers run concurrently, so requests that arrive while others are on the
// GPU are admitted as memory frees up and their work overlaps on the device.
// Every result is that request's sort alone: requests never share memory.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/qms.h"
#include "qms_cta.cuh"
#include "qms_host.h"

namespace qms {
namespace {

using Clock = std::chrono::steady_clock;

inline double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

inline size_t r256(size_t x) { return (x + 255) / 256 * 256; }

inline size_t key_bytes(int dtype) { return (dtype == QMS_U64 || dtype == QMS_I64) ? 8 : 4; }

inline int xform(int dtype) {
  return dtype == QMS_F32 ? XF_F32 : (dtype == QMS_I64 ? XF_I64 : XF_NONE);
}

constexpr uint64_t kShortMax = static_cast<uint64_t>(CTA_MAX_TILES) * TILE;

struct Req {
  uint64_t id = 0;
  const void* in = nullptr;
  void* out = nullptr;
  uint64_t n = 0;
  int dtype = 0;
  int pivot = 0;
  bool in_place = false;  // in == out is a device array: sorted where it is
  size_t bytes = 0;       // budget charge
  void* slot = nullptr;   // device copy of the keys (not in place)
  cudaEvent_t ready = nullptr;  // recorded once the keys are in the slot
  int rc = QMS_OK;
  bool done = false;
  int batch = 0;
  Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace
}  // namespace qms

struct qms_server {
  size_t budget = 0;
  int max_slots = 0;
  int max_batch = 0;
  int device = 0;
  cudaMemPool_t pool = nullptr;  // the slots' memory pool (keeps up to the budget)
  std::mutex mu;
  std::condition_variable cv_work, cv_ready, cv_done;
  std::deque<qms::Req*> pending;  // submitted, not admitted yet
  std::deque<qms::Req*> ready;    // admitted: slot held, keys staged or on their way
  std::unordered_map<uint64_t, qms::Req*> reqs;
  uint64_t next_id = 1;
  size_t used = 0, peak_used = 0;
  int in_flight = 0, peak_in_flight = 0;
  uint64_t completed = 0, keys_done = 0, batches = 0, batched_reqs = 0;
  bool stop = false;
  bool paused = false;
  bool staging_done = false;
  std::thread stager;
  std::vector<std::thread> workers;
};

namespace qms {
namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool fits(const qms_server* S, const Req* r) {
  return S->in_flight < S->max_slots && S->used + r->bytes <= S->budget;
}

void admit(qms_server* S, Req* r) {
  S->used += r->bytes;
  S->peak_used = std::max(S->peak_used, S->used);
  ++S->in_flight;
  S->peak_in_flight = std::max(S->peak_in_flight, S->in_flight);
  r->t_admit = Clock::now();
}

// Sorts one long request alone through the grid-wide driver, in its slot.
int run_long(Req* r, cudaStream_t st) {
  qms_options opt{};
  opt.pivot = r->pivot;
  return qms_sort(r->in_place ? r->out : r->slot, r->n, r->dtype, &opt, st, nullptr);
}

template <class K>
int run_group_typed(std::vector<Req*>& g, cudaStream_t st, int pivot) {
  // One allocation: Desc + ticket, then the segment descriptors; the keys
  // are in the requests' slots (or in place).
  const size_t hdr = r256(sizeof(Desc)) + 256;
  const size_t total = hdr + r256(g.size() * sizeof(SegDesc));
  unsigned char* base = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&base), total, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return QMS_ENOMEM;
  }
  int rc = QMS_OK;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == QMS_OK) rc = QMS_ECUDA;
  };
  Desc* desc = reinterpret_cast<Desc*>(base);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(base + r256(sizeof(Desc)));
  SegDesc* segs = reinterpret_cast<SegDesc*>(base + hdr);
  // Longest first.
  std::vector<size_t> ord(g.size());
  for (size_t i = 0; i < g.size(); ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return g[a]->n > g[b]->n; });
  std::vector<SegDesc> hs(g.size());
  for (size_t j = 0; j < ord.size(); ++j) {
    Req* r = g[ord[j]];
    hs[j] = SegDesc{r->in_place ? r->out : r->slot, r->n, xform(r->dtype), 0};
  }
  ok(cudaMemsetAsync(base, 0, hdr, st));
  ok(cudaMemcpyAsync(segs, hs.data(), hs.size() * sizeof(SegDesc), cudaMemcpyHostToDevice, st));
  ok(smem_attr(reinterpret_cast<const void*>(k_batched_ptrs<K, false>), cta_smem_bytes<K, false>()));
  int dev = 0, sms = 0, occ = 0;
  ok(cudaGetDevice(&dev));
  ok(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched_ptrs<K, false>, NT,
                                                   cta_smem_bytes<K, false>()));
  const unsigned grid = static_cast<unsigned>(std::max<size_t>(
      1, std::min<size_t>(g.size(), static_cast<size_t>(sms) * std::max(occ, 1))));
  if (rc == QMS_OK) {
    k_batched_ptrs<K, false><<<grid, NT, cta_smem_bytes<K, false>(), st>>>(
        segs, static_cast<uint32_t>(g.size()), ticket, pivot, desc);
    ok(cudaGetLastError());
  }
  unsigned err = 0;
  ok(cudaMemcpyAsync(&err, &desc->err, sizeof(err), cudaMemcpyDeviceToHost, st));
  cudaFreeAsync(base, st);
  ok(cudaStreamSynchronize(st));
  if (err && rc == QMS_OK) rc = QMS_EINTERNAL;
  return rc;
}

// Admission and staging, in arrival order: a request is admitted once its
// bytes fit the budget (and a slot count is free); its device slot is
// allocated and its keys start their upload at once, so admitted requests
// hold their share of the budget while they wait for a worker, and uploads
// overlap the sorts of earlier requests.
void stager_loop(qms_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    st = nullptr;
  }
  while (true) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        return (S->stop && S->pending.empty()) ||
               (!S->paused && !S->pending.empty() && fits(S, S->pending.front()));
      });
      if (S->pending.empty()) break;  // stopping and drained
      r = S->pending.front();
      S->pending.pop_front();
      admit(S, r);
    }
    int rc = QMS_OK;
    if (!r->in_place) {
      const size_t kb = r->n * key_bytes(r->dtype);
      if ((S->pool ? cudaMallocFromPoolAsync(&r->slot, kb, S->pool, st)
                   : cudaMallocAsync(&r->slot, kb, st)) != cudaSuccess) {
        (void)cudaGetLastError();
        r->slot = nullptr;
        rc = QMS_ENOMEM;
      } else if (cudaMemcpyAsync(r->slot, r->in, kb, cudaMemcpyDefault, st) != cudaSuccess) {
        (void)cudaGetLastError();
        rc = QMS_ECUDA;
      }
    }
    if (rc == QMS_OK && (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventRecord(r->ready, st) != cudaSuccess)) {
      (void)cudaGetLastError();
      rc = QMS_ECUDA;
    }
    r->rc = rc;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->ready.push_back(r);
    }
    S->cv_ready.notify_one();
  }
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->staging_done = true;
  }
  S->cv_ready.notify_all();
}

// Workers take admitted requests in order: a request longer than
// kShortMax keys runs alone through the grid-wide rounds; shorter ones
// waiting at the head are sorted together in one launch (one block each).
void worker_loop(qms_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    st = nullptr;
  }
  while (true) {
    std::vector<Req*> g;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_ready.wait(lk, [&] {
        return (!S->paused && !S->ready.empty()) || (S->staging_done && S->ready.empty());
      });
      if (S->ready.empty()) break;  // staging finished and everything sorted
      Req* h = S->ready.front();
      S->ready.pop_front();
      g.push_back(h);
      if (h->n <= kShortMax && h->rc == QMS_OK) {
        // Continuous batching: every admitted short request of the same key
        // width waiting behind the head joins this launch.
        while (!S->ready.empty() && static_cast<int>(g.size()) < S->max_batch) {
          Req* r = S->ready.front();
          if (r->n > kShortMax || key_bytes(r->dtype) != key_bytes(h->dtype) || r->rc != QMS_OK) break;
          S->ready.pop_front();
          g.push_back(r);
        }
      }
      if (!S->ready.empty()) S->cv_ready.notify_one();
    }
    for (Req* r : g)
      if (r->ready) cudaStreamWaitEvent(st, r->ready, 0);  // its keys are in the slot
    int rc = g[0]->rc;
    if (rc == QMS_OK) {
      if (g.size() == 1 && g[0]->n > kShortMax) {
        rc = run_long(g[0], st);
      } else {
        rc = key_bytes(g[0]->dtype) == 8 ? run_group_typed<uint64_t>(g, st, g[0]->pivot)
                                         : run_group_typed<uint32_t>(g, st, g[0]->pivot);
      }
    }
    for (Req* r : g) {
      if (r->in_place || r->slot == nullptr) continue;
      if (rc == QMS_OK &&
          cudaMemcpyAsync(r->out, r->slot, r->n * key_bytes(r->dtype), cudaMemcpyDefault, st) != cudaSuccess) {
        (void)cudaGetLastError();
        rc = QMS_ECUDA;
      }
      cudaFreeAsync(r->slot, st);
      r->slot = nullptr;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == QMS_OK) rc = QMS_ECUDA;
    for (Req* r : g) {
      if (r->ready) cudaEventDestroy(r->ready);
      r->ready = nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const auto now = Clock::now();
      for (Req* r : g) {
        r->rc = rc;
        r->done = true;
        r->t_done = now;
        r->batch = static_cast<int>(g.size());
        S->used -= r->bytes;
        --S->in_flight;
        ++S->completed;
        S->keys_done += r->n;
      }
      if (g.size() > 1 || g[0]->n <= kShortMax) {
        ++S->batches;
        S->batched_reqs += g.size();
      }
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

void fill_info(const Req* r, qms_request_info* info) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->status = r->rc;
  info->n = r->n;
  info->batch_size = r->batch;
  info->queue_ms = ms_since(r->t_submit, r->t_admit);
  info->latency_ms = ms_since(r->t_submit, r->t_done);
}

}  // namespace
}  // namespace qms

using namespace qms;

extern "C" {

int qms_server_create(size_t hbm_budget_bytes, int max_slots, int workers, int max_batch,
                      qms_server** out) {
  if (out == nullptr || hbm_budget_bytes == 0 || max_slots < 1 || workers < 1 || workers > 64 ||
      max_batch < 1)
    return QMS_EINVAL;
  *out = nullptr;
  auto* S = new (std::nothrow) qms_server();
  if (!S) return QMS_ENOMEM;
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  S->max_batch = max_batch;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete S;
    return QMS_ECUDA;
  }
  // The slots come from a pool of the server's own that keeps up to the
  // budget mapped: slots freed by the workers are reused by the stager
  // without mapping device memory again.  (Without a pool: the device's
  // default one.)
  {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    if (cudaMemPoolCreate(&S->pool, &props) == cudaSuccess) {
      uint64_t keep = hbm_budget_bytes;
      cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      (void)cudaGetLastError();
      S->pool = nullptr;
    }
  }
  S->stager = std::thread(stager_loop, S);
  for (int i = 0; i < workers; ++i) S->workers.emplace_back(worker_loop, S);
  *out = S;
  return QMS_OK;
}

int qms_server_submit(qms_server* S, const void* in, void* out, size_t n, int dtype, int pivot,
                      uint64_t* ticket) {
  if (!S || !ticket || dtype < QMS_U32 || dtype > QMS_F32 || pivot < QMS_PIVOT_M3 ||
      pivot > QMS_PIVOT_HYBRID)
    return QMS_EINVAL;
  if (n > 0 && (in == nullptr || out == nullptr)) return QMS_EINVAL;
  auto* r = new (std::nothrow) Req();
  if (!r) return QMS_ENOMEM;
  r->in = in;
  r->out = out;
  r->n = n;
  r->dtype = dtype;
  r->pivot = pivot;
  r->in_place = (in == out) && n > 0 && is_device_ptr(out);
  const size_t data = r->in_place ? 0 : r256(n * key_bytes(dtype));
  r->bytes = data + n / 16 + 65536;  // slot plus the sort's workspace (about n/27 bytes)
  if (r->bytes > S->budget) {
    delete r;
    return QMS_EBUDGET;
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete r;
      return QMS_EINVAL;
    }
    r->id = S->next_id++;
    if (n <= 1) {  // nothing to sort
      r->done = true;
      ++S->completed;
      S->keys_done += n;
      r->t_admit = r->t_done = r->t_submit;
      if (n == 1 && in != out) {
        if (cudaMemcpy(out, in, key_bytes(dtype), cudaMemcpyDefault) != cudaSuccess) {
          (void)cudaGetLastError();
          r->rc = QMS_ECUDA;
        }
      }
    } else {
      S->pending.push_back(r);
    }
    S->reqs[r->id] = r;
    *ticket = r->id;
  }
  S->cv_work.notify_one();
  return QMS_OK;
}

int qms_server_poll(qms_server* S, uint64_t ticket, int* done, qms_request_info* info) {
  if (!S || !done) return QMS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return QMS_EINVAL;
  Req* r = it->second;
  *done = r->done ? 1 : 0;
  if (!r->done) return QMS_EAGAIN;
  fill_info(r, info);
  S->reqs.erase(it);
  delete r;
  return QMS_OK;
}

int qms_server_wait(qms_server* S, uint64_t ticket, double timeout_ms, qms_request_info* info) {
  if (!S) return QMS_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return QMS_EINVAL;
  Req* r = it->second;
  const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                      [&] { return r->done; });
  if (!ok) return QMS_ETIMEOUT;
  fill_info(r, info);
  S->reqs.erase(it);
  delete r;
  return QMS_OK;
}

int qms_server_get_stats(qms_server* S, qms_server_stats* out) {
  if (!S || !out) return QMS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = S->completed;
  out->keys = S->keys_done;
  out->batches = S->batches;
  out->batched_requests = S->batched_reqs;
  out->pending = S->pending.size();
  out->in_flight = static_cast<uint64_t>(S->in_flight);
  out->peak_in_flight = static_cast<uint64_t>(S->peak_in_flight);
  out->used_bytes = S->used;
  out->peak_used_bytes = S->peak_used;
  out->budget_bytes = S->budget;
  return QMS_OK;
}

int qms_server_pause(qms_server* S, int paused) {
  if (!S) return QMS_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->paused = paused != 0;
  }
  S->cv_work.notify_all();
  S->cv_ready.notify_all();
  return QMS_OK;
}

int qms_server_destroy(qms_server* S) {
  if (!S) return QMS_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->paused = false;
  }
  S->cv_work.notify_all();
  S->cv_ready.notify_all();
  S->stager.join();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->reqs) delete kv.second;
  if (S->pool) {
    cudaDeviceSynchronize();  // every slot has been freed on its worker's stream
    cudaMemPoolDestroy(S->pool);
  }
  delete S;
  return QMS_OK;
}

}  // extern "C"
