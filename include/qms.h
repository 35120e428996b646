/* qms.h -- C ABI of the GB300 QuickMergesort library (libqms.so).
 *
 * The method is QuickMergesort (Edelkamp & Weiss, "QuickMergesort: Practically
 * Efficient Constant-Factor Optimal Sorting", arXiv 1804.10062): choose a
 * pivot (median-of-3, median-of-sqrt(n), median of medians, or the hybrid of
 * Sec. 4), partition the array in place, Mergesort one side using the other
 * side as a swap buffer (buffer elements are permuted, never overwritten),
 * and continue on the remaining side (Sec. 2 and the Fig. 3 listing).  The
 * problem statement is internal sorting: n elements, ascending, with only
 * O(log n) extra words beyond the array (Sec. 1).  On the GPU the extra
 * memory is O(n / 256 + 1) words, about n/27 bytes plus an 18 KB descriptor
 * (per-tile counters and prefixes of the partition, merge-path splits,
 * overlapped-merge flags); there is no n-sized scratch.
 *
 * Conventions for every call:
 *   - Key and payload pointers are DEVICE pointers owned by the caller; sorts
 *     are in place and ascending.  Keys: uint32, uint64, int64 (signed order)
 *     or float32 (IEEE order with -0 < +0; NaN keys are not supported).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered; unless stated otherwise a call
 *     returns after its work on `stream` has finished.
 *   - Return value: QMS_OK (0) or a negative QMS_E* code.  Nothing aborts,
 *     traps or exits.  n = 0 and n = 1 are valid no-ops.
 *   - `opt` may be NULL (median-of-3, no counting).  `stats` may be NULL.
 */
#ifndef QMS_H_
#define QMS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define QMS_OK 0
#define QMS_EINVAL (-1)   /* null pointer, bad dtype/pivot, size out of range */
#define QMS_ENOMEM (-2)   /* device workspace could not be allocated         */
#define QMS_EBUDGET (-3)  /* server: request larger than the HBM budget      */
#define QMS_ECUDA (-4)    /* a CUDA runtime call or kernel launch failed      */
#define QMS_ETIMEOUT (-5) /* a bounded device or host wait gave up            */
#define QMS_EAGAIN (-6)   /* server poll: request not finished yet            */
#define QMS_EINTERNAL (-7)/* a device-side consistency check failed          */

/* Key types (dtype arguments). */
#define QMS_U32 0
#define QMS_U64 1
#define QMS_I64 2
#define QMS_F32 3

/* Pivot rules (qms_options.pivot).
 *   M3     : median of positions b, b + floor(n/2), e - 1 (Sec. 2, Thm. 1).
 *   SQRTN  : median of an evenly spaced sample of the largest odd k <=
 *            ceil(sqrt n) elements, k capped at 16383 (Sec. 2, Thm. 2).
 *   MOM    : exact median of the floor(n/3) medians of consecutive triples
 *            (MoMQuickMergesort, Sec. 4; the selection is a radix select).
 *   HYBRID : M3, but a pivot whose rank lies outside [n/16, n - 1 - n/16]
 *            makes the next round MOM (HybridQuickMergesort, Sec. 4). */
#define QMS_PIVOT_M3 0
#define QMS_PIVOT_SQRTN 1
#define QMS_PIVOT_MOM 2
#define QMS_PIVOT_HYBRID 3

/* Kernel classes of the per-kernel device-time profile. */
#define QMS_K_LEAF 0          /* base case / Mergesort leaves                  */
#define QMS_K_MERGE_SPLIT 1   /* merge-path windows of a swap-merge level      */
#define QMS_K_MERGE 2         /* swap-merge level                              */
#define QMS_K_PART_LOCAL 3    /* partition: local partition of every tile      */
#define QMS_K_PART_SCAN 4     /* partition: scan of the tile counts            */
#define QMS_K_PART_EXCHANGE 5 /* partition: exchange of misplaced elements     */
#define QMS_K_PIVOT 6         /* pivot selection (all rules) and placement     */
#define QMS_K_BATCH 7         /* batched-form kernels                          */
#define QMS_NKINDS 8

/* Optional per-kernel-class profile, filled when qms_options.profile is set:
 * device time from CUDA events recorded around every launch on the call's
 * stream, and the algorithmic bytes each class must move (keys and payloads
 * read plus written, counted from the sizes it was launched on). */
typedef struct {
  double ms[QMS_NKINDS];
  uint64_t bytes[QMS_NKINDS];
  uint64_t launches[QMS_NKINDS];
} qms_profile;

/* qms_options.flags */
#define QMS_FLAG_ASYNC 1       /* qms_sort / qms_sort_pairs without stats: return once
                                  the sort is enqueued on the stream (no host wait)  */
#define QMS_FLAG_HOST_DRIVEN 2 /* run the rounds from the host (one launch per step,
                                  one device-to-host read per round) instead of the
                                  device-driven CUDA graph; implied by `profile`     */
#define QMS_FLAG_LARGER_SIDE 4 /* Mergesort the larger side, with a buffer of half its
                                  size from the other side (Sec. 2, Fig. 1; Fig. 3's
                                  "out" with its overlapped final merge), whenever it
                                  exceeds 8192 keys and that buffer fits.  Default:
                                  Fig. 3's side rule with a full-size buffer          */
#define QMS_FLAG_TEST_WITHHOLD 8 /* test hook for failure handling: the overlapped
                                  merge of QMS_FLAG_LARGER_SIDE rounds never marks
                                  its first tile done, so the waits on that tile run
                                  out after spin_limit polls and the sort returns
                                  QMS_ETIMEOUT (its output is then unspecified)       */
#define QMS_FLAG_DEVICE_DRIVEN 16 /* run the rounds as the device-driven CUDA graph even
                                  when the call waits for its result (by default a
                                  waiting call of 2^16 keys or more runs them from
                                  the host); ignored with `profile` or
                                  QMS_FLAG_HOST_DRIVEN                                 */

typedef struct {
  int pivot;       /* QMS_PIVOT_*                                              */
  int count_cmps;  /* nonzero: use the counting kernels and report
                      qms_stats.comparisons (element comparisons, Sec. 5)      */
  int flags;       /* QMS_FLAG_*                                               */
  int spin_limit;  /* polls of one completion flag before a bounded device wait
                      gives up with QMS_ETIMEOUT; <= 0: the default, 2^20 polls
                      (about a second).  Only the overlapped merge waits.     */
  qms_profile* profile; /* NULL, or accumulates per-kernel device times (host-
                           driven rounds, CUDA events around every launch)    */
} qms_options;

typedef struct {
  uint64_t comparisons; /* element comparisons made (count_cmps only)          */
  uint64_t aux_bytes;   /* device workspace used (about n/27 bytes + 18 KB)    */
  uint64_t rounds;      /* partition rounds                                      */
  uint64_t mom_rounds;  /* rounds that used a median-of-medians pivot            */
  uint64_t launches;    /* kernels launched                                      */
  double ms;            /* host wall time of the call                            */
} qms_stats;

/* Library version (major * 10000 + minor * 100 + patch). */
int qms_version(void);
/* Static string for an error code. */
const char* qms_error_string(int code);

/* Frees, on the current device, the cached instances of the device-driven
 * sort (one instantiated CUDA graph per key type, payload, counting mode and
 * pivot rule, each with a workspace for the largest array it has sorted,
 * about n/27 bytes for at least 2^20 keys) after their last launches have
 * finished.  An instance another host thread is setting up is kept.  Later
 * calls build what they need again.  The paper has no counterpart.
 * Errors: QMS_ECUDA. */
int qms_release_cached(void);

/* Sorts d_keys[0, n) in place, ascending (the QuickMergesort driver loop of
 * Fig. 3: partition, Mergesort the side left of the midpoint test, continue
 * on the other side; a last range of at most one Mergesort leaf -- 16384
 * keys, 8192 with payloads -- is finished by the base case).  The round
 * loop runs on the device as one CUDA graph with conditional nodes
 * (instances are cached per key type, pivot rule and device; the first call
 * of a kind builds one), and the call returns after the sort finished; with
 * QMS_FLAG_ASYNC and stats == NULL it returns once the sort is enqueued on
 * `stream`.  A call that waits for arrays of 2^16 keys or more runs the
 * rounds from the host instead (as QMS_FLAG_HOST_DRIVEN), which measured
 * faster: one small read-back per round costs less than the graph's
 * conditional nodes.  QMS_FLAG_DEVICE_DRIVEN keeps such a call on the graph.  Errors: QMS_EINVAL (d_keys NULL
 * with n > 1, bad dtype or pivot), QMS_ENOMEM, QMS_ECUDA, QMS_EINTERNAL,
 * QMS_ETIMEOUT (a bounded device wait gave up; see qms_options.spin_limit). */
int qms_sort(void* d_keys, size_t n, int dtype, const qms_options* opt, void* stream,
             qms_stats* stats);

/* As qms_sort, and moves the uint32 payload d_vals[i] with key d_keys[i].
 * The order among equal keys is unspecified (QuickMergesort is not stable);
 * the (key, payload) multiset is preserved.  n must be < 2^32. */
int qms_sort_pairs(void* d_keys, uint32_t* d_vals, size_t n, int dtype, const qms_options* opt,
                   void* stream, qms_stats* stats);

/* Batched form: sorts every segment d_keys[off[i], off[i+1]) independently,
 * i < nseg, where off = d_offsets (DEVICE array of nseg + 1 non-decreasing
 * uint64 offsets into d_keys).  Each segment is one QuickMergesort (the same
 * method as qms_sort).  Segments of up to 64 * 8192 keys are sorted by one
 * thread block each in one persistent launch, longest first (an atomic ticket
 * hands out the next segment); longer segments run through the grid-wide
 * driver.  d_vals may be NULL; with payloads the total length must be < 2^32.
 * Extra device memory: O(nseg) words.  Errors: QMS_EINVAL (decreasing
 * offsets, bad dtype/pivot), QMS_ENOMEM, QMS_ECUDA, QMS_EINTERNAL. */
int qms_sort_batched(void* d_keys, uint32_t* d_vals, const uint64_t* d_offsets, size_t nseg,
                     int dtype, const qms_options* opt, void* stream, qms_stats* stats);

/* ---- Batched form: plan and autotuner ------------------------------------
 * qms_sort_batched maps every segment length bin b (segments of
 * (2^(b-1), 2^b] keys, b < QMS_BATCH_BINS; b = 0 holds single keys) to a
 * kernel configuration.  The group configurations QMS_BCFG_G32 ..
 * QMS_BCFG_G512W and QMS_BCFG_G1024W sort a segment that fits their tile
 * with the base case (Fig. 3's driver never partitions a range of one tile
 * or less) inside one group of threads -- a warp, or a block-sized group;
 * groups of at most 512 threads share a block.  QMS_BCFG_PAIR sorts the two
 * halves of a segment in a cluster of two blocks and merges them through
 * distributed shared memory.  QMS_BCFG_QMS runs the QuickMergesort rounds
 * of a segment in one block.
 * Segments longer than 2^(QMS_BATCH_BINS-1) keys always take the rounds.
 * The default plan takes, per bin, the smallest group whose tile holds it.
 * The autotuner times every admissible configuration per bin on the
 * current GPU and keeps the fastest; the plan is stored per key width,
 * payload and SM count in the JSON file
 *   $QMS_AUTOTUNE_DIR/batched_k<4|8>_v<0|1>_sm<count>.json
 * (default directory $HOME/.cache/qms_gb300), which later processes read on
 * their first batched call.  The paper has no batched form. */
#define QMS_BATCH_BINS 17
#define QMS_BCFG_G32 0    /* one warp, 16 keys per thread: up to 512 keys   */
#define QMS_BCFG_G64 1    /* 64 threads x 16: up to 1024                    */
#define QMS_BCFG_G128 2   /* 128 x 16: up to 2048                           */
#define QMS_BCFG_G256 3   /* 256 x 16: up to 4096                           */
#define QMS_BCFG_G512 4   /* 512 x 16: up to 8192                           */
#define QMS_BCFG_G256W 5  /* 256 x 32: up to 8192 (4-byte keys, no payload) */
#define QMS_BCFG_G512W 6  /* 512 x 32: up to 16384 (4-byte keys, no payload)*/
#define QMS_BCFG_QMS 7    /* one block per segment, QuickMergesort rounds   */
#define QMS_BCFG_G1024W 8 /* 1024 x 32, one group per block: up to 32768
                             (4-byte keys, no payload)                      */
#define QMS_BCFG_PAIR 9   /* a cluster of two 1024 x 32 blocks, merged through
                             distributed shared memory: up to 65536 (4-byte
                             keys, no payload)                              */

/* Times every configuration per length bin on the current device (about a
 * second of GPU work), installs the fastest plan for (dtype's key width,
 * with_payload) on this device and writes the plan file.  report (may be
 * NULL) receives a text table of the timings, truncated to report_len.
 * Errors: QMS_EINVAL, QMS_ENOMEM, QMS_ECUDA, QMS_EINTERNAL. */
int qms_batched_autotune(int dtype, int with_payload, void* stream, char* report,
                         size_t report_len);

/* The plan in use on the current device (loading the plan file on first
 * use): cfg[b] for b < nbins (bins beyond QMS_BATCH_BINS read as
 * QMS_BCFG_QMS); *tuned = 1 when it came from the autotuner or its file. */
int qms_batched_get_plan(int dtype, int with_payload, int* cfg, int nbins, int* tuned);

/* Installs a plan for the current device (nbins == QMS_BATCH_BINS); every
 * entry must exist for these keys and hold its bin.  QMS_EINVAL otherwise. */
int qms_batched_set_plan(int dtype, int with_payload, const int* cfg, int nbins);

/* Host-only helpers (no GPU): read a plan file written for sm_count SMs
 * into cfg (QMS_EAGAIN, with the default plan in cfg, when the file is
 * missing or was written for other keys or another SM count), and write
 * one (ns_per_key may be NULL). */
int qms_batched_plan_read(const char* path, int dtype, int with_payload, int sm_count, int* cfg,
                          int nbins);
int qms_batched_plan_write(const char* path, int dtype, int with_payload, int sm_count,
                           const int* cfg, const double* ns_per_key, int nbins);
/* Static name of a configuration ("group32x16", ..., "block_qms"). */
const char* qms_batched_config_name(int cfg);

/* ---- Served form --------------------------------------------------------
 * A request server with continuous batching (no counterpart in the paper,
 * which sorts one array; each request is one QuickMergesort).  Requests are
 * admitted in arrival order against a device-memory budget -- the bytes the
 * server itself holds for a request: a device slot for its keys, unless the
 * keys are a device array sorted in place (in == out), plus the sort's
 * workspace (charged as n/16 bytes + 64 KB) -- and a maximum number of
 * admitted requests.  A staging thread admits the next request as soon as
 * it fits, allocates its slot and starts the upload of its keys, so admitted
 * requests hold their share of the budget while they wait and uploads
 * overlap earlier sorts.  Worker threads, each with its own stream, take
 * admitted requests in order: a request longer than 64 * 8192 keys runs
 * alone through the grid-wide rounds; shorter ones waiting at the head are
 * sorted together in one persistent launch (one block each, longest first).
 * Results are copied out and the slot freed before a request completes.
 * Requests never share memory, so each result equals that request's sort
 * alone. */
typedef struct qms_server qms_server;

typedef struct {
  int status;         /* QMS_OK or the error of this request              */
  int batch_size;     /* requests sorted in the same launch (1 = alone)    */
  uint64_t n;
  double queue_ms;    /* submit -> admitted                                */
  double latency_ms;  /* submit -> result written                          */
} qms_request_info;

typedef struct {
  uint64_t completed, keys, batches, batched_requests, pending, in_flight, peak_in_flight;
  uint64_t used_bytes, peak_used_bytes, budget_bytes;
} qms_server_stats;

/* Creates a server on the current device.  hbm_budget_bytes: device bytes
 * the server may hold for admitted requests; max_slots: admitted requests at
 * once; workers: worker threads/streams (1..64); max_batch: requests per
 * batched launch.  Errors: QMS_EINVAL, QMS_ENOMEM, QMS_ECUDA. */
int qms_server_create(size_t hbm_budget_bytes, int max_slots, int workers, int max_batch,
                      qms_server** out);

/* Queues a request to sort n keys of `dtype` read from `in` and written
 * sorted to `out`; in/out may be host or device pointers (unified
 * addressing decides the copy direction) and must stay valid until the
 * request is done.  in == out on a device array sorts it in place.
 * Non-blocking.  *ticket identifies the request.  Errors: QMS_EINVAL,
 * QMS_EBUDGET (the request alone exceeds the budget), QMS_ENOMEM. */
int qms_server_submit(qms_server* srv, const void* in, void* out, size_t n, int dtype, int pivot,
                      uint64_t* ticket);

/* Non-blocking: *done = 1 and QMS_OK when the request has finished (info
 * filled; the ticket is then released), else *done = 0 and QMS_EAGAIN.
 * QMS_EINVAL for an unknown ticket. */
int qms_server_poll(qms_server* srv, uint64_t ticket, int* done, qms_request_info* info);

/* Blocks up to timeout_ms for the request; QMS_ETIMEOUT if it has not
 * finished by then (the ticket stays valid). */
int qms_server_wait(qms_server* srv, uint64_t ticket, double timeout_ms, qms_request_info* info);

int qms_server_get_stats(qms_server* srv, qms_server_stats* out);

/* Host-side control for failure handling and tests: while paused, nothing
 * new is admitted and workers take no new request (work already on the GPU
 * finishes); waits on queued requests then run into their timeouts.
 * paused = 0 resumes. */
int qms_server_pause(qms_server* srv, int paused);

/* Finishes every queued request, stops the workers and frees the server. */
int qms_server_destroy(qms_server* srv);

/* ---- Step-level entry points (one step of a round each; used by the
 * ---- parity tests of the individual kernels). ------------------------- */

/* Base case X (Fig. 3 msort leaf): sorts d_keys[0, n), n <= 8192, in one
 * thread block (d_vals may be NULL). */
int qms_tile_sort(void* d_keys, uint32_t* d_vals, size_t n, int dtype, void* stream);

/* One partition step (Sec. 2): chooses a pivot of d_keys[0, n) (n >= 3) with
 * rule `pivot`, partitions in place and writes the pivot's final index to
 * *k_out and the number of further keys equal to the pivot placed right
 * after it to *eq_out (nonzero only when the duplicate guard ran the second
 * pass).  Afterwards keys[0, k) < pivot, keys[k, k + 1 + eq) == pivot and
 * keys[k + 1 + eq, n) >= pivot (> pivot when eq was computed). */
int qms_partition(void* d_keys, uint32_t* d_vals, size_t n, int dtype, int pivot, void* stream,
                  uint64_t* k_out, uint64_t* eq_out);

/* Mergesort with a swap buffer (Fig. 3 "out", in its full-buffer form):
 * sorts d_keys[0, m) using the m slots d_keys[buf, buf + m) as buffer
 * (buf >= m, so the regions are disjoint); the buffer's multiset is preserved
 * and its order permuted. */
int qms_mergesort(void* d_keys, uint32_t* d_vals, size_t m, size_t buf, int dtype, void* stream);

/* Mergesort with a half-size buffer (Fig. 3 "out" itself): sorts d_keys[0, m)
 * using the ceil(m/2) slots d_keys[buf, buf + ceil(m/2)) as buffer (buf >= m).
 * The second half is sorted into the buffer, the first half into the tail of
 * the part, and the overlapped final merge fills the part.  The buffer's
 * multiset is preserved and its order permuted.  Errors: QMS_EINVAL (bad
 * dtype, d_keys NULL with m > 1, buf < m), QMS_ENOMEM, QMS_ECUDA,
 * QMS_EINTERNAL (a bounded wait of the overlapped merge ran out). */
int qms_mergesort_half(void* d_keys, uint32_t* d_vals, size_t m, size_t buf, int dtype,
                       void* stream);

/* ---- Allocation-free sort -------------------------------------------- */

/* Largest n accepted by qms_sort_noalloc. */
#define QMS_NOALLOC_MAX_N (1ull << 24)

/* qms_sort without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * e.g. an application that gives the whole GPU memory to its own pool
 * allocator and forbids any other cudaMalloc, or a latency-critical loop in
 * which an allocation could synchronise the device or fail under memory
 * pressure.  The sort's round descriptor and per-tile counters live in one
 * fixed file-scope device array of about 900 KB, which every GPU that loads
 * the library holds until the process exits.  The caller passes the keys as
 * with qms_sort (keys only; opt->profile must be NULL).
 *   - n > QMS_NOALLOC_MAX_N (2^24) returns QMS_EINVAL; nothing runs.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     The address is kept for the life of the process, so the library must
 *     not be used across a cudaDeviceReset.
 *   - All calls share the one array and it keeps the last call's contents
 *     (each call clears what must start at zero).  Calls that overlap on the
 *     GPU (other streams, other host threads) race on it: serialise them.
 *   - The rounds run from the host: the call reads one small result back
 *     per round and returns once the sort has finished on `stream`
 *     (QMS_FLAG_ASYNC has no effect).  QMS_FLAG_LARGER_SIDE, count_cmps and
 *     spin_limit behave as in qms_sort.
 * Errors as qms_sort. */
int qms_sort_noalloc(void* d_keys, size_t n, int dtype, const qms_options* opt, void* stream,
                     qms_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* QMS_H_ */
