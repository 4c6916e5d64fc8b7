/*
 * ms.h -- C ABI of the GB300 (sm_103a) stable multisplit library (libms.so).
 *
 * The operation is the multisplit primitive of "GPU Multisplit: an extended
 * study of a parallel algorithm" (Ashkiani, Davidson, Meyer, Owens), Section
 * 3.1: permute n 32-bit keys (or key-value pairs) into m contiguous buckets in
 * ascending bucket-ID order, keeping the input order inside every bucket
 * (stable), and report where every bucket starts.  The final position of
 * element i in bucket j is Eq. 1 of Section 4.2:
 *     p(i) = sum_{k<j} h_k + |{u_r in B_j : r < i}|.
 * The radix sort of Section 7.1 is built from multisplit passes whose bucket
 * identifier is the radix digit f_k(u) = (u >> kr) & (2^r - 1).
 *
 * Conventions for every entry point:
 *   - Pointers named *_in / *_out / offsets are DEVICE pointers on the current
 *     CUDA device, owned by the caller.  Keys and values are copied bit for
 *     bit (float keys travel as their raw bits).  Inputs and outputs must not
 *     overlap.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls are asynchronous with respect to the host: they enqueue
 *     work on `stream` and return.
 *   - The library owns its scratch memory (histogram matrix, look-back status
 *     words).  It takes it from a library-owned, stream-ordered memory pool on
 *     the calling stream and returns it on the same stream, so a call is safe
 *     to overlap with calls on other streams.
 *   - Errors are status codes; nothing is thrown across the ABI.  Argument
 *     errors are detected on the host before anything is enqueued.  A device
 *     side failure (a bounded wait that ran out) is recorded in a per-device
 *     status word that ms_device_status() returns.
 *   - n may be 0 (offsets are then all 0).  n must be < 2^32.
 */
#ifndef MS_H_
#define MS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MS_OK = 0,
  MS_ERR_INVALID_ARG = 1,   /* a bad argument; nothing was enqueued */
  MS_ERR_UNSUPPORTED = 2,   /* a valid request this build does not handle */
  MS_ERR_OUT_OF_MEMORY = 3, /* the scratch allocation failed */
  MS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  MS_ERR_TIMEOUT = 5        /* a device-side bounded wait expired */
} ms_status;

/* Bucket identifiers (Section 6 "Bucket identification", Section 7.1, 7.3). */
typedef enum {
  /* range splitters (Section 7.3 "Range histogram"): `splitters` holds m-1
   * nondecreasing uint32 values s_1..s_{m-1} in DEVICE memory; the bucket of u
   * is the number of splitters <= u (u < s_1 -> 0, u >= s_{m-1} -> m-1). */
  MS_BUCKET_RANGE_U32 = 0,
  /* delta buckets on float32 keys (Section 6, Section 7.3 "Even histogram"):
   * q = (x - x0) / delta rounded to nearest in binary32, b = floor(q), then
   * b <= 0 -> 0, b >= m (and +inf, NaN) -> m-1. */
  MS_BUCKET_DELTA_F32 = 1,
  /* radix digit (Section 7.1): (u >> shift) & (2^bits - 1); m must be 2^bits,
   * 0 <= bits <= 8 (<= 16 for ms_multisplit_keys / _pairs), shift + bits <= 32. */
  MS_BUCKET_RADIX = 2,
  /* u mod m. */
  MS_BUCKET_MOD = 3
} ms_bucket_kind;

typedef struct {
  int32_t kind;               /* an ms_bucket_kind */
  uint32_t m;                 /* number of buckets, 1 <= m <= 256; up to 65536
                               * for ms_multisplit_keys / ms_multisplit_pairs */
  const uint32_t *splitters;  /* RANGE_U32 only: device pointer, m-1 entries */
  float x0, delta;            /* DELTA_F32 only: delta > 0 and finite */
  uint32_t shift, bits;       /* RADIX only */
} ms_bucket_spec;

/* Stable multisplit of keys (Section 3.1, Eq. 1).
 * With 257 <= m <= 65536 buckets (Section 6.3, larger multisplits) the call
 * runs two multisplit passes over the 8-bit digits of the bucket id, least
 * significant first, through a library pool buffer of n words (per array),
 * then a bisection per bucket for the offsets; the result is the same stable
 * multisplit, for every identifier kind.
 *   keys_in[n]   -> keys_out[n]: the keys grouped by bucket, buckets ascending,
 *                   input order kept inside each bucket.
 *   offsets[m+1] -> offsets[j] = start of bucket j in keys_out, offsets[m] = n
 *                   (the paper's optional "beginning index of each bucket",
 *                   with one extra entry).  May be NULL if not wanted.
 * Errors: MS_ERR_INVALID_ARG for a NULL data pointer with n > 0, keys_in ==
 * keys_out, n >= 2^32 or a bad spec (see ms_bucket_spec). */
ms_status ms_multisplit_keys(const uint32_t *keys_in, size_t n, const ms_bucket_spec *spec,
                             uint32_t *keys_out, uint32_t *offsets, void *stream);

/* Stable multisplit of key-value pairs (Section 3.1; values are opaque 32-bit
 * words carried along the same permutation as their keys). */
ms_status ms_multisplit_pairs(const uint32_t *keys_in, const uint32_t *vals_in, size_t n,
                              const ms_bucket_spec *spec, uint32_t *keys_out, uint32_t *vals_out,
                              uint32_t *offsets, void *stream);

/* LSD radix sort built on multisplit (Section 7.1): a stable sort of the keys
 * (and values) by the key bits [begin_bit, end_bit), 0 <= begin_bit <=
 * end_bit <= 32, in passes of 8-bit digits (the last pass takes the bits
 * left over).  vals_in / vals_out may both be NULL (keys only).  keys_out /
 * vals_out must not overlap the inputs.  The library holds one ping-pong
 * buffer of n words (per array) in its pool during the call. */
ms_status ms_radix_sort(const uint32_t *keys_in, const uint32_t *vals_in, size_t n, int begin_bit,
                        int end_bit, uint32_t *keys_out, uint32_t *vals_out, void *stream);

/* The same sort with r-bit digits, 1 <= r <= 8 (Section 6.3, the radix-width
 * study of the sort table): ceil((end_bit - begin_bit) / r) multisplit passes
 * into 2^r buckets, the last pass taking the bits left over (r = 7 on 32 bits:
 * four 7-bit passes and one 4-bit pass).  Arguments and errors as for
 * ms_radix_sort; MS_ERR_INVALID_ARG for r outside 1..8. */
ms_status ms_radix_sort_r(const uint32_t *keys_in, const uint32_t *vals_in, size_t n, int begin_bit,
                          int end_bit, int r, uint32_t *keys_out, uint32_t *vals_out, void *stream);

/* Device histogram (Section 7.3, "Even" and "Range" histograms built on the
 * multisplit's pre-scan): counts[b] = number of keys whose bucket is b, for
 * 0 <= b < m, under the same bucket identifiers (range splitters = Range,
 * float32 delta buckets = Even).  keys: device, n words; counts: device, m
 * words, overwritten.  Reads the keys once; no permutation is made.
 * Errors: MS_ERR_INVALID_ARG for a bad spec, counts == NULL, keys == NULL
 * with n > 0, or n >= 2^32. */
ms_status ms_histogram(const uint32_t *keys, size_t n, const ms_bucket_spec *spec, uint32_t *counts,
                       void *stream);

/* Keys-only stable multisplit that allocates nothing (the paper has no
 * counterpart; this is a deployment variant of ms_multisplit_keys).  For
 * callers that must not allocate device memory during the call: hot loops
 * that forbid allocator calls, or processes whose device memory is owned by
 * another allocator.  Same arguments, result and argument errors as
 * ms_multisplit_keys; the scratch comes from a fixed 1 MiB array in device
 * memory that every GPU loading the library holds until exit.
 *   - The first call on each device (with it current) looks up the array's
 *     device address; the first call that uses a given kernel variant (picked
 *     by the bucket kind, m and the size class of n) sets that kernel's
 *     attributes and queries its occupancy; later calls skip these host-side
 *     steps.  None of this allocates.
 *   - All calls share the array: calls that overlap on the GPU race and
 *     corrupt each other's results; serialize them (one stream, or events).
 *   - The scratch must hold 4*m*G + 16 bytes, plus 8*ceil(m*G/4096) for
 *     m > 32 (G = CTAs of the launch, at most SMs x resident CTAs per SM;
 *     about 610 KiB at most on a 152-SM GB300).  A call needing more gets
 *     MS_ERR_OUT_OF_MEMORY and its outputs are not touched.
 *   - Device-side failures (an expired bounded wait, a failed bounds check)
 *     are recorded in a header word of the fixed array, not in the word
 *     ms_device_status() reads: ms_noalloc_status() reports them.  Each call
 *     starts from a clear word, so a failure never shortens the waits of a
 *     later call. */
ms_status ms_multisplit_keys_noalloc(const uint32_t *keys_in, size_t n, const ms_bucket_spec *spec,
                                     uint32_t *keys_out, uint32_t *offsets, void *stream);

/* Reads and clears the device-side status of ms_multisplit_keys_noalloc on
 * the calling device (no counterpart in the paper): MS_OK, MS_ERR_TIMEOUT if a
 * bounded wait of any such call expired since the last read, MS_ERR_CUDA for
 * another recorded failure (a failed bounds check) or a failed CUDA call.
 * Synchronizes `stream` first; covers every call enqueued before that point. */
ms_status ms_noalloc_status(void *stream);

/* Failure-path test aid of the entry point above (no counterpart in the
 * paper): enqueues on `stream` the look-back scan kernel as the second of two
 * scan tiles on the fixed array's scratch, with the first tile's status never
 * published, so its bounded wait runs out (after about a quarter of a second)
 * and records MS_ERR_TIMEOUT exactly where an expired wait inside
 * ms_multisplit_keys_noalloc would.  Shares the array with that entry point:
 * serialize it with those calls. */
ms_status ms_test_expire_lookback_noalloc(void *stream);

/* ---- Batched multisplit: many independent arrays in one persistent launch.
 * Not in the paper (it runs one problem per launch); the same method applied
 * to thousands of uneven arrays at once.  All segments of a plan share one
 * bucket identifier and are all keys-only (vals_in = vals_out = NULL) or all
 * key-value.  Each segment's result equals ms_multisplit_keys/_pairs on it. */
typedef struct {
  const uint32_t *keys_in;  /* device, n keys */
  const uint32_t *vals_in;  /* device, n values, or NULL for keys only */
  uint32_t *keys_out;       /* device, n keys */
  uint32_t *vals_out;       /* device, n values, or NULL */
  uint32_t *offsets;        /* device, m+1 bucket starts, or NULL */
  size_t n;                 /* < 2^32; 0 allowed */
} ms_segment;

typedef struct ms_batch_plan ms_batch_plan;

/* Reads the host array segs[num_segments] (copied; the device buffers it
 * names must stay valid while the plan is used, as must spec->splitters) and
 * builds the work list: items of up to 8 consecutive 4096-key tiles of one
 * segment (one tile for the kernel of more than 32 buckets), first for the
 * histograms of segments longer than one tile, then for the post-scans.  Allocates
 * the plan's device memory with cudaMalloc and uploads the list
 * (synchronous; do it once, outside any capture).  The plan is key-value if
 * any segment has vals_in; every non-empty segment must then carry values.
 * Errors: MS_ERR_INVALID_ARG (bad spec, NULL/overlapping buffers, mixed
 * keys-only and key-value segments), MS_ERR_OUT_OF_MEMORY, MS_ERR_CUDA. */
ms_status ms_batch_plan_create(const ms_segment *segs, uint32_t num_segments, const ms_bucket_spec *spec,
                               ms_batch_plan **plan);

/* A plan whose segments change from run to run (for a serving loop): sized
 * for at most max_segments segments totalling max_elements keys, all keys-only
 * (pairs = 0) or all key-value (pairs = 1).  Allocates device memory and two
 * pinned staging areas (synchronous).  Starts with no segments. */
ms_status ms_batch_plan_create_dynamic(uint32_t max_segments, uint64_t max_elements, int pairs,
                                       const ms_bucket_spec *spec, ms_batch_plan **plan);

/* Replaces a dynamic plan's segments: validates segs as ms_batch_plan_create
 * does, builds the work list into a pinned staging area and enqueues its upload
 * on `stream` (asynchronous; waits only if the staging area's upload of two
 * calls ago has not finished).  Runs that follow on the same stream use the new
 * segments; a run must not be in flight on another stream.  Exceeding the
 * plan's capacity gives MS_ERR_INVALID_ARG. */
ms_status ms_batch_plan_set_segments(ms_batch_plan *plan, const ms_segment *segs, uint32_t num_segments,
                                     void *stream);

/* Enqueues on `stream` one memset of the plan's flags and one persistent
 * kernel that multisplits every segment.  Allocates nothing and does not
 * synchronize, so it can be captured in a CUDA graph.  Runs of one plan must
 * not overlap on the GPU (they share the plan's flags and histograms).  Must
 * be called with the plan's device current. */
ms_status ms_batch_run(ms_batch_plan *plan, void *stream);

/* The same work, captured into a CUDA graph on the first call (made on a
 * private stream) and launched on `stream` by every call.  The graph reads the
 * plan's work list from device memory, so it follows later
 * ms_batch_plan_set_segments calls. */
ms_status ms_batch_run_graph(ms_batch_plan *plan, void *stream);

/* Waits for the device, then frees the plan (NULL is fine). */
ms_status ms_batch_plan_destroy(ms_batch_plan *plan);

/* The batched multisplit in one call, over segment descriptors that live in
 * DEVICE memory (the batching form of Section 3.1's multisplit; the paper
 * runs one problem per launch).  segs_dev: device array of num_segments
 * ms_segment, all keys-only or all key-value as for ms_batch_plan_create.
 * offsets: device array of num_segments * (m + 1) words, segment i's bucket
 * starts at offsets[i * (m + 1)] (then each descriptor's own `offsets` field
 * is ignored), or NULL to use the descriptors' fields.  The call reads the
 * descriptors back to the host -- it synchronizes `stream` for that -- builds
 * the work list, and enqueues one memset and one persistent launch on
 * `stream` through a plan the library keeps per (device, spec, keys-only or
 * key-value) and grows as needed; spec->splitters must stay valid until that
 * work is done.  Calls that reuse a cached plan are ordered one after another
 * on the GPU even from different streams.  Each segment's result equals
 * ms_multisplit_keys / ms_multisplit_pairs on it.  Errors as for
 * ms_batch_plan_create, checked before anything is enqueued. */
ms_status ms_multisplit_pairs_batched(const ms_segment *segs_dev, uint32_t num_segments,
                                      const ms_bucket_spec *spec, uint32_t *offsets, void *stream);

/* Releases what the library holds on every device it has used: the scratch
 * memory pool, the device status word, the plans cached by
 * ms_multisplit_pairs_batched, and the stage-timing events.  Waits for each
 * of those devices first.  A later call starts afresh (it creates the state
 * again).  Returns MS_ERR_INVALID_ARG, and releases nothing, while a batch plan
 * made by the caller is still alive (destroy it first).  Safe to call twice;
 * must not run concurrently with other calls of this library.  The fixed
 * array of ms_multisplit_keys_noalloc is part of the loaded library and stays. */
ms_status ms_shutdown(void);

/* Reads and clears the calling device's status word: MS_OK, or
 * MS_ERR_TIMEOUT if any bounded device-side wait expired since the last read.
 * Synchronizes `stream` first. */
ms_status ms_device_status(void *stream);

/* Stage timing, a tracing aid in the spirit of the paper's per-stage timing
 * (Table 4: pre-scan, scan, post-scan).  ms_stage_timing(1) clears the record
 * and starts recording CUDA events on the launching stream around the three
 * kernels of every multisplit (including each radix-sort pass) issued
 * afterwards by this process; ms_stage_timing(0) stops recording (the record
 * is kept).  ms_stage_times() waits for the recorded events and returns the
 * summed milliseconds per stage and the number of recorded multisplits; any
 * output pointer may be NULL.  Recording adds one event per stage boundary;
 * clearing while another thread is inside a multisplit call is not supported.
 * Returns MS_ERR_CUDA if an event query fails. */
ms_status ms_stage_timing(int enable);
ms_status ms_stage_times(double *prescan_ms, double *scan_ms, double *postscan_ms, uint64_t *multisplits);

/* Failure-path test aid.  Runs the look-back scan kernel as the second of two
 * scan tiles while the first tile's status word is never published, so its
 * bounded wait must run out (after about one second).  The kernel then records
 * MS_ERR_TIMEOUT in the device status word and returns; it touches only
 * library scratch.  Returns MS_OK when the launch was enqueued; the caller then
 * reads ms_device_status(), which must report MS_ERR_TIMEOUT. */
ms_status ms_test_expire_lookback(void *stream);

/* Kernel-variant tuning (not in the paper, which fixed its parameters per
 * architecture by hand, Section 6 "Parameters").  Every multisplit looks up
 * its variant by (bucket kind, pairs 0/1, ceil(log2 m) in 0..8, size class of
 * n from ms_tune_size_class: 0 below 2^16, 1 below 2^20, 2 below 2^24, 3
 * otherwise).  A variant is: shape of the post-scan tile (0: 8 warps x 16
 * keys per lane, 1: 16 x 8, 2: 8 x 8), rank mode (0: warp ballots, allowed
 * for ceil(log2 m) <= 5; 1: per-warp peer tables; 2: per-thread bucket
 * counters, allowed for ceil(log2 m) <= 5, with shape 0: 256 threads x 16
 * keys, 1: the same with a 3-tile ring (keys only), 2: 256 threads x 8 keys;
 * 3: peers found by eight ballots, per-warp bucket counters, any m) and
 * reorder (1: reorder each tile in shared memory before
 * writing, 0: write from registers; 0 requires rank mode 0 and
 * ceil(log2 m) <= 3).  Unset entries use built-in defaults.  The tuner in
 * paper_1701_01189_gb300/autotune.py measures the candidates and sets the
 * fastest.  MS_ERR_INVALID_ARG for out-of-range arguments. */
int ms_tune_size_class(size_t n);
ms_status ms_tune_set(int kind, int pairs, int log2m, int size_class, int shape, int rank, int reorder);
ms_status ms_tune_get(int kind, int pairs, int log2m, int size_class, int *shape, int *rank, int *reorder);
ms_status ms_tune_reset(void);

/* How ms_radix_sort makes its passes, per keys-only / key-value (pairs 0/1)
 * and size class: method 0 one-sweep kernels (each pass reads and writes the
 * data once; tiles learn their digit offsets by decoupled look-back), 1 one
 * three-stage multisplit per digit (pre-scan, scan, post-scan with the radix
 * digit identifier; variants from the table above).  Unset entries use 0
 * (n >= 2^30 always uses 1).  MS_ERR_INVALID_ARG for out-of-range arguments.
 * ms_tune_reset clears these entries too. */
ms_status ms_tune_set_sort(int pairs, int size_class, int method);
ms_status ms_tune_get_sort(int pairs, int size_class, int *method);

/* The kernel of batched plans (not in the paper), per (bucket kind, pairs 0/1,
 * ceil(log2 m) in 0..8, size class of the plan's mean segment length as for
 * ms_tune_size_class): rank 2 = per-thread bucket counters (m <= 32, shape
 * 0 only), 1 = per-warp peer tables, 3 = peers found by ballots with per-warp
 * counters; shape 0 = 8 warps x 16 keys per lane, 1 = 16 warps x 8 keys
 * (both 4096-key tiles).  Read when a plan is created (ms_batch_plan_create,
 * ms_batch_plan_create_dynamic, and the plans of ms_multisplit_pairs_batched);
 * unset entries use rank 2 for m <= 32 and rank 1 beyond, shape 0.
 * MS_ERR_INVALID_ARG for out-of-range arguments.  ms_tune_reset clears these
 * entries too. */
ms_status ms_tune_set_batch(int kind, int pairs, int log2m, int size_class, int shape, int rank);
ms_status ms_tune_get_batch(int kind, int pairs, int log2m, int size_class, int *shape, int *rank);

/* Human-readable name of a status code (static storage). */
const char *ms_status_string(ms_status s);

/* Library version string (static storage). */
const char *ms_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MS_H_ */
