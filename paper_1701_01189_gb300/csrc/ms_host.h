// ms_host.h -- host-side internals shared by the C ABI and the per-kind
// launcher translation units (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ms_device.cuh"

namespace ms {

// Per-device state, created on the first call made with that device current.
struct DeviceCtx {
  int device = -1;
  int sm_count = 0;
  cudaMemPool_t pool = nullptr;  // library-owned stream-ordered pool for scratch
  uint32_t* d_err = nullptr;     // device status word (MS_OK or MS_ERR_TIMEOUT)
};

// One multisplit request, validated, in kernel terms.
struct Call {
  const uint32_t* keys_in;
  const uint32_t* vals_in;  // nullptr: keys only
  uint32_t* keys_out;
  uint32_t* vals_out;
  uint32_t* offsets;        // nullptr: not wanted
  uint32_t n;
  int kind;
  DevSpec sp;
  cudaStream_t stream;
  void* ws_fixed;        // non-null: caller-provided scratch of ws_capacity bytes (no allocation, no tracing)
  size_t ws_capacity;
  uint32_t* counts;      // non-null: histogram only -- counts[b] for b < m, no permutation (ms_histogram)
};

// Kernel variant of one multisplit: post-scan tile shape (0: 8 warps x 16
// keys, 1: 16 x 8, 2: 8 x 8), rank mode (kRankBallot only for m <= 8,
// kRankTable) and whether the tile is reordered before the writes.
struct Variant {
  int shape;
  int rank;
  int reorder;
};

// Size class of n for tuning: 0: < 2^16, 1: < 2^20, 2: < 2^24, 3: larger.
int size_class(uint32_t n);
// The tuned (or default) variant for a request (ms_tune.cu).
Variant choose_variant(const Call& c);
// The tuned (or default) kernel of a batched plan for its identifier and mean
// segment length: rank kRankThread (k_batch_tc, m <= 32), kRankTable or
// kRankVote (k_batch) and, for k_batch, the tile shape (0: 8 warps x 16 keys,
// 1: 16 warps x 8 keys) (ms_tune.cu).
Variant choose_batch_variant(int kind, bool pairs, uint32_t nbits, uint64_t mean_n);
// How the radix sort makes its passes: 0 one-sweep kernels, 1 three-stage
// multisplits with the radix-digit identifier (ms_tune.cu).
int choose_sort_method(uint32_t n, bool pairs);

// Runs the three stages for one request.  Defined per bucket kind in
// ms_kind_<kind>.cu.
cudaError_t run_multisplit_range(const Call& c, DeviceCtx& ctx);
cudaError_t run_multisplit_delta(const Call& c, DeviceCtx& ctx);
cudaError_t run_multisplit_radix(const Call& c, DeviceCtx& ctx);
cudaError_t run_multisplit_mod(const Call& c, DeviceCtx& ctx);

cudaError_t run_multisplit(const Call& c, DeviceCtx& ctx);

// Stage timing (ms_trace.cu): trace_begin records the start event and returns
// a slot (-1 when timing is off); trace_mark records event `stage` (1..3).
int trace_begin(cudaStream_t s);
void trace_mark(int slot, int stage, cudaStream_t s);

// Shared argument handling of the C ABI (ms_api.cu).
}  // namespace ms
#include "ms.h"
namespace ms {
ms_status to_status(cudaError_t e);
ms_status make_devspec(const ms_bucket_spec* spec, DevSpec* out, int* kind);
bool overlap(const void* a, const void* b, size_t bytes);
// The calling device's state, created on first use (allocates: not inside a capture).
ms_status current_device_ctx(DeviceCtx** out);

// An identifier with 257 .. 2^16 buckets (ms_wide.cu): the kernel kind of its
// digit passes (kWide, or kRadix for a radix digit of 9..16 bits), its bucket
// count fm, its super-bucket count mc = ceil(fm / 256), and the kernel spec of
// the whole bucket id (dshift 0, every bit kept).
struct WideSpec {
  int kind;
  uint32_t fm, mc;
  DevSpec full;
};
ms_status make_wide_spec(const ms_bucket_spec* spec, WideSpec* out);
// Stable multisplit by a wide identifier: two digit passes through a pool
// buffer, then the bucket offsets (c.offsets, fm + 1 entries, if not null).
cudaError_t run_wide(const Call& c, const WideSpec& w, DeviceCtx& ctx);

// LSD radix sort with one sweep per digit (ms_onesweep.cu); n < 2^30.
cudaError_t run_onesweep_sort(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t n, int begin_bit, int end_bit,
                              uint32_t* keys_out, uint32_t* vals_out, cudaStream_t s, DeviceCtx& ctx);

// Batch plans alive on a device, not counting the library's own cached plans
// of ms_multisplit_pairs_batched (ms_batch.cu), and the release of those.
int batch_live_plans(int dev);
void batch_cache_release(int dev);
// Releases the stage-timing events (ms_trace.cu).
void trace_release();

// Scratch from the library pool, ordered on `stream`.
cudaError_t scratch_alloc(DeviceCtx& ctx, void** p, size_t bytes, cudaStream_t stream);
cudaError_t scratch_free(void* p, cudaStream_t stream);

}  // namespace ms
