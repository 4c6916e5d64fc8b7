// ms_scan.cuh -- the global stage (Section 4.3, Alg. 1 "Scan stage"): one
// exclusive prefix sum over the row-vectorised histogram matrix
//   H_row = [H[0][0..G-1], H[1][0..G-1], ..., H[m-1][0..G-1]],
// computed in a single pass with decoupled look-back (Merrill and Garland,
// "Single-pass parallel prefix scan with decoupled look-back", 2016): each CTA
// takes the next tile by ticket, publishes its aggregate, walks back over its
// predecessors' published values until it meets an inclusive prefix, then
// publishes its own inclusive prefix.  The result G_row[b * G + c] is the
// first two terms of Eq. 2 for bucket b and chunk c.  (Alg. 1 as printed reads
// G_row[i * m + j]; with m rows of length G the element is G_row[i * G + j].)
//
// Every wait on a predecessor is bounded; when the bound is reached the CTA
// records MS_ERR_TIMEOUT in the device status word and carries on with a zero
// contribution, so the kernel always ends.
#pragma once

#include "ms_device.cuh"

namespace ms {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr unsigned long long kFlagAggregate = 1ull << 32;
constexpr unsigned long long kFlagPrefix = 2ull << 32;
constexpr uint32_t kSpinLimit = 1u << 20;

struct ScanArgs {
  uint32_t* data;                // in: H_row, out: exclusive prefix (in place)
  uint32_t len;                  // m * G
  uint32_t G;                    // row length
  uint32_t* offsets;             // optional: offsets[b] = prefix at b * G, offsets[m] = total
  uint32_t m;
  unsigned long long* status;    // one word per scan tile, zeroed before the launch
  uint32_t* ticket;              // zeroed before the launch
  uint32_t* err;                 // device status word
};

// Waits (bounded) until the status word at p carries a flag; returns it.
__device__ __forceinline__ unsigned long long wait_status(const unsigned long long* p, uint32_t* err) {
  unsigned long long v = ld_relaxed_u64(p);
  uint32_t spins = 0;
  while ((v >> 32) == 0) {
    // give up at the bound, or at once when another wait has already given up
    if (++spins > kSpinLimit || (spins > 64 && (*(volatile uint32_t*)err & kDevErrTimeout))) {
      atomicOr(err, kDevErrTimeout);
      return kFlagPrefix;  // value 0, treated as a prefix: stop looking back
    }
    __nanosleep(spins < 64 ? 32 : 256);
    v = ld_relaxed_u64(p);
  }
  return v;
}

// Launches the look-back scan over a.len entries (stream-ordered); the status
// words and the ticket must be zero.  Defined in ms_scan.cu.
cudaError_t launch_scan_lookback(const ScanArgs& a, cudaStream_t stream);

// Launches exactly `ctas` CTAs of the same kernel (failure-path test aid).
cudaError_t launch_scan_tiles(const ScanArgs& a, uint32_t ctas, cudaStream_t stream);

}  // namespace ms
