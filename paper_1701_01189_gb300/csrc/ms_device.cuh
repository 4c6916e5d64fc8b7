// ms_device.cuh -- device-side building blocks of the multisplit kernels (sm_103a).
//
// Bucket identifiers (Section 6 "Bucket identification", Section 7.1 radix
// digit, Section 7.3 range / even histogram), and the warp-level direct solve
// of Section 5.5: per 32-key window, ceil(log2 m) ballots give every lane the
// bucket of every other lane (Section 5.4 "ballot-based voting"), from which a
// lane derives
//   * the histogram of the bucket equal to its lane id (Alg. 2), and
//   * the local offset of its own key among the earlier lanes of the same
//     bucket.  Alg. 3 as printed tests the bits of the lane id; the text of
//     Section 5.5.2 says the lane compares against its own key's bucket, which
//     is what is done here.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ms {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kMaxM = 256;
// Identifiers with more buckets (up to 2^16) run as two passes over the
// digits of the bucket id (kWide).
constexpr uint32_t kMaxWideM = 65536;

// Bits of the per-device status word.
constexpr uint32_t kDevErrTimeout = 1u;  // a bounded wait expired
constexpr uint32_t kDevErrBounds = 2u;   // an index failed its bounds check (the access was skipped)

// kWide: one 8-bit digit of the bucket id of an identifier with more than 256
// buckets (its kind in DevSpec::base), least significant digit first.
enum Kind : int { kRange = 0, kDelta = 1, kRadix = 2, kMod = 3, kWide = 4 };

// How the post-scan ranks keys: ballot voting or peer tables inside each
// warp, per-thread bucket counters (m <= 32; ms_tc.cuh), or peers found by
// ballots with per-warp bucket counters in shared memory (any m).
enum RankMode : int { kRankBallot = 0, kRankTable = 1, kRankThread = 2, kRankVote = 3 };

// Bucket identifier parameters as the kernels see them (built by the host
// from an ms_bucket_spec).
struct DevSpec {
  uint32_t m;                 // 1..256
  uint32_t nbits;             // ceil(log2 m); 0 when m == 1
  const uint32_t* splitters;  // kRange: m-1 nondecreasing values (device)
  float x0, delta;            // kDelta
  float rdelta;               // kDelta: 1 / delta rounded to binary32 (the fast path of delta_bucket)
  uint32_t shift, mask;       // kRadix: shift < 32
  uint32_t mod_magic, mod_sh1, mod_sh2;  // kMod: multiply-shift constants
  uint32_t m_pad;             // m rounded up to a multiple of 32 (at least 32)
  uint32_t lut_bits;          // kRange: key bits indexing the splitter lookup table
  // kWide only: the identifier is `base` (kRange, kDelta or kMod) with fm
  // buckets (257 .. 2^16; for kRange fm-1 splitters and mc = ceil(fm / 256)
  // super-buckets), and the kernel's bucket is (f(u) >> dshift) & dmask.
  uint32_t base, fm, mc, dshift, dmask;
  const uint32_t* wlut;  // kWide range: global lookup table of 2^wlb cells (ms_bucket.cuh)
  uint32_t wlb;
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Exclusive prefix sum over the first `count` threads of the block (count <=
// 32 * number of warps); every thread passes v (0 beyond count).  Returns the
// exclusive prefix; *total gets the sum.  Uses s_warp (one word per warp) and
// two block barriers; all threads of the block must call it.
template <int NW>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  uint32_t wpre = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const uint32_t s = s_warp[i];
    wpre += (i < (int)w) ? s : 0u;
    tot += s;
  }
  *total = tot;
  __syncthreads();  // s_warp may be reused right after
  return wpre + x - v;
}

// Programmatic dependent launch: a kernel lets the next one in the stream
// start early (launch_dependents); the dependent kernel waits for the earlier
// grid to complete, and its writes to be visible, before reading its results.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Relaxed 64-bit loads and stores at GPU scope for look-back status words
// (flag in the high half, value in the low half, so a reader never sees a
// flag without its value).
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

}  // namespace ms
