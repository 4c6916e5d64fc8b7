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

// Eq. 2 for chunk c from the chunk-major histograms H[c' * mp + b] (rows of
// mp words, mp a power of two with m <= mp <= 32 and 4 <= mp, zero beyond m):
// end[b] = (keys of buckets < b) + (keys of bucket b in chunks c' <= c), the
// end of bucket b's share of chunk c in the output; CTA 0 also writes the
// m + 1 bucket starts.  The first 256 threads read H as 16-byte vectors (a
// vector is 4 buckets of one chunk; consecutive threads, consecutive
// vectors), so a thread always sums the same 4 buckets; the sums are reduced
// over the lanes, then over the warps, and warp 0 scans the bucket totals.
// All threads of the block (>= 256) call it; s_scr: 2 * 8 * 32 words of
// scratch (end: m words).  Ends with a block barrier.
__device__ __forceinline__ void chunk_offsets(const uint32_t* H, uint32_t G, uint32_t m, uint32_t mp, uint32_t c,
                                              uint32_t* end, uint32_t* s_scr, uint32_t* offsets) {
  const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5;
  const uint32_t q = mp >> 2;                        // vectors per row: 1, 2, 4 or 8
  const uint32_t lq = q >= 8u ? 3u : q >= 4u ? 2u : q >= 2u ? 1u : 0u;
  const uint32_t b0 = (t & (q - 1u)) << 2;           // this thread's buckets b0 .. b0 + 3
  uint32_t inc[4] = {0u, 0u, 0u, 0u}, all[4] = {0u, 0u, 0u, 0u};
  if (t < 256u) {
    const uint32_t nvec = G * q;
    const uint4* hv = reinterpret_cast<const uint4*>(H);
#pragma unroll 16
    for (uint32_t i = t; i < nvec; i += 256u) {
      const uint4 v = __ldcg(hv + i);
      const bool le = (i >> lq) <= c;
      all[0] += v.x;
      all[1] += v.y;
      all[2] += v.z;
      all[3] += v.w;
      inc[0] += le ? v.x : 0u;
      inc[1] += le ? v.y : 0u;
      inc[2] += le ? v.z : 0u;
      inc[3] += le ? v.w : 0u;
    }
  }
  // lanes equal modulo q hold the same buckets
#pragma unroll
  for (uint32_t d = 16u; d > 0u; d >>= 1) {
    if (d >= q) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        all[k] += __shfl_xor_sync(kFull, all[k], d);
        inc[k] += __shfl_xor_sync(kFull, inc[k], d);
      }
    }
  }
  if (t < 256u && lane < q) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      s_scr[w * 32u + b0 + k] = inc[k];
      s_scr[256u + w * 32u + b0 + k] = all[k];
    }
  }
  __syncthreads();
  if (t < 32u) {
    uint32_t tot = 0, incs = 0;
    if (t < mp) {
#pragma unroll
      for (uint32_t k = 0; k < 8u; ++k) {
        incs += s_scr[k * 32u + t];
        tot += s_scr[256u + k * 32u + t];
      }
    }
    uint32_t x = tot;  // inclusive scan of the bucket totals over the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, d);
      if (t >= (uint32_t)d) x += y;
    }
    const uint32_t start = x - tot;
    if (t < m) end[t] = start + incs;
    if (c == 0u && offsets != nullptr) {
      if (t < m) offsets[t] = start;
      if (t == m - 1u) offsets[m] = x;
    }
  }
  __syncthreads();
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
