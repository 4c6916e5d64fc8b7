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

// Bits of the per-device status word.
constexpr uint32_t kDevErrTimeout = 1u;  // a bounded wait expired
constexpr uint32_t kDevErrBounds = 2u;   // an index failed its bounds check (the access was skipped)

enum Kind : int { kRange = 0, kDelta = 1, kRadix = 2, kMod = 3 };

// Bucket identifier parameters as the kernels see them (built by the host
// from an ms_bucket_spec).
struct DevSpec {
  uint32_t m;                 // 1..256
  uint32_t nbits;             // ceil(log2 m); 0 when m == 1
  const uint32_t* splitters;  // kRange: m-1 nondecreasing values (device)
  float x0, delta;            // kDelta
  uint32_t shift, mask;       // kRadix: shift < 32
  uint32_t mod_magic, mod_sh1, mod_sh2;  // kMod: multiply-shift constants
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Range splitters go to shared memory as a table of 2^nbits - 1 entries
// padded with 0xffffffff, so the search below needs no bounds test.
__device__ __forceinline__ void load_splitter_table(const DevSpec& sp, uint32_t* tbl) {
  const uint32_t P = 1u << sp.nbits;
  for (uint32_t i = threadIdx.x; i + 1 < P; i += blockDim.x)
    tbl[i] = (i + 1 < sp.m) ? sp.splitters[i] : 0xffffffffu;
}

// f(u) for the bucket kind KIND.
template <int KIND>
__device__ __forceinline__ uint32_t bucket_of(uint32_t u, const DevSpec& sp, const uint32_t* tbl) {
  if constexpr (KIND == kRange) {
    // number of table entries <= u, by halving steps over a table of
    // 2^nbits - 1 sorted entries; the padding only counts when u is
    // 0xffffffff, and the clamp to m-1 absorbs it.
    uint32_t pos = 0;
    for (uint32_t h = (1u << sp.nbits) >> 1; h > 0; h >>= 1) pos += (tbl[pos + h - 1] <= u) ? h : 0u;
    return min(pos, sp.m - 1);
  } else if constexpr (KIND == kDelta) {
    const float x = __uint_as_float(u);
    const float q = __fdiv_rn(__fsub_rn(x, sp.x0), sp.delta);  // IEEE round-to-nearest
    const float f = floorf(q);
    if (!(f < (float)sp.m)) return sp.m - 1;  // f >= m, +inf, NaN
    if (f <= 0.0f) return 0u;                 // negative, -0, -inf
    return (uint32_t)f;
  } else if constexpr (KIND == kRadix) {
    return (u >> sp.shift) & sp.mask;
  } else {
    // u mod m by the multiply-shift division of Granlund and Montgomery
    // ("Division by invariant integers using multiplication", PLDI 1994,
    // unsigned case): q = (t + ((u - t) >> sh1)) >> sh2 with t = mulhi(M, u).
    const uint32_t t = __umulhi(sp.mod_magic, u);
    const uint32_t q = (t + ((u - t) >> sp.mod_sh1)) >> sp.mod_sh2;
    return u - q * sp.m;
  }
}

// Ballot-based voting of one 32-key window (Section 5.4): after the loop,
// `own` holds the valid lanes whose bucket equals this lane's bucket b, and
// `lane_bm` the valid lanes whose bucket equals this lane's id (Alg. 2; only
// meaningful for lane ids < m <= 32).
template <int MAXBITS>
__device__ __forceinline__ void window_vote(uint32_t b, bool valid, uint32_t nbits, uint32_t& own,
                                            uint32_t& lane_bm) {
  const uint32_t vb = __ballot_sync(kFull, valid);
  const uint32_t lane = lane_id();
  own = vb;
  lane_bm = vb;
#pragma unroll
  for (int k = 0; k < MAXBITS; ++k) {
    if (k < (int)nbits) {
      const uint32_t bal = __ballot_sync(kFull, (b >> k) & 1u);
      own &= ((b >> k) & 1u) ? bal : ~bal;
      lane_bm &= ((lane >> k) & 1u) ? bal : ~bal;
    }
  }
}

// Same voting, `own` only (buckets up to 256: eight ballots).
__device__ __forceinline__ uint32_t window_peers(uint32_t b, bool valid, uint32_t nbits) {
  uint32_t own = __ballot_sync(kFull, valid);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < (int)nbits) {
      const uint32_t bal = __ballot_sync(kFull, (b >> k) & 1u);
      own &= ((b >> k) & 1u) ? bal : ~bal;
    }
  }
  return own;
}

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
