// ms_bucket.cuh -- bucket identifiers as the kernels evaluate them (Section 6
// "Bucket identification", Section 7.1 radix digit, Section 7.3 even / range
// histogram).
//
// Range splitters (binary search over splitters, Section 7.3) are the costly
// identifier: ceil(log2 m) dependent compare-and-select steps per key.  On
// GB300 the SMs have about 22 bytes of HBM bandwidth per cycle to keep up
// with, so the search is replaced by a lookup table in shared memory indexed
// by the top LB bits of the key: each cell stores the bucket of its first key
// and the one splitter inside the cell, if any; cells holding two or more
// splitters are flagged and fall back to the full search.  The result equals
// the search for every key (both count the splitters <= u).
#pragma once

#include "ms_device.cuh"

namespace ms {

constexpr uint32_t kLutFlag = 0x80000000u;

// Number of splitters <= u in the sorted table tbl[0 .. 2^NB - 2] (padded with
// 0xffffffff), clamped to m-1.  NB halving steps.
template <int NB>
__device__ __forceinline__ uint32_t range_search(uint32_t u, const uint32_t* tbl, uint32_t m) {
  uint32_t pos = 0;
#pragma unroll
  for (int s = NB - 1; s >= 0; --s) {
    const uint32_t h = 1u << s;
    pos += (tbl[pos + h - 1] <= u) ? h : 0u;
  }
  return min(pos, m - 1);
}

// Table of the super-bucket splitters of a wide range identifier: entry i is
// s_{256(i+1)}, the first splitter of super-bucket i+1 (mc - 1 of them),
// padded with 0xffffffff to 2^NB - 1 entries.  The count of these <= u is
// floor(f(u) / 256): with nondecreasing splitters, f(u) >= 256 j exactly when
// s_{256 j} <= u.  No barrier.
template <int NB>
__device__ __forceinline__ void build_wide_table(const DevSpec& sp, uint32_t* tbl) {
  constexpr uint32_t P = (1u << NB) - 1u;
  if (sp.base == kRange)
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
      tbl[i] = (i + 1u < sp.mc) ? sp.splitters[256u * (i + 1u) - 1u] : 0xffffffffu;
}

// f(u) of a wide identifier (fm > 256 buckets) and then its digit
// (f(u) >> dshift) & dmask.  Range: the super-bucket S from the table of
// build_wide_table, then a bisection over the at most 255 splitters inside S
// (s_{256S+1} ..), read through the read-only cache.  Delta and mod as for
// 256 buckets or fewer, with fm buckets.
template <int NB>
__device__ __forceinline__ uint32_t wide_bucket(uint32_t u, const DevSpec& sp, const uint32_t* tbl) {
  uint32_t b;
  if (sp.base == kRange) {
    uint32_t S = 0;
    if constexpr (NB > 0) S = range_search<NB>(u, tbl, sp.mc);
    const uint32_t* blk = sp.splitters + 256u * S;
    const uint32_t cnt = min(255u, sp.fm - 1u - 256u * S);
    uint32_t pos = 0;
#pragma unroll
    for (int s = 7; s >= 0; --s) {
      const uint32_t h = 1u << s, i = pos + h - 1u;
      pos += (i < cnt && __ldg(blk + i) <= u) ? h : 0u;
    }
    b = 256u * S + pos;
  } else if (sp.base == kDelta) {
    const float x = __uint_as_float(u);
    const float f = floorf(__fdiv_rn(__fsub_rn(x, sp.x0), sp.delta));
    b = !(f < (float)sp.fm) ? sp.fm - 1u : (f <= 0.0f ? 0u : (uint32_t)f);
  } else {
    const uint32_t t = __umulhi(sp.mod_magic, u);
    const uint32_t q = (t + ((u - t) >> sp.mod_sh1)) >> sp.mod_sh2;
    b = u - q * sp.fm;
  }
  return (b >> sp.dshift) & sp.dmask;
}

// Builds the splitter table (2^NB - 1 words) and, for range buckets, the
// lookup table of 2^lb cells (uint2 each).  All threads of the block call it;
// ends with a block barrier.
template <int KIND, int NB>
__device__ __forceinline__ void build_bucket_tables(const DevSpec& sp, uint32_t* tbl, uint2* lut) {
  if constexpr (KIND == kWide) build_wide_table<NB>(sp, tbl);
  if constexpr (KIND == kRange) {
    const uint32_t P = 1u << NB;
    for (uint32_t i = threadIdx.x; i + 1 < P; i += blockDim.x)
      tbl[i] = (i + 1 < sp.m) ? sp.splitters[i] : 0xffffffffu;
    __syncthreads();
    const uint32_t cells = 1u << sp.lut_bits;
    const uint32_t sh = 32u - sp.lut_bits;
    for (uint32_t cidx = threadIdx.x; cidx < cells; cidx += blockDim.x) {
      const uint32_t first = cidx << sh;
      const uint32_t last = first | ((1u << sh) - 1u);
      // lo = splitters < first; hi = splitters <= last (m-1 real splitters)
      const uint32_t lo = (first == 0u) ? 0u : range_search<NB>(first - 1u, tbl, sp.m + 1);
      const uint32_t hi = range_search<NB>(last, tbl, sp.m + 1);
      const uint32_t lo_c = min(lo, sp.m - 1), hi_c = min(hi, sp.m - 1);
      const uint32_t cnt = hi_c - lo_c;
      uint2 e;
      if (cnt == 0u) {
        // no splitter in the cell: bucket lo for every key in it
        e = (lo_c == 0u) ? make_uint2(0u, 0xffffffffu) : make_uint2(lo_c - 1u, 0u);
      } else if (cnt == 1u) {
        e = make_uint2(lo_c, tbl[lo_c]);
      } else {
        e = make_uint2(kLutFlag, 0u);
      }
      lut[cidx] = e;
    }
  }
  __syncthreads();
}

// f(u).  For kRange the tables of build_bucket_tables must be in place.
template <int KIND, int NB>
__device__ __forceinline__ uint32_t bucket_of(uint32_t u, const DevSpec& sp, const uint32_t* tbl,
                                              const uint2* lut) {
  if constexpr (KIND == kRange) {
    if constexpr (NB == 0) {
      return 0u;
    } else {
      const uint2 e = lut[u >> (32u - sp.lut_bits)];
      uint32_t b = e.x + (u >= e.y ? 1u : 0u);
      if (e.x & kLutFlag) b = range_search<NB>(u, tbl, sp.m);
      return b;
    }
  } else if constexpr (KIND == kDelta) {
    const float x = __uint_as_float(u);
    const float q = __fdiv_rn(__fsub_rn(x, sp.x0), sp.delta);  // IEEE round-to-nearest
    const float f = floorf(q);
    if (!(f < (float)sp.m)) return sp.m - 1;  // f >= m, +inf, NaN
    if (f <= 0.0f) return 0u;                 // negative, -0, -inf
    return (uint32_t)f;
  } else if constexpr (KIND == kRadix) {
    return (u >> sp.shift) & sp.mask;
  } else if constexpr (KIND == kWide) {
    return wide_bucket<NB>(u, sp, tbl);
  } else {
    // u mod m by the multiply-shift division of Granlund and Montgomery
    // ("Division by invariant integers using multiplication", PLDI 1994,
    // unsigned case): q = (t + ((u - t) >> sh1)) >> sh2 with t = mulhi(M, u).
    const uint32_t t = __umulhi(sp.mod_magic, u);
    const uint32_t q = (t + ((u - t) >> sp.mod_sh1)) >> sp.mod_sh2;
    return u - q * sp.m;
  }
}

}  // namespace ms
