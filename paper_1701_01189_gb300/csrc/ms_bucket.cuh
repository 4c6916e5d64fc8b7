// ms_bucket.cuh -- bucket identifiers as the kernels evaluate them (Section 6
// "Bucket identification", Section 7.1 radix digit, Section 7.3 even / range
// histogram).
//
// Range splitters (binary search over splitters, Section 7.3) are the costly
// identifier: ceil(log2 m) dependent compare-and-select steps per key.  On
// GB300 the SMs have about 22 bytes of HBM bandwidth per cycle to keep up
// with, so the search is replaced by a lookup table in shared memory indexed
// by the top lb bits of the key: each cell stores the bucket of its first key
// and the one splitter inside the cell, if any; a cell holding two or more
// splitters is flagged and stores how many, and its keys compare against
// those few splitters directly (the full search only past kCellScan of them).
// The result equals the search for every key (both count the splitters <= u).
#pragma once

#include "ms_device.cuh"

namespace ms {

// A flagged cell with at most this many splitters resolves its keys by that
// many independent compares; more take the full search.
constexpr uint32_t kCellScan = 4;

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

// Packed splitter lookup table: 2^lb cells of the key space (its top lb
// bits), one 32-bit word each --
//   bits 0 .. BB-1  lo, the bucket of the cell's first key (m <= 2^BB);
//   bit BB          flag: the cell holds two or more splitters;
//   bits BB+1 ..    unflagged: the low 32 - lb bits of the cell's splitter, or
//                   2^(32-lb) (above every key of the cell) when it holds none;
//                   flagged: the number of splitters in the cell (at most 255)
// -- stored W = 2^lw times side by side (lane l reads copy l mod W).  Needs
// lb >= BB + 2.  tbl (the splitter table, 2^BB - 1 entries padded with
// 0xffffffff) must be in place.  All threads of the block call it; no
// barrier after the last writes.
template <int BB>
__device__ __forceinline__ void build_packed_lut(const DevSpec& sp, uint32_t lb, uint32_t lw, const uint32_t* tbl,
                                                 uint32_t* lut) {
  const uint32_t sh = 32u - lb, fmask = (1u << sh) - 1u, W = 1u << lw, cells = 1u << lb;
  if constexpr (BB <= 5) {
    // up to 32 buckets: two short bisections per cell (lo = splitters below the
    // cell's first key, hi = splitters up to its last key)
    for (uint32_t cell = threadIdx.x; cell < cells; cell += blockDim.x) {
      const uint32_t first = cell << sh, last = first | fmask;
      const uint32_t lo = min(first == 0u ? 0u : range_search<BB>(first - 1u, tbl, sp.m + 1u), sp.m - 1u);
      const uint32_t hi = min(range_search<BB>(last, tbl, sp.m + 1u), sp.m - 1u);
      uint32_t e;
      if (hi == lo)
        e = lo | ((fmask + 1u) << (BB + 1));
      else if (hi == lo + 1u)
        e = lo | ((tbl[lo] & fmask) << (BB + 1));
      else
        e = lo | (1u << BB) | (min(hi - lo, 255u) << (BB + 1));
      for (uint32_t r = 0; r < W; ++r) lut[(cell << lw) + r] = e;
    }
    return;
  }
  // more buckets: lo of a cell = the splitters of the cells before it -- count
  // the splitters per cell (in copy 0 of each cell), then one exclusive scan
  // over the cells.  Thread t takes cells [t * per, (t+1) * per) (cells a
  // multiple of blockDim.x).
  __shared__ uint32_t s_lut_warp[32];
  for (uint32_t c = threadIdx.x; c < cells; c += blockDim.x) lut[c << lw] = 0u;
  __syncthreads();
  for (uint32_t k = threadIdx.x; k + 1u < sp.m; k += blockDim.x) atomicAdd(lut + ((tbl[k] >> sh) << lw), 1u);
  __syncthreads();
  const uint32_t per = cells / blockDim.x, c0 = threadIdx.x * per;
  uint32_t sum = 0;
  for (uint32_t i = 0; i < per; ++i) sum += lut[(c0 + i) << lw];
  // exclusive scan of the per-thread sums over the block
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  uint32_t x = sum;
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31u) s_lut_warp[wid] = x;
  __syncthreads();
  uint32_t lo = x - sum;
  for (uint32_t i = 0; i < wid; ++i) lo += s_lut_warp[i];
  for (uint32_t i = 0; i < per; ++i) {
    const uint32_t cnt = lut[(c0 + i) << lw];  // read before the cell's words are written
    uint32_t e;
    if (cnt == 0u)
      e = lo | ((fmask + 1u) << (BB + 1));
    else if (cnt == 1u)
      e = lo | ((tbl[lo] & fmask) << (BB + 1));
    else
      e = lo | (1u << BB) | (min(cnt, 255u) << (BB + 1));
    for (uint32_t r = 0; r < W; ++r) lut[((c0 + i) << lw) + r] = e;
    lo += cnt;
  }
}

// Bucket of u from its cell's word e when the cell is not flagged.
template <int BB>
__device__ __forceinline__ uint32_t packed_fast(uint32_t u, uint32_t e, uint32_t fmask) {
  return (e & ((1u << BB) - 1u)) + ((u & fmask) >= (e >> (BB + 1)) ? 1u : 0u);
}

// Bucket of u in a flagged cell (word e): lo plus the cell's splitters <= u,
// which are tbl[lo .. lo + count - 1].
template <int BB>
__device__ __forceinline__ uint32_t range_in_cell(uint32_t u, uint32_t e, const uint32_t* tbl, uint32_t m) {
  const uint32_t lo = e & ((1u << BB) - 1u), cnt = e >> (BB + 1);
  if (cnt > kCellScan) return range_search<BB>(u, tbl, m);
  uint32_t b = lo;
#pragma unroll
  for (uint32_t k = 0; k < kCellScan; ++k) b += (k < cnt && tbl[lo + k] <= u) ? 1u : 0u;
  return b;
}

// Delta bucket: floor((x - x0) / delta) with binary32 round-to-nearest
// subtraction and division, clamped into [0, m-1] (NaN -> m-1).
// Fast path without the division: with r = delta^-1 rounded, q' = (x - x0) r
// rounded is q (1 + e1)(1 + e2) for the exact quotient q, |e1|, |e2| <= 2^-24,
// so it lies within 3.01 |q'| 2^-24 of the rounded quotient fl(q); when q' is
// farther than q' 2^-22 from every integer (and inside (0, m)), floor(fl(q))
// is floor(q').  Keys near a bucket edge, negative, infinite or NaN take the
// division.
__device__ __forceinline__ uint32_t delta_bucket(uint32_t u, float x0, float delta, float rdelta, uint32_t m) {
  const float d = __fsub_rn(__uint_as_float(u), x0);
  const float qa = __fmul_rn(d, rdelta);
  const float k = floorf(qa);
  const float fr = __fsub_rn(qa, k);            // exact: qa and k are within a factor of two (or k = 0)
  const float eps = __fmul_rn(qa, 0x1p-22f);  // exact: a power of two
  if (qa > 0.0f && qa < (float)m && fr > eps && __fsub_rn(1.0f, fr) > eps) return (uint32_t)k;
  const float f = floorf(__fdiv_rn(d, delta));  // IEEE round-to-nearest
  if (!(f < (float)m)) return m - 1u;           // f >= m, +inf, NaN
  if (f <= 0.0f) return 0u;                     // negative, -0, -inf
  return (uint32_t)f;
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

// Global lookup table of a wide range identifier (kWideLutFlag and the
// k_wide_lut kernel that builds it): 2^wlb cells of the key space, one word
// each -- bits 0..15 the bucket of the cell's first key, bit 16 flag (two or
// more splitters in the cell), from bit 17 the low 32 - wlb bits of the cell's
// one splitter (2^(32-wlb) when it holds none) or, flagged, the number of
// its splitters (at most 255).  18 <= wlb <= 20 (at most 4 MB, in L2).
constexpr uint32_t kWideLutFlag = 1u << 16;

// f(u) of a wide identifier (fm > 256 buckets) and then its digit
// (f(u) >> dshift) & dmask.  Range: the cell's word in the global lookup
// table; keys of a flagged cell compare against its few splitters, or past
// kCellScan of them take the super-bucket S from the table of
// build_wide_table and a bisection over the at most 255 splitters inside S
// (s_{256S+1} ..), read through the read-only cache.  Delta and mod as for
// 256 buckets or fewer, with fm buckets.
template <int NB>
__device__ __forceinline__ uint32_t wide_bucket(uint32_t u, const DevSpec& sp, const uint32_t* tbl) {
  uint32_t b;
  if (sp.base == kRange) {
    const uint32_t sh = 32u - sp.wlb, e = __ldg(sp.wlut + (u >> sh));
    const uint32_t lo = e & 0xffffu, f = e >> 17;  // f: the splitter's low bits, or the count if flagged
    if (!(e & kWideLutFlag)) {
      b = lo + ((u & ((1u << sh) - 1u)) >= f ? 1u : 0u);
    } else if (f <= kCellScan) {
      const uint32_t cnt = f;
      b = lo;
#pragma unroll
      for (uint32_t k = 0; k < kCellScan; ++k) b += (k < cnt && __ldg(sp.splitters + lo + k) <= u) ? 1u : 0u;
    } else {
      // more splitters in the cell: super-bucket, then a bisection inside it
      uint32_t S = 0;
      if constexpr (NB > 0) S = range_search<NB>(u, tbl, sp.mc);
      const uint32_t* blk = sp.splitters + 256u * S;
      const uint32_t n_in = min(255u, sp.fm - 1u - 256u * S);
      uint32_t pos = 0;
#pragma unroll
      for (int s = 7; s >= 0; --s) {
        const uint32_t h = 1u << s, i = pos + h - 1u;
        pos += (i < n_in && __ldg(blk + i) <= u) ? h : 0u;
      }
      b = 256u * S + pos;
    }
  } else if (sp.base == kDelta) {
    // always the division: with up to 2^16 buckets the edge margin of
    // delta_bucket's fast path catches enough keys that most warps run both
    const float f = floorf(__fdiv_rn(__fsub_rn(__uint_as_float(u), sp.x0), sp.delta));
    b = !(f < (float)sp.fm) ? sp.fm - 1u : (f <= 0.0f ? 0u : (uint32_t)f);
  } else {
    const uint32_t t = __umulhi(sp.mod_magic, u);
    const uint32_t q = (t + ((u - t) >> sp.mod_sh1)) >> sp.mod_sh2;
    b = u - q * sp.fm;
  }
  return (b >> sp.dshift) & sp.dmask;
}

// Identifiers whose bucket the post-scans recompute from the reordered key at
// write-out instead of storing a bucket byte per position (a scattered
// shared-memory store and a load).  The radix digit costs two ALU
// instructions: 4-9% faster sorts on GB300.  The modulo bucket costs a
// multiply-high, a multiply and a subtract: recomputing it is 4% faster for
// key-value pairs with 32 or 64 buckets and no faster for keys alone.  For
// delta buckets the recomputation was up to 9% slower, so they keep the byte.
template <int KIND, bool PAIRS>
__host__ __device__ constexpr bool cheap_bucket() {
  return KIND == kRadix || (PAIRS && KIND == kMod);
}

// Builds the splitter table (2^NB - 1 words) and, for range buckets, the
// packed lookup table of 2^(lut_bits + 1) cells, one copy.  All threads of
// the block call it; ends with a block barrier.
template <int KIND, int NB>
__device__ __forceinline__ void build_bucket_tables(const DevSpec& sp, uint32_t* tbl, uint32_t* lut) {
  if constexpr (KIND == kWide) build_wide_table<NB>(sp, tbl);
  if constexpr (KIND == kRange) {
    const uint32_t P = 1u << NB;
    for (uint32_t i = threadIdx.x; i + 1 < P; i += blockDim.x)
      tbl[i] = (i + 1 < sp.m) ? sp.splitters[i] : 0xffffffffu;
    __syncthreads();
    if constexpr (NB > 0) build_packed_lut<NB>(sp, sp.lut_bits + 1u, 0u, tbl, lut);
  }
  __syncthreads();
}

// f(u).  For kRange the tables of build_bucket_tables must be in place.
template <int KIND, int NB>
__device__ __forceinline__ uint32_t bucket_of(uint32_t u, const DevSpec& sp, const uint32_t* tbl,
                                              const uint32_t* lut) {
  if constexpr (KIND == kRange) {
    if constexpr (NB == 0) {
      return 0u;
    } else {
      const uint32_t sh = 31u - sp.lut_bits;  // lut_bits + 1 key bits index the cells
      const uint32_t e = lut[u >> sh];
      if (e & (1u << NB)) return range_in_cell<NB>(u, e, tbl, sp.m);
      return packed_fast<NB>(u, e, (1u << sh) - 1u);
    }
  } else if constexpr (KIND == kDelta) {
    return delta_bucket(u, sp.x0, sp.delta, sp.rdelta, sp.m);
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
