// ms_tc.cuh -- the pre-scan and post-scan of the multisplit (Section 4.6 /
// 5.3) for up to 32 buckets, ranked with per-thread bucket counters.
//
// Localization (Section 4.4): CTA c owns a chunk of consecutive 4096-key
// tiles (first level, one column of H per chunk); a tile is solved as a whole
// (second level) by 256 threads, thread t owning the 16 consecutive keys
// [16t, 16t+16) of the tile (third level).  The direct solve of Section 4.5
// is done with a counter per (bucket, thread) in shared memory instead of the
// warp ballots of Section 5.4: a thread adds 1 to the counter of each of its
// keys' buckets with a shared-memory atomic that returns the count before
// the increment -- the key's rank among the earlier keys of its bucket in
// that thread -- and one exclusive scan over the counters in (bucket, thread)
// order then gives every (bucket, thread) its first position in the
// bucket-ordered tile (both terms of the block-level local offset of Section
// 5.5.4 at once).  Position = scan value + rank; the tile is permuted in
// place in shared memory (the block-level reordering of Section 5.6.2) and
// written out with consecutive threads on consecutive positions, so global
// writes are coalesced per bucket run.
//
// Why on GB300: an SM must move about 22 bytes of HBM traffic per cycle, so a
// 32-key window may cost only ~35 warp instructions in the post-scan.  The
// ballot ranks cost about 3 ceil(log2 m) + 10 per window before the reorder;
// the counter ranks cost two instructions per key (address, atomic) plus
// m/16 per key for the scan, independent of the key distribution.
//
// Tiles arrive in shared memory by TMA tensor copies with the 128-byte
// swizzle (the 16-byte chunk c of 128-byte row r lands at chunk c ^ (r & 7)),
// so a thread's 64 contiguous bytes are read with four conflict-free 16-byte
// loads.  The pre-scan reads the keys straight into registers with 16-byte
// loads, keeping the last part of every chunk in L2 (evict_last) for the
// post-scan, which walks its chunk last tile first.  The global scan of H
// (Section 4.3, Eq. 2) is not a separate step: every post-scan CTA reads the
// whole of H (m x G words, a few tens of KB from L2) and reduces the two terms
// its chunk needs -- the keys of all smaller buckets and the keys of its
// bucket in earlier chunks -- so no CTA scans H alone while the others wait.
// The post-scan, launched as a programmatic dependent, starts its set-up and
// first copies while the pre-scan drains.
#pragma once

#include <cuda.h>

#include "ms_bucket.cuh"
#include "ms_kernels.cuh"
#include "ms_tma.cuh"

namespace ms {

constexpr int kTcThreads = 256;
constexpr int kTcKpt = 16;                         // keys per thread
constexpr uint32_t kTcTile = kTcThreads * kTcKpt;  // 4096 keys = 128 rows of 32 words
constexpr uint32_t kTcRow = 288;                   // words per bucket row: 256 counters + 4 pad words per 32
constexpr uint32_t kTcMaxM = 32;
constexpr uint32_t kTcBulkMaxM = 8;  // post-scan write-out by one bulk copy per bucket run up to this m

// Counter rows (a power of two >= 4 and >= m): the scan covers R * 256 counters.
__host__ __device__ constexpr uint32_t tc_rows(uint32_t m) { return m <= 4 ? 4u : m <= 8 ? 8u : m <= 16 ? 16u : 32u; }

// Padded index of flattened counter i = b * 256 + t: 4 pad words after every
// 32 keep both the per-thread atomics (bank = lane) and the 16-byte raking
// loads (thread r reads R consecutive counters) free of bank conflicts.
__device__ __forceinline__ uint32_t tc_pad(uint32_t i) { return i + ((i >> 5) << 2); }

// Word position of tile element p in a slot filled by a 128-byte-swizzle tensor
// copy of 32-word rows (row p >> 5, 16-byte chunk (p >> 2) & 7 XOR row & 7).
__device__ __forceinline__ uint32_t tc_swz(uint32_t p) { return p ^ (((p >> 5) & 7u) << 2); }

// Word position of element p of the bucket-ordered tile: the low 5 bits XOR
// the 32-word row index, so the scatter of 32 keys whose positions step by a
// power of two (few buckets: a thread's keys of one bucket are spread evenly)
// and the write-out of 32 consecutive positions both hit 32 different banks.
__device__ __forceinline__ uint32_t tc_rswz(uint32_t p) { return p ^ ((p >> 5) & 31u); }


// 16-byte read-only load that does not allocate in L1, with an L2 policy.
__device__ __forceinline__ uint4 ldg_v4_policy(const uint32_t* p, uint64_t policy) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(policy));
  return v;
}

// One 2-D tensor copy (box 32 words x 128 rows) into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_tile_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// Exclusive scan over the 256 threads with one block barrier.  s_warp (8
// words) must not be rewritten before the caller's next block barrier.
__device__ __forceinline__ uint32_t tc_block_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  const uint4 a = *reinterpret_cast<const uint4*>(s_warp);
  const uint4 b = *reinterpret_cast<const uint4*>(s_warp + 4);
  const uint32_t ws[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint32_t pre = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    pre += (i < (int)w) ? ws[i] : 0u;
    tot += ws[i];
  }
  *total = tot;
  return pre + x - v;
}

// Splitter lookup table of these kernels (range buckets): the packed table of
// build_packed_lut (ms_bucket.cuh) with BB = 5 for m <= 32 and 8 for m <= 256.
constexpr uint32_t kTcLutFlag = 32u;  // the flag bit for BB = 5

__host__ __device__ constexpr uint32_t tc_lut_words(int kind, uint32_t lb, uint32_t lw) {
  return kind == kRange ? (1u << (lb + lw)) : 0u;
}

// Splitter table (2^BB - 1 entries, padded with 0xffffffff) and lookup table.
// All threads of the block call it; ends with a block barrier.
template <int KIND, int BB = 5>
__device__ __forceinline__ void tc_build_tables(const DevSpec& sp, uint32_t lb, uint32_t lw, uint32_t* tbl,
                                                uint32_t* lut) {
  if constexpr (KIND == kWide) build_wide_table<BB>(sp, tbl);
  if constexpr (KIND == kRange) {
    constexpr uint32_t P = (1u << BB) - 1u;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) tbl[i] = (i + 1 < sp.m) ? sp.splitters[i] : 0xffffffffu;
    __syncthreads();
    build_packed_lut<BB>(sp, lb, lw, tbl, lut);
  }
  __syncthreads();
}

// Bucket of u by the fast path.  For range buckets the bucket returned for a
// key of a flagged cell is wrong; callers OR the table words into `flag` and
// redo the flagged keys with tc_fixup (rare: the fast path stays lean).
struct TcLut {
  const uint32_t* lut;
  uint32_t sh;    // 32 - lb
  uint32_t lw;    // log2 of the copies
  uint32_t rep;   // this lane's copy
  uint32_t fmask; // 2^sh - 1
  const uint32_t* tbl;  // splitter table (kWide: super-bucket splitters)
  __device__ __forceinline__ uint32_t word(uint32_t u) const { return lut[((u >> sh) << lw) + rep]; }
};

template <int KIND, int BB = 5>
__device__ __forceinline__ uint32_t tc_bucket(uint32_t u, const DevSpec& sp, const TcLut& L, uint32_t& flag) {
  if constexpr (KIND == kRange) {
    const uint32_t e = L.word(u);
    flag |= e;
    return packed_fast<BB>(u, e, L.fmask);
  } else if constexpr (KIND == kWide) {
    return wide_bucket<BB>(u, sp, L.tbl);
  } else {
    return bucket_of<KIND, BB>(u, sp, nullptr, nullptr);
  }
}

template <int N, int BB = 5>
__device__ __forceinline__ void tc_fixup(const uint32_t (&key)[N], uint32_t (&bk)[N], const TcLut& L,
                                         const uint32_t* tbl, uint32_t m) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint32_t e = L.word(key[i]);
    // m <= 32: five halving steps; m <= 256: the cell's few splitters
    if constexpr (BB <= 5) {
      if (e & (1u << BB)) bk[i] = range_search<BB>(key[i], tbl, m);
    } else {
      if (e & (1u << BB)) bk[i] = range_in_cell<BB>(key[i], e, tbl, m);
    }
  }
}

// ---------------------------------------------------------------------------
// Pre-scan: per-chunk bucket histograms, H[b * hsb + c * hsc] for bucket b
// and chunk c -- bucket-major (hsb = G, hsc = 1) for the look-back scan of
// m > 32, chunk-major (hsb = 1, hsc = m) for the post-scans of m <= 32, which
// read H whole -- and, optionally, the bucket totals (the device histogram).
struct TcPreArgs {
  const uint32_t* keys;
  uint32_t n;
  uint32_t tiles_per_chunk;  // K
  uint32_t num_tiles;        // L
  uint32_t G;                // chunks
  uint32_t keep_from;        // chunk-relative tile index from which loads keep their lines in L2
                             // (the grid: any number of CTAs, each an equal run of the tiles)
  uint32_t vec;              // keys 16-byte aligned
  uint32_t* H;               // m * G words, zero before the launch (the parts of a chunk add their
                             // counts), or nullptr
  uint32_t hsb, hsc;         // strides of H: bucket, chunk
  uint32_t* tot;             // m bucket totals, zero before the launch, or nullptr
  uint32_t lb, lw;           // lookup table: 2^lb cells, 2^lw copies (range buckets)
  DevSpec sp;
};

// How the pre-scan counts: per-(bucket, thread) 32-bit counters (m <= 32),
// eight 8-bit counters in one 64-bit register per thread (m <= 8), or
// per-lane 8-bit counters per warp, four buckets to a word in the lane's own
// bank (m <= 256).
enum TcCount : int { kCountThread = 0, kCountReg = 1, kCountLaneBytes = 2 };

__host__ __device__ constexpr uint32_t tc_mpad(uint32_t m) { return m <= 32 ? 32u : ((m + 31u) & ~31u); }

template <int KIND, int MODE>
__host__ size_t tc_prescan_smem(uint32_t m, uint32_t lb, uint32_t lw) {
  const uint32_t cnt_words = MODE == kCountLaneBytes ? (kTcThreads / 32) * tc_mpad(m) * 9u : tc_rows(m) * kTcRow;
  const uint32_t tbl_words = MODE == kCountLaneBytes ? 256u : 32u;
  return 4u * (size_t)(cnt_words + tbl_words + tc_lut_words(KIND, lb, lw));
}

// Tiles of keys in flight per thread in the pre-scan's main loop.  Range
// buckets (a lookup-table probe and a splitter compare per key) gain from a
// third tile at two CTAs per SM (3-4 us of 68 at 2^26 keys on GB300); delta
// buckets lost 15 us that way and modulo buckets nothing, so they keep two
// tiles at three CTAs per SM.
template <int KIND, int MODE>
__host__ __device__ constexpr int tc_prescan_depth() {
  return (KIND == kRange && MODE != kCountLaneBytes) ? 3 : 2;
}

// CTAs per SM the pre-scan is compiled for: two where a third tile in flight
// (range buckets, up to 32 of them) or the range lookup of the byte counters
// (more than 32 buckets: it spills at 80 registers) needs the registers,
// three otherwise (measured on GB300, 2^26 keys: delta buckets, 64 of them,
// 92 -> 78 us; 256 of them, 99 -> 88 us).
template <int KIND, int MODE>
__host__ __device__ constexpr int tc_prescan_min_ctas() {
  return (tc_prescan_depth<KIND, MODE>() == 3 || (MODE == kCountLaneBytes && KIND == kRange)) ? 2 : 3;
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(kTcThreads, tc_prescan_min_ctas<KIND, MODE>()) k_prescan_tc(TcPreArgs a) {
  constexpr int BB = MODE == kCountLaneBytes ? 8 : 5;  // bits of a bucket in the lookup table
  constexpr int NW = kTcThreads / 32;
  extern __shared__ __align__(16) uint32_t smem[];
  const DevSpec& sp = a.sp;
  const uint32_t m = sp.m, R = tc_rows(m), m_pad = tc_mpad(m);
  const uint32_t cnt_words = MODE == kCountLaneBytes ? NW * m_pad * 9u : R * kTcRow;
  uint32_t* s_cnt = smem;
  uint32_t* s_tbl = smem + cnt_words;
  uint32_t* s_lut = s_tbl + (MODE == kCountLaneBytes ? 256u : 32u);
  const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5;
  const TcLut L{s_lut, 32u - a.lb, a.lw, lane & ((1u << a.lw) - 1u), (1u << (32u - a.lb)) - 1u, s_tbl};

  for (uint32_t i = t; i < cnt_words; i += kTcThreads) s_cnt[i] = 0u;
  tc_build_tables<KIND, BB>(sp, a.lb, a.lw, s_tbl, s_lut);  // ends with a barrier
  pdl_launch_dependents();

  uint32_t* my = s_cnt + t + ((t >> 5) << 2);  // kCountThread/kCountReg: counter (bucket 0, thread t)
  uint32_t* wwords = s_cnt + w * m_pad * 8u;   // kCountLaneBytes: this warp's byte counters
  uint32_t* wtot = s_cnt + NW * m_pad * 8u + w * m_pad;  // ... and its 32-bit totals
  // this CTA's share of the tiles: an equal run of them, cut at chunk
  // boundaries, each piece's counts added into its chunk's column of H (so
  // the grid is one wave whatever the number of chunks)
  const uint32_t nct = gridDim.x;
  const uint32_t K = a.tiles_per_chunk;
  uint32_t ta, tz;
  if (nct == a.G) {  // one CTA per chunk
    ta = blockIdx.x * K;
    tz = min(a.num_tiles, ta + K);
  } else {
    ta = (uint32_t)((uint64_t)a.num_tiles * blockIdx.x / nct);
    tz = (uint32_t)((uint64_t)a.num_tiles * (blockIdx.x + 1u) / nct);
  }
  const uint32_t nfull = a.n / kTcTile;  // tiles [0, nfull) are full
  const uint64_t pol_first = policy_evict_first(), pol_last = policy_evict_last();

  uint64_t creg = 0;       // kCountReg: eight 8-bit counters
  uint32_t since = 0;      // keys counted by this thread since the last flush
  auto flush = [&]() {
    if constexpr (MODE == kCountReg) {
      for (uint32_t b = 0; b < m; ++b) {
        const uint32_t v = (uint32_t)(creg >> (8u * b)) & 0xffu;
        if (v) atomicAdd(my + b * kTcRow, v);
      }
      creg = 0;
    } else if constexpr (MODE == kCountLaneBytes) {
      prescan_flush(wwords, wtot, m_pad, lane);
    }
    since = 0;
  };
  auto count1 = [&](uint32_t b) {
    if constexpr (MODE == kCountThread) {
      atomicAdd(my + b * kTcRow, 1u);
    } else if constexpr (MODE == kCountReg) {
      creg += 1ull << (8u * b);
    } else {
      atomicAdd(wwords + ((b >> 2) << 5) + lane, 1u << ((b & 3u) << 3));
    }
  };
  auto count16 = [&](uint32_t (&key)[16]) {
    uint32_t bk[16];
    uint32_t flag = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) bk[i] = tc_bucket<KIND, BB>(key[i], sp, L, flag);
    if constexpr (KIND == kRange)
      if (flag & (1u << BB)) tc_fixup<16, BB>(key, bk, L, s_tbl, m);
    if constexpr (MODE != kCountThread)
      if (since + 16u > 255u) flush();  // a byte counter must not overflow
#pragma unroll
    for (int i = 0; i < 16; ++i) count1(bk[i]);
    since += 16u;
  };
  // thread (w, lane) holds words w*512 + j*128 + 4*lane + e of the tile; the
  // last tiles of every chunk keep their lines in L2 for the post-scan
  auto load16 = [&](uint32_t (&key)[16], uint32_t tile) {
    const uint64_t pol = (tile % K >= a.keep_from) ? pol_last : pol_first;
    const uint32_t* src = a.keys + (size_t)tile * kTcTile + w * 512u + 4u * lane;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 v = ldg_v4_policy(src + 128 * j, pol);
      key[4 * j + 0] = v.x;
      key[4 * j + 1] = v.y;
      key[4 * j + 2] = v.z;
      key[4 * j + 3] = v.w;
    }
  };
  auto put = [&](uint32_t b, uint32_t c, uint32_t cnt) {
    if (cnt == 0u) return;
    if (a.H != nullptr) atomicAdd(a.H + (size_t)b * a.hsb + (size_t)c * a.hsc, cnt);
    if (a.tot != nullptr) atomicAdd(a.tot + b, cnt);
  };

  // counts tiles [t0, t1) of chunk c and adds them into its column of H
  auto piece = [&](uint32_t c, uint32_t t0, uint32_t t1) {
    const uint32_t tv1 = a.vec ? max(t0, min(t1, nfull)) : t0;
    // full, aligned tiles: 16-byte loads, the next D - 1 tiles' loads in
    // flight while this one is counted
    if (t0 < tv1) {
      constexpr int D = tc_prescan_depth<KIND, MODE>();
      uint32_t kbuf[D][16];
#pragma unroll
      for (int d = 0; d < D - 1; ++d)
        if (t0 + d < tv1) load16(kbuf[d], t0 + d);
      for (uint32_t tile = t0; tile < tv1; tile += D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          if (tile + d >= tv1) break;
          if (tile + d + D - 1 < tv1) load16(kbuf[(d + D - 1) % D], tile + d + D - 1);
          count16(kbuf[d]);
        }
      }
    }
    // the partial last tile, or every tile of an unaligned input (at most 16
    // keys per thread per tile, so the byte counters are flushed per tile)
    for (uint32_t tile = tv1; tile < t1; ++tile) {
      const size_t tb = (size_t)tile * kTcTile;
      const uint32_t rem = (uint32_t)min((size_t)kTcTile, (size_t)a.n - tb);
      if constexpr (MODE != kCountThread)
        if (since + 16u > 255u) flush();
      for (uint32_t p = t; p < rem; p += kTcThreads) {
        uint32_t flag = 0;
        const uint32_t u = a.keys[tb + p];
        uint32_t b = tc_bucket<KIND, BB>(u, sp, L, flag);
        if constexpr (KIND == kRange)
          if (flag & (1u << BB)) b = range_in_cell<BB>(u, L.word(u), s_tbl, m);
        count1(b);
      }
      since += 16u;
    }
    if constexpr (MODE != kCountThread) flush();
    __syncthreads();

    // column c of H: the counts of this piece
    if constexpr (MODE == kCountLaneBytes) {
      for (uint32_t b = t; b < m; b += kTcThreads) {
        uint32_t s2 = 0;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) s2 += s_cnt[NW * m_pad * 8u + ww * m_pad + b];
        put(b, c, s2);
      }
    } else {
      // warp w sums buckets w, w+8, w+16, w+24 over the 256 threads
      for (uint32_t b = w; b < m; b += kTcThreads / 32) {
        const uint32_t* row = s_cnt + b * kTcRow + lane;
        uint32_t s2 = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) s2 += row[36 * k];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s2 += __shfl_xor_sync(kFull, s2, d);
        if (lane == 0) put(b, c, s2);
      }
    }
  };

  if (nct == a.G) {
    piece(blockIdx.x, ta, tz);  // one chunk
  } else {
    for (uint32_t t0 = ta; t0 < tz;) {
      const uint32_t c = t0 / K;  // the chunk of this piece
      const uint32_t t1 = min(tz, (c + 1u) * K);
      piece(c, t0, t1);
      t0 = t1;
      if (t0 < tz) {  // counters cleared for the next piece
        __syncthreads();
        for (uint32_t i = t; i < cnt_words; i += kTcThreads) s_cnt[i] = 0u;
        __syncthreads();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Post-scan.
struct TcPostArgs {
  const uint32_t* keys_in;
  const uint32_t* vals_in;
  uint32_t* keys_out;
  uint32_t* vals_out;
  uint32_t n;
  uint32_t tiles_per_cta;
  uint32_t num_tiles;
  uint32_t G;
  const uint32_t* H;   // chunk histograms, chunk-major H[c * R + b] (G * R words, R = tc_rows(m))
  uint32_t* offsets;   // m + 1 bucket starts (written by CTA 0), or nullptr
  uint32_t* err;       // device status word
  uint32_t tma;        // 1: full tiles arrive by tensor copies (inputs 16-byte aligned)
  uint32_t lb, lw;     // lookup table: 2^lb cells, 2^lw copies (range buckets)
  DevSpec sp;
};

// Dynamic shared memory (words), from a 1024-byte-aligned base: a ring of
// STAGES slots, each holding a tile's keys in T + 256 words (then its values
// in as many, for pairs; 256 spare words keep every part 1024-byte aligned for
// the swizzled tensor copies and give the reordered tile room for the
// per-bucket padding below); counters R * 288; splitter table (32); lookup
// table.  1 KB of slack for the alignment.
template <int KIND, bool PAIRS, int STAGES, int KPT, bool BULK>
struct TcPostLayout {
  static constexpr uint32_t T = kTcThreads * KPT;
  // words of one array (keys or values) in a slot: 256 spare words for the
  // padded runs of the bulk write-out, none otherwise
  static constexpr uint32_t kPart = T + (BULK ? 256u : 0u);
  static constexpr uint32_t kSlotWords = kPart * (PAIRS ? 2u : 1u);
  // a bucket byte per reordered position for the write-out without bulk
  // copies, unless the identifier is cheap to evaluate again
  static constexpr bool kBytes = !BULK && !cheap_bucket<KIND, PAIRS>();
  static __host__ __device__ uint32_t cnt(uint32_t) { return STAGES * kSlotWords; }
  static __host__ __device__ uint32_t bkt(uint32_t m) { return cnt(m) + tc_rows(m) * kTcRow; }
  static __host__ __device__ uint32_t tbl(uint32_t m) { return bkt(m) + (kBytes ? T / 4 : 0u); }
  static __host__ __device__ uint32_t lut(uint32_t m) { return tbl(m) + 32; }
  static __host__ size_t bytes(uint32_t m, uint32_t lb, uint32_t lw) {
    return 1024u + 4u * (size_t)(lut(m) + tc_lut_words(KIND, lb, lw));
  }
};

// Bucket of u for the post-scan.  Range buckets: a key of a flagged cell gets
// a value >= 32 (the flag bit stays in the sum) that tc_fix_marked replaces
// by the search; every other key gets its bucket (< 32), so the flagged keys
// are found without reading the table again.
template <int KIND>
__device__ __forceinline__ uint32_t tc_bucket_marked(uint32_t u, const DevSpec& sp, const TcLut& L) {
  if constexpr (KIND == kRange) {
    const uint32_t e = L.word(u);
    return (e & 63u) + ((u & L.fmask) >= (e >> 6) ? 1u : 0u);
  } else {
    return bucket_of<KIND, 5>(u, sp, nullptr, nullptr);
  }
}

template <int N>
__device__ __forceinline__ void tc_fix_marked(const uint32_t (&key)[N], uint32_t (&bk)[N], const uint32_t* tbl,
                                              uint32_t m) {
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (bk[i] >= 32u) bk[i] = range_search<5>(key[i], tbl, m);
}

// KPT keys per thread (16, or 8: a 2048-key tile, half the registers per
// thread, more CTAs per SM).
//
// Write-out.  BULK (up to kTcBulkMaxM buckets: runs of T/m keys or more) by
// bulk copies: the tile is reordered in place in its slot with bucket b's run
// placed at tile position + 4b + (delta_b mod 4), where delta_b = (the run's
// first global position) - (its first tile position), so that every run sits
// at the same address modulo 16 bytes in shared memory as in the output;
// thread b then writes run b with one bulk copy (TMA) of its 16-byte-aligned
// interior and at most three plain stores at each end -- the copy engine
// reads shared memory and writes HBM without the load/store units.  A slot is
// refilled only after its bulk copies have read it.  More buckets (short runs,
// where a copy per run costs more than it saves): the tile is reordered in
// place with the XOR swizzle of tc_rswz and written by consecutive threads on
// consecutive positions, each position's bucket from a stored byte (or from
// the key again, for radix digits).
template <int KIND, bool PAIRS, int STAGES, int KPT, bool BULK>
__global__ void __launch_bounds__(kTcThreads, KPT == 8 ? 3 : 2)
    k_postscan_tc(const __grid_constant__ CUtensorMap tmk, const __grid_constant__ CUtensorMap tmv, TcPostArgs a) {
  static_assert(KPT == 8 || KPT == 16, "8 or 16 keys per thread");
  using Lay = TcPostLayout<KIND, PAIRS, STAGES, KPT, BULK>;
  constexpr uint32_t T = Lay::T;
  extern __shared__ __align__(16) uint32_t smem_raw[];
  __shared__ __align__(8) uint64_t s_bar[STAGES];
  __shared__ uint32_t s_pend[STAGES];  // 1 + index of the tile whose copy is in flight in the slot, 0 if none
  __shared__ uint32_t s_run[kTcMaxM], s_off[kTcMaxM], s_start[kTcMaxM], s_delta[kTcMaxM];
  __shared__ __align__(16) uint32_t s_scr[2 * 8 * 32];  // scratch of chunk_offsets
  __shared__ __align__(16) uint32_t s_warp[8];
  const DevSpec& sp = a.sp;
  const uint32_t m = sp.m, R = tc_rows(m);
  const uint32_t sa = smem_addr(smem_raw);
  uint32_t* base = smem_raw + (((1024u - (sa & 1023u)) & 1023u) >> 2);
  uint32_t* ring = base;
  constexpr uint32_t PART = Lay::kPart, SLOT = Lay::kSlotWords;
  uint32_t* s_cnt = base + Lay::cnt(m);
  uint8_t* s_bkt = reinterpret_cast<uint8_t*>(base + Lay::bkt(m));
  uint32_t* s_tbl = base + Lay::tbl(m);
  uint32_t* s_lut = base + Lay::lut(m);

  const uint32_t t = threadIdx.x;
  const TcLut L{s_lut, 32u - a.lb, a.lw, t & ((1u << a.lw) - 1u), (1u << (32u - a.lb)) - 1u, s_tbl};
  const uint32_t c = blockIdx.x;
  const uint32_t t0 = c * a.tiles_per_cta;
  const uint32_t t1 = min(t0 + a.tiles_per_cta, a.num_tiles);
  const uint32_t ntiles = t1 > t0 ? t1 - t0 : 0u;
  // the chunk is walked last tile first: the pre-scan read those last, so
  // they are the ones still in L2
  auto tile_of = [&](uint32_t j) { return t1 - 1u - j; };
  auto is_full = [&](uint32_t j) { return (size_t)(tile_of(j) + 1u) * T <= a.n; };

  auto issue = [&](uint32_t j) {  // thread 0: start the copies of tile j into its slot
    if (!a.tma || j >= ntiles || !is_full(j)) return;
    const uint32_t slot = j % STAGES;
    const int y = (int)(tile_of(j) * (T / 32u));
    const uint64_t pol = policy_evict_first();
    mbar_arrive_expect_tx(s_bar + slot, T * 4u * (PAIRS ? 2u : 1u));
    tma_tile_2d(ring + slot * SLOT, &tmk, 0, y, s_bar + slot, pol);
    if constexpr (PAIRS) tma_tile_2d(ring + slot * SLOT + PART, &tmv, 0, y, s_bar + slot, pol);
    s_pend[slot] = j + 1u;
  };

  if (t == 0) {
    for (int k = 0; k < STAGES; ++k) {
      mbar_init(s_bar + k, 1);
      s_pend[k] = 0u;
    }
    fence_mbar_init();
  }
  for (uint32_t i = t; i < R * kTcRow; i += kTcThreads) s_cnt[i] = 0u;
  __syncthreads();
  if (t == 0)
    for (uint32_t j = 0; j < (uint32_t)STAGES; ++j) issue(j);  // inputs are not written by the pre-scan
  tc_build_tables<KIND>(sp, a.lb, a.lw, s_tbl, s_lut);  // ends with a barrier
  pdl_wait();  // H complete (the pre-scan grid has finished)
  chunk_offsets(a.H, a.G, m, R, c, s_run, s_scr, a.offsets);

  uint32_t* my = s_cnt + t + ((t >> 5) << 2);  // counter (bucket 0, thread t)
  uint32_t phase = 0;                          // bit k: parity of slot k's next completion
  // output addresses in words modulo 4: the runs are placed to match the keys'
  // (the values take the bulk copies too when theirs is the same)
  const uint32_t rk = (uint32_t)(reinterpret_cast<uintptr_t>(a.keys_out) >> 2) & 3u;
  const bool vbulk = !PAIRS || (((uint32_t)(reinterpret_cast<uintptr_t>(a.vals_out) >> 2) & 3u) == rk);

  auto tile_body = [&](auto full_tag, uint32_t j) -> bool {
    constexpr bool FULL = decltype(full_tag)::value;
    const uint32_t tile = tile_of(j), slot = j % STAGES;
    const size_t tb = (size_t)tile * T;
    const uint32_t tile_n = FULL ? T : (uint32_t)((size_t)a.n - tb);
    uint32_t* sk = ring + slot * SLOT;
    uint32_t* sv = sk + PART;
    (void)sv;
    bool ok = true;
    if (FULL && a.tma) {
      ok = mbar_wait(s_bar + slot, (phase >> slot) & 1u, a.err);
      if (ok) phase ^= 1u << slot;
    } else {
      for (uint32_t p = t; p < tile_n; p += kTcThreads) {
        sk[tc_swz(p)] = __ldcs(a.keys_in + tb + p);
        if constexpr (PAIRS) sv[tc_swz(p)] = __ldcs(a.vals_in + tb + p);
      }
      __syncthreads();
    }

    // (A) this thread's KPT keys (and values), tile elements [KPT t, KPT t + KPT)
    uint32_t key[KPT], bk[KPT], pos[KPT];
    uint32_t val[PAIRS ? KPT : 1];
#pragma unroll
    for (int j4 = 0; j4 < KPT / 4; ++j4) {
      const uint4 v = *reinterpret_cast<const uint4*>(sk + tc_swz(KPT * t + 4u * j4));
      key[4 * j4 + 0] = v.x;
      key[4 * j4 + 1] = v.y;
      key[4 * j4 + 2] = v.z;
      key[4 * j4 + 3] = v.w;
      if constexpr (PAIRS) {
        const uint4 x = *reinterpret_cast<const uint4*>(sv + tc_swz(KPT * t + 4u * j4));
        val[4 * j4 + 0] = x.x;
        val[4 * j4 + 1] = x.y;
        val[4 * j4 + 2] = x.z;
        val[4 * j4 + 3] = x.w;
      }
    }
    // (B) buckets
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      bk[i] = tc_bucket_marked<KIND>(key[i], sp, L);
      any |= bk[i];
    }
    if constexpr (KIND == kRange)
      if (any >= 32u) tc_fix_marked<KPT>(key, bk, s_tbl, m);
    // (C) rank of each key among the earlier keys of its bucket in this thread
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if (FULL || KPT * t + i < tile_n) pos[i] = atomicAdd(my + bk[i] * kTcRow, 1u);
    }
    // the previous tile's bulk copies out of the other slot have read it
    if constexpr (BULK)
      if (t < m) bulk_wait_read_all();
    if (__syncthreads_or(!ok)) return false;  // (1) counts complete; the previous tile is written out
    if (t == 0 && j > 0) {
      // the previous tile's slot is free again: refill it
      s_pend[(j - 1u) % STAGES] = 0u;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(j - 1u + STAGES);
    }
    if (t == 0) s_pend[slot] = 0u;

    // (D) one exclusive scan over the counters in (bucket, thread) order:
    // thread r rakes counters [r*R, r*R + R)
    {
      uint4* seg = reinterpret_cast<uint4*>(s_cnt + tc_pad(t * R));
      uint32_t sum = 0;
      for (uint32_t g = 0; g < R / 4u; ++g) {
        const uint4 v = seg[g];
        sum += v.x + v.y + v.z + v.w;
      }
      uint32_t total;
      uint32_t run = tc_block_scan(sum, s_warp, &total);  // contains barrier (2)
      if (((t * R) & 255u) == 0u) {
        const uint32_t b = (t * R) >> 8;
        if (b < m) s_start[b] = run;  // counter (b, 0): where bucket b starts in the tile
      }
      // rows b >= m (R > m) stay zero: no key counts there, and nothing reads them
      for (uint32_t g = 0; t * R < m * 256u && g < R / 4u; ++g) {
        const uint4 v = seg[g];
        uint4 o;
        o.x = run;
        run += v.x;
        o.y = run;
        run += v.y;
        o.z = run;
        run += v.z;
        o.w = run;
        run += v.w;
        seg[g] = o;
      }
    }
    __syncthreads();  // (3) scanned counters and bucket starts visible

    // (E) per bucket: the run's global start, its offset in the reordered slot
    uint32_t gs = 0, cnt = 0;
    if (t < m) {
      const uint32_t start = s_start[t];
      const uint32_t end = (t + 1u < m) ? s_start[t + 1u] : tile_n;
      cnt = end - start;
      gs = s_run[t] - cnt;
      s_run[t] = gs;
      s_delta[t] = gs - start;
      if constexpr (BULK) s_off[t] = 4u * t + ((gs - start + rk) & 3u);
    }
    // positions, then clear this thread's counters (rows < m; the scan wrote
    // every one of them) for the next tile
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if (FULL || KPT * t + i < tile_n) pos[i] += my[bk[i] * kTcRow];
    }
    for (uint32_t b = 0; b < m; ++b) my[b * kTcRow] = 0u;
    if constexpr (BULK) __syncthreads();  // (3b) s_off visible
    // (F) permute the tile in place (every thread read its keys before (1))
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if (FULL || KPT * t + i < tile_n) {
        const uint32_t p = pos[i];
        if (p < T) {
          if constexpr (BULK) {
            const uint32_t q = p + s_off[bk[i]];
            sk[q] = key[i];
            if constexpr (PAIRS) sv[q] = val[i];
          } else {
            const uint32_t q = tc_rswz(p);
            sk[q] = key[i];
            if constexpr (PAIRS) sv[q] = val[i];
            if constexpr (Lay::kBytes) s_bkt[q] = (uint8_t)bk[i];
          }
        } else {
          atomicOr(a.err, kDevErrBounds);
        }
      }
    }
    if constexpr (BULK) fence_proxy_async_smem();  // the permuted tile, for the bulk copies
    __syncthreads();                               // (4)

    if constexpr (BULK) {
      // (G) thread b writes bucket b's run: the 16-byte-aligned interior by
      // one bulk copy, the ends by plain stores
      if (t < m && cnt > 0u) {
        if ((size_t)gs + cnt <= a.n) {
          const uint32_t q0 = s_start[t] + s_off[t];  // the run in the slot
          const uint32_t ge = gs + cnt;
          // [a0, a1): the positions whose output addresses are 16-byte aligned
          const uint32_t a0 = min(ge, gs + ((4u - ((gs + rk) & 3u)) & 3u));
          const uint32_t a1 = max(a0, ge - ((ge + rk) & 3u));
          if (a1 > a0) {
            const uint64_t pol = policy_evict_first();
            bulk_s2g(a.keys_out + a0, sk + q0 + (a0 - gs), (a1 - a0) * 4u, pol);
            if (PAIRS && vbulk) bulk_s2g(a.vals_out + a0, sv + q0 + (a0 - gs), (a1 - a0) * 4u, pol);
          }
          bulk_commit();
          auto put = [&](uint32_t g) {
            __stcs(a.keys_out + g, sk[q0 + (g - gs)]);
            if constexpr (PAIRS) __stcs(a.vals_out + g, sv[q0 + (g - gs)]);
          };
          for (uint32_t g = gs; g < a0; ++g) put(g);
          for (uint32_t g = a1; g < ge; ++g) put(g);
          if constexpr (PAIRS)  // values aligned unlike the keys: plain stores for the interior too
            if (!vbulk)
              for (uint32_t g = a0; g < a1; ++g) __stcs(a.vals_out + g, sv[q0 + (g - gs)]);
        } else {
          atomicOr(a.err, kDevErrBounds);
        }
      }
    } else {
      // (G) consecutive threads write consecutive positions of each bucket run
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        const uint32_t p = t + k * kTcThreads;
        if (FULL || p < tile_n) {
          const uint32_t q = tc_rswz(p);
          const uint32_t kq = sk[q];
          uint32_t b;
          if constexpr (Lay::kBytes) {
            b = s_bkt[q];
          } else {
            b = tc_bucket_marked<KIND>(kq, sp, L);
          }
          const uint32_t g = s_delta[b] + p;
          if (g < a.n) {
            __stcs(a.keys_out + g, kq);
            if constexpr (PAIRS) __stcs(a.vals_out + g, sv[q]);
          } else {
            atomicOr(a.err, kDevErrBounds);
          }
        }
      }
    }
    return true;
  };

  for (uint32_t j = 0; j < ntiles; ++j) {
    const bool ok = is_full(j) ? tile_body(std::true_type{}, j) : tile_body(std::false_type{}, j);
    if (!ok) {
      // a copy never completed: drain the copies still in flight (bounded), then stop
      if (t == 0)
        for (int k = 0; k < STAGES; ++k)
          if (s_pend[k] != 0u) mbar_drain(s_bar + k, (phase >> k) & 1u);
      if constexpr (BULK)
        if (t < m) bulk_wait_all();
      __syncthreads();
      return;
    }
  }
  if constexpr (BULK)
    if (t < m) bulk_wait_all();  // shared memory must outlive the bulk copies reading it
}

}  // namespace ms
