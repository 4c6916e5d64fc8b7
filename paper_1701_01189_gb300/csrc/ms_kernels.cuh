// ms_kernels.cuh -- the post-scan of the multisplit with warp-level ranks
// (Section 4.6 / 5.3: stable local offsets, block-level reordering in shared
// memory, coalesced scatter), used for m > 32 and as a tuning variant, and the
// per-lane byte-counter flush of the pre-scan.  The pre-scan is ms_tc.cuh.
//
// Localization (Section 4.4; the "Block-level Multisplit" of Section 5.3):
// each CTA owns a chunk of consecutive tiles (first level, one column of H per
// chunk); a tile of T = NW*32*ITEMS keys is reordered as a whole (second
// level); warp w owns ITEMS consecutive 32-key windows of the tile (third
// level); each window is solved directly by the warp (fourth level).  Key
// (w, i, lane) sits at tile offset w*32*ITEMS + i*32 + lane, so that order is
// the input order and the ranks below are stable.
//
// H is bucket-major, H[b * G + c], so one exclusive scan over the
// row-vectorised H yields both global terms of Eq. 2.
//
// GB300 budget: with ~22 bytes of HBM traffic per SM cycle to sustain, a
// window of 32 keys may cost only ~37 warp instructions in the post-scan.
// Hence:
//  * the pre-scan's per-lane 8-bit counters (ms_tc.cuh, m > 32): a
//    fire-and-forget shared atomic per key in the lane's own bank, flushed by
//    prescan_flush into 32-bit warp totals before any byte can overflow;
//  * post-scan ranks: for m <= 32 the ballot voting of Section 5.4 (Alg. 2 and
//    the corrected Alg. 3: one ballot per bucket bit); for larger m a per-warp
//    "peer table" in shared memory: each lane ORs its lane bit into the entry
//    of its bucket, reads back the mask of its peers, and the lowest peer
//    advances the warp's counter of that bucket (the same information the
//    ballots give, at a cost that does not grow with log m).
#pragma once

#include <type_traits>

#include "ms_bucket.cuh"
#include "ms_tma.cuh"

namespace ms {

struct PostscanArgs {
  const uint32_t* keys_in;
  const uint32_t* vals_in;
  uint32_t* keys_out;
  uint32_t* vals_out;
  uint32_t n;
  DevSpec sp;
  uint32_t tiles_per_cta;
  uint32_t num_tiles;
  uint32_t G;
  const uint32_t* Gx;  // m <= 32: chunk-major histograms H[c * mp + b] (mp: 4, 8, 16 or 32 >= m); m > 32:
                       // the exclusive scan of
                       // the row-vectorised, bucket-major H (m*G entries)
  uint32_t* offsets;   // m <= 32: the m + 1 bucket starts, written by CTA 0 (or nullptr)
  uint32_t* err;       // device status word
  uint32_t prefetch;   // 1: bulk-prefetch the next tiles into L2
  uint32_t reverse;    // 1: walk the chunk's tiles last to first
};

// L2 prefetch of a contiguous block (16-byte aligned address and size).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int KIND>
__host__ __device__ constexpr uint32_t lut_words(uint32_t lut_bits) {
  return KIND == kRange ? (2u << lut_bits) : 0u;
}

// Per-lane 8-bit counters, four buckets per 32-bit word, laid out so that
// lane l only ever touches bank l: word (q, l) = q*32 + l holds the counts of
// buckets 4q..4q+3 seen by lane l.  A count is bumped with a shared-memory
// atomic add of 1 << 8*(b & 3) that nothing waits for.
//
// Flush (before any byte can overflow): lane l sums the columns of its word
// groups q = l, l+32, ... over the 32 lanes, reading them in a rotated order
// so no two lanes hit one bank, and adds the four per-bucket sums into the
// warp's 32-bit totals; then every lane zeroes its own words.
__device__ __forceinline__ void prescan_flush(uint32_t* wwords, uint32_t* wtot, uint32_t m_pad, uint32_t lane) {
  __syncwarp();
  const uint32_t groups = m_pad >> 2;
  for (uint32_t q = lane; q < groups; q += 32) {
    uint32_t lo = 0, hi = 0;  // 16-bit lanes: buckets (4q, 4q+2) and (4q+1, 4q+3)
#pragma unroll 8
    for (uint32_t s = 0; s < 32; ++s) {
      const uint32_t v = wwords[q * 32 + ((lane + s) & 31u)];
      lo += v & 0x00ff00ffu;
      hi += (v >> 8) & 0x00ff00ffu;
    }
    wtot[4 * q + 0] += lo & 0xffffu;
    wtot[4 * q + 1] += hi & 0xffffu;
    wtot[4 * q + 2] += lo >> 16;
    wtot[4 * q + 3] += hi >> 16;
  }
  __syncwarp();
  for (uint32_t q = 0; q < groups; ++q) wwords[q * 32 + lane] = 0u;
  __syncwarp();
}

// Ranks the ITEMS windows of one warp (Section 5.5: a direct solve per
// 32-key window).  wk points at this lane's first key (the warp's keys are
// wk[i*32] for window i); `avail` is the number of keys of the warp's share
// counted from its first key (only read when !FULL).  On return rb[i] holds
// the key's rank among the earlier keys of its bucket in this warp (low 16
// bits) and the bucket (bits 16..23), and wc[b] (table mode) or wc[lane]
// (ballot mode) the warp's count of bucket b.
template <int KIND, int NB, int ITEMS, int RANK, bool FULL>
__device__ __forceinline__ void rank_windows(const uint32_t* wk, uint32_t avail, const DevSpec& sp,
                                             const uint32_t* s_tbl, const uint32_t* s_lut, uint32_t* wc,
                                             uint32_t* wpeer, uint32_t m_pad, uint32_t m, const uint32_t* lane_x,
                                             uint32_t lt_mask, uint32_t lane, uint32_t (&rb)[ITEMS]) {
  if constexpr (RANK == kRankTable || RANK == kRankVote) {
    for (uint32_t b = lane; b < m_pad; b += 32) wc[b] = 0u;
    __syncwarp();
  }
  uint32_t run = 0;  // ballot mode: keys of bucket `lane` in earlier windows of this warp
  (void)run;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const bool valid = FULL || (uint32_t)(i * 32) + lane < avail;
    const uint32_t b = valid ? bucket_of<KIND, NB>(wk[i * 32], sp, s_tbl, s_lut) : 0u;
    if constexpr (RANK == kRankBallot) {
      // Section 5.4 / Alg. 2 / Alg. 3: NB ballots give every lane the bucket
      // of every lane of the window.
      const uint32_t vb = FULL ? kFull : __ballot_sync(kFull, valid);
      uint32_t own = vb, lane_bm = vb;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const uint32_t bal = __ballot_sync(kFull, (b >> k) & 1u);
        own &= ((b >> k) & 1u) ? bal : ~bal;
        lane_bm &= bal ^ lane_x[k];
      }
      const uint32_t before = __shfl_sync(kFull, run, b & 31u);
      rb[i] = (before + __popc(own & lt_mask)) | (b << 16);
      run += __popc(lane_bm);
    } else if constexpr (RANK == kRankVote) {
      // Section 5.4's voting for any m: NB ballots give every lane the mask
      // of the lanes whose bucket equals its own (no shared memory, so no
      // conflicts however skewed the buckets); the lowest of them advances
      // the warp's counter of the bucket by the group's size.
      const uint32_t vb = FULL ? kFull : __ballot_sync(kFull, valid);
      uint32_t own = vb;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if ((uint32_t)k < sp.nbits) {  // uniform: only the bits a bucket can have
          const uint32_t bal = __ballot_sync(kFull, (b >> k) & 1u);
          own &= ((b >> k) & 1u) ? bal : ~bal;
        }
      }
      const uint32_t lt = own & lt_mask;
      uint32_t before = 0;
      if (valid && lt == 0u) before = atomicAdd(wc + b, (uint32_t)__popc(own));
      before = __shfl_sync(kFull, before, (__ffs(own) - 1) & 31);
      rb[i] = (before + __popc(lt)) | (b << 16);
    } else {
      // peer table (two, alternating by window): OR the lane bit into the
      // bucket's entry, read the peers back; the lowest peer advances the
      // warp's counter of the bucket and clears the entry.
      uint32_t* tb = wpeer + (i & 1) * m_pad;
      if (valid) atomicOr(tb + b, 1u << lane);
      __syncwarp();
      const uint32_t own = valid ? tb[b] : 0u;
      __syncwarp();
      const uint32_t lt = own & lt_mask;
      uint32_t before = 0;
      if (valid && lt == 0u) {
        before = atomicAdd(wc + b, (uint32_t)__popc(own));
        tb[b] = 0u;
      }
      before = __shfl_sync(kFull, before, (__ffs(own) - 1) & 31);
      rb[i] = (before + __popc(lt)) | (b << 16);
    }
  }
  if constexpr (RANK == kRankBallot) wc[lane] = (lane < m) ? run : 0u;
}

// One exclusive scan over the per-warp bucket counters s_cnt[w*S + b] in
// bucket-major order, in place: afterwards s_cnt[w*S + b] is where warp w's
// keys of bucket b start in the reordered tile -- earlier buckets of the tile
// (Section 5.6.2, item 2) plus earlier warps of the same bucket (Section
// 5.5.4, third term).  Returns the tile's key count.  All threads call it;
// it contains block barriers and ends with one.
template <int NW>
__device__ __forceinline__ uint32_t scan_tile_counters(uint32_t* s_cnt, uint32_t S, uint32_t m_pad, uint32_t* s_warp) {
  constexpr int LOGNW = NW == 8 ? 3 : NW == 16 ? 4 : 5;
  const uint32_t ept = m_pad >> 5;  // entries per thread (1..8)
  uint32_t pre[8];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if ((uint32_t)k < ept) {
      const uint32_t e = threadIdx.x * ept + k;
      const uint32_t v = s_cnt[(e & (NW - 1)) * S + (e >> LOGNW)];
      pre[k] = sum;
      sum += v;
    }
  }
  uint32_t total;
  const uint32_t excl = block_exclusive_scan<NW>(sum, s_warp, &total);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if ((uint32_t)k < ept) {
      const uint32_t e = threadIdx.x * ept + k;
      s_cnt[(e & (NW - 1)) * S + (e >> LOGNW)] = excl + pre[k];
    }
  }
  __syncthreads();
  return total;
}

// ---------------------------------------------------------------------------
// Post-scan.
//
// Each CTA walks the tiles of its chunk.  Full tiles arrive by bulk
// asynchronous copies (TMA) into a ring of STAGES shared-memory slots, issued
// by one thread STAGES tiles ahead and completed on one mbarrier per slot, so
// HBM latency overlaps the work on earlier tiles; the partial last tile (and
// every tile when the inputs are not 16-byte aligned) is copied in by the
// threads themselves.  Keys are read from the slot twice (ranking, then the
// scatter), so they do not occupy registers in between.
//
// REORDER = 1: the block-level reordering of Section 5.6.2 (writes coalesced
// per bucket run).  REORDER = 0: each key goes from its slot straight to its
// final position (the no-reorder design of Section 5.3's DMS), which for a
// few buckets already gives runs of consecutive addresses per warp store.
//
// Dynamic shared memory, in order: STAGES mbarriers (64 bytes), the ring
// (STAGES*T keys, STAGES*T values), splitter table (256 words), LUT, s_run,
// s_delta (256 words each), s_warp (32), counters NW*(m_pad+1), two peer
// tables per warp (table mode), and with REORDER the reorder buffers (T keys,
// T values, T bucket bytes).
template <int KIND, int NW, int ITEMS, bool PAIRS, int RANK, int REORDER, int STAGES>
struct PostLayout {
  static constexpr uint32_t T = NW * 32 * ITEMS;
  static constexpr uint32_t kRing = 16;  // words: after the mbarriers
  static constexpr uint32_t kRingWords = STAGES * T * (PAIRS ? 2 : 1);
  static __host__ __device__ uint32_t tbl() { return kRing + kRingWords; }
  static __host__ __device__ uint32_t lut() { return tbl() + 256; }
  static __host__ __device__ uint32_t run(uint32_t lb) { return lut() + lut_words<KIND>(lb); }
  static __host__ __device__ uint32_t cnt(uint32_t lb) { return run(lb) + 256 + 256 + 32; }
  static __host__ __device__ uint32_t peer(uint32_t lb, uint32_t m_pad) { return cnt(lb) + NW * (m_pad + 1); }
  static __host__ __device__ uint32_t reorder(uint32_t lb, uint32_t m_pad) {
    return (peer(lb, m_pad) + (RANK == kRankTable ? 2 * NW * m_pad : 0u) + 3u) & ~3u;
  }
  static __host__ size_t bytes(uint32_t m_pad, uint32_t lb) {
    return 4u * (size_t)(reorder(lb, m_pad) + (REORDER ? T * (PAIRS ? 2u : 1u) : 0u)) + (REORDER ? T : 0u);
  }
};

template <int KIND, int NB, int NW, int ITEMS, bool PAIRS, int RANK, int REORDER, int MINB, int STAGES>
__global__ void __launch_bounds__(NW * 32, MINB) k_postscan(PostscanArgs a) {
  using Lay = PostLayout<KIND, NW, ITEMS, PAIRS, RANK, REORDER, STAGES>;
  constexpr int THREADS = NW * 32;
  constexpr uint32_t T = Lay::T;
  static_assert(NW >= 8, "the per-bucket phase needs >= 256 threads");
  static_assert(NW == 8 || NW == 16 || NW == 32, "NW must be 8, 16 or 32");
  static_assert(RANK != kRankBallot || NB <= 5, "lane-histogram ballot ranks need m <= 32");
  static_assert(STAGES >= 1 && STAGES <= 4, "1..4 ring slots");
  extern __shared__ __align__(16) uint32_t smem[];
  const DevSpec& sp = a.sp;
  const uint32_t m = sp.m, m_pad = sp.m_pad, S = m_pad + 1, lb = sp.lut_bits;
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* ring_k = smem + Lay::kRing;
  uint32_t* ring_v = ring_k + STAGES * T;  // pairs
  uint32_t* s_tbl = smem + Lay::tbl();
  uint32_t* s_lut = smem + Lay::lut();
  uint32_t* s_run = smem + Lay::run(lb);
  uint32_t* s_delta = s_run + 256;
  uint32_t* s_warp = s_delta + 256;
  uint32_t* s_cnt = smem + Lay::cnt(lb);           // [w * S + b]
  uint32_t* s_peer = smem + Lay::peer(lb, m_pad);  // [w][2][m_pad]
  uint32_t* s_keys = smem + Lay::reorder(lb, m_pad);
  uint32_t* s_vals = s_keys + T;
  uint8_t* s_bkt = reinterpret_cast<uint8_t*>(s_keys + T * (PAIRS ? 2 : 1));
  __shared__ uint32_t s_pend[STAGES];  // 1 + index of the tile whose copy is in flight in the slot, 0 if none

  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t c = blockIdx.x;
  const uint32_t t0 = c * a.tiles_per_cta;
  const uint32_t t1 = min(t0 + a.tiles_per_cta, a.num_tiles);
  const uint32_t ntiles = t1 > t0 ? t1 - t0 : 0u;
  auto tile_of = [&](uint32_t j) { return a.reverse ? t1 - 1 - j : t0 + j; };
  auto is_full = [&](uint32_t j) { return (size_t)(tile_of(j) + 1) * T <= a.n; };
  const bool use_tma = a.prefetch != 0u;  // inputs 16-byte aligned

  // thread 0: start the copy of this CTA's tile j into its ring slot
  auto issue = [&](uint32_t j) {
    if (!use_tma || j >= ntiles || !is_full(j)) return;
    const uint32_t slot = j % STAGES;
    const size_t base = (size_t)tile_of(j) * T;
    mbar_arrive_expect_tx(s_bar + slot, T * 4u * (PAIRS ? 2u : 1u));
    bulk_g2s(ring_k + slot * T, a.keys_in + base, T * 4u, s_bar + slot);
    if constexpr (PAIRS) bulk_g2s(ring_v + slot * T, a.vals_in + base, T * 4u, s_bar + slot);
    s_pend[slot] = j + 1;
  };

  if (threadIdx.x == 0) {
    for (int k = 0; k < STAGES; ++k) {
      mbar_init(s_bar + k, 1);
      s_pend[k] = 0;
    }
    fence_mbar_init();
  }
  if (RANK == kRankTable)
    for (uint32_t i = threadIdx.x; i < 2 * NW * m_pad; i += THREADS) s_peer[i] = 0u;
  __syncthreads();  // mbarriers initialised
  if (threadIdx.x == 0)
    for (uint32_t j = 0; j < (uint32_t)STAGES; ++j) issue(j);  // inputs are not written by the pre-scan
  build_bucket_tables<KIND, NB>(sp, s_tbl, s_lut);  // ends with a barrier
  pdl_wait();  // H complete (scanned, for m > 32)
  // next global position of each bucket: chunk start (forward) or chunk end (reverse)
  if (m <= 32u) {
    // Eq. 2 from the chunk histograms (rows of 4, 8, 16 or 32 words; the 512
    // words from s_delta on -- s_delta, s_warp, the start of s_cnt -- as
    // scratch: each is written before it is read again)
    const uint32_t mp = m <= 4u ? 4u : m <= 8u ? 8u : m <= 16u ? 16u : 32u;
    chunk_offsets(a.Gx, a.G, m, mp, c, s_run, s_delta, a.offsets);
    if (!a.reverse) {
      for (uint32_t b = threadIdx.x; b < m; b += THREADS) s_run[b] -= __ldcg(a.Gx + (size_t)c * mp + b);
      __syncthreads();
    }
  } else {
    const uint32_t len = m * a.G;
    for (uint32_t b = threadIdx.x; b < m; b += THREADS) {
      const uint32_t e = b * a.G + c;
      s_run[b] = a.reverse ? ((e + 1 < len) ? a.Gx[e + 1] : a.n) : a.Gx[e];
    }
    __syncthreads();
  }

  uint32_t* wc = s_cnt + w * S;
  uint32_t* wpeer = s_peer + w * 2 * m_pad;
  const uint32_t lt_mask = lanemask_lt();
  // Alg. 2: per ballot, the mask that keeps the lanes whose bucket bit equals
  // the same bit of this lane's id
  uint32_t lane_x[NB > 0 ? NB : 1];
#pragma unroll
  for (int k = 0; k < NB; ++k) lane_x[k] = ((lane >> k) & 1u) ? 0u : 0xffffffffu;
  const uint32_t off0 = w * (32 * ITEMS) + lane;
  // bit k: parity of the next completion of slot k's mbarrier (a slot filled
  // by plain loads for a partial tile does not advance its barrier)
  uint32_t phase = 0;

  // One tile.  FULL: all T keys present (no per-key bounds tests).
  auto tile_body = [&](auto full_tag, uint32_t j) -> bool {
    constexpr bool FULL = decltype(full_tag)::value;
    const uint32_t tile = tile_of(j);
    const size_t tbase = (size_t)tile * T;
    const uint32_t tile_n = FULL ? T : (uint32_t)((size_t)a.n - tbase);
    const uint32_t slot = j % STAGES;
    const uint32_t* rk = ring_k + slot * T;
    const uint32_t* rv = ring_v + slot * T;
    (void)rv;
    bool ok = true;
    if (FULL && use_tma) {
      ok = mbar_wait(s_bar + slot, (phase >> slot) & 1u, a.err);
      phase ^= 1u << slot;
    } else {
      // copy the tile into the slot with plain loads (no copy is in flight there)
      for (uint32_t p = threadIdx.x; p < tile_n; p += THREADS) {
        ring_k[slot * T + p] = __ldcs(a.keys_in + tbase + p);
        if constexpr (PAIRS) ring_v[slot * T + p] = __ldcs(a.vals_in + tbase + p);
      }
      __syncthreads();
    }
    uint32_t rb[ITEMS];  // rank in warp (low 16 bits) | bucket << 16
    rank_windows<KIND, NB, ITEMS, RANK, FULL>(rk + off0, tile_n - min(tile_n, off0 - lane), sp, s_tbl, s_lut, wc,
                                              wpeer, m_pad, m, lane_x, lt_mask, lane, rb);
    if (__syncthreads_or(!ok)) return false;

    // where each (bucket, warp) starts in the reordered tile
    const uint32_t total = scan_tile_counters<NW>(s_cnt, S, m_pad, s_warp);

    // Per bucket: global position minus tile position.
    if (threadIdx.x < m) {
      const uint32_t b = threadIdx.x;
      const uint32_t tstart = s_cnt[b];
      const uint32_t tend = (b + 1 < m_pad) ? s_cnt[b + 1] : total;
      const uint32_t hist = tend - tstart;
      uint32_t g = s_run[b];
      if (a.reverse) {
        g -= hist;
        s_run[b] = g;
      } else {
        s_run[b] = g + hist;
      }
      s_delta[b] = g - tstart;
    }
    if constexpr (REORDER) {
      // Reorder the tile (a local stable multisplit of Section 4.7).
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        if (FULL || off0 + i * 32 < tile_n) {
          const uint32_t b = rb[i] >> 16;
          const uint32_t p = wc[b] + (rb[i] & 0xffffu);
          if (p < T) {
            s_keys[p] = rk[off0 + i * 32];
            if constexpr (PAIRS) s_vals[p] = rv[off0 + i * 32];
            if constexpr (!cheap_bucket<KIND, PAIRS>()) s_bkt[p] = (uint8_t)b;
          } else {
            atomicOr(a.err, kDevErrBounds);
          }
        }
      }
      __syncthreads();
      // the slot is free again: start the copy of the tile STAGES ahead
      if (threadIdx.x == 0) {
        s_pend[slot] = 0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(j + STAGES);
      }
      // Consecutive threads hold consecutive keys of one bucket run: the
      // global writes are coalesced per run.
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const uint32_t p = threadIdx.x + k * THREADS;
        if (FULL || p < tile_n) {
          const uint32_t kq = s_keys[p];
          uint32_t b;
          if constexpr (cheap_bucket<KIND, PAIRS>())
            b = bucket_of<KIND, NB>(kq, sp, s_tbl, s_lut);
          else
            b = s_bkt[p];
          const uint32_t g = s_delta[b] + p;
          if (g < a.n) {
            __stcs(a.keys_out + g, kq);
            if constexpr (PAIRS) __stcs(a.vals_out + g, s_vals[p]);
          } else {
            atomicOr(a.err, kDevErrBounds);
          }
        }
      }
    } else {
      __syncthreads();  // s_delta ready
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        if (FULL || off0 + i * 32 < tile_n) {
          const uint32_t b = rb[i] >> 16;
          const uint32_t g = s_delta[b] + wc[b] + (rb[i] & 0xffffu);
          if (g < a.n) {
            __stcs(a.keys_out + g, rk[off0 + i * 32]);
            if constexpr (PAIRS) __stcs(a.vals_out + g, rv[off0 + i * 32]);
          } else {
            atomicOr(a.err, kDevErrBounds);
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        s_pend[slot] = 0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(j + STAGES);
      }
    }
    __syncthreads();
    return true;
  };

  for (uint32_t j = 0; j < ntiles; ++j) {
    const bool ok = is_full(j) ? tile_body(std::true_type{}, j) : tile_body(std::false_type{}, j);
    if (!ok) {
      // a copy never completed: wait (bounded) for the copies still in flight, then stop
      if (threadIdx.x == 0)
        for (int k = 0; k < STAGES; ++k)
          if (s_pend[k] != 0u) mbar_wait(s_bar + k, (phase >> k) & 1u, a.err);
      __syncthreads();
      return;
    }
  }
}

template <int KIND, int NW, int ITEMS, bool PAIRS, int RANK, int REORDER, int STAGES>
__host__ size_t postscan_smem_bytes(uint32_t m_pad, uint32_t lut_bits) {
  return PostLayout<KIND, NW, ITEMS, PAIRS, RANK, REORDER, STAGES>::bytes(m_pad, lut_bits);
}

}  // namespace ms
