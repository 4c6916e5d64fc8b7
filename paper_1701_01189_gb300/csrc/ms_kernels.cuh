// ms_kernels.cuh -- the three stages of the multisplit (Section 4.6 / 5.3):
// pre-scan (local histograms), global scan of the histogram matrix H, and
// post-scan (local offsets, block-level reordering, coalesced scatter).
//
// Localization (Section 4.4, Section 5.3 "Block-level Multisplit"): each CTA
// owns a chunk of consecutive tiles (first level); a tile of T = NW*32*ITEMS
// keys is reordered as a whole (second level); each warp owns ITEMS
// consecutive 32-key windows of the tile (third level); each window is solved
// directly with warp ballots (fourth level).  H has one column per CTA chunk
// and is stored bucket-major, H[b * G + c], so that one exclusive scan over
// the row-vectorised H yields both global terms of Eq. 2.
#pragma once

#include "ms_device.cuh"

namespace ms {

struct PrescanArgs {
  const uint32_t* keys;
  uint32_t n;
  DevSpec sp;
  uint32_t tiles_per_cta;  // K: tiles of one chunk
  uint32_t num_tiles;      // L = ceil(n / T)
  uint32_t G;              // chunks (CTAs)
  uint32_t* H;             // m * G, bucket-major
};

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
  const uint32_t* Gx;  // exclusive scan of row-vectorised H
  uint32_t* err;       // device status word
};

// Shared memory words used by both kernels before the tile buffers.
template <int NW, bool SMALLM>
struct SmemLayout {
  static constexpr int kStride = SMALLM ? 32 : kMaxM;  // counters per warp
  static constexpr int kTbl = 0;                      // 256 splitter-table words
  static constexpr int kCnt = 256;                    // NW * kStride counters
  static constexpr int kRun = kCnt + NW * kStride;    // 256: next global position per bucket
  static constexpr int kDelta = kRun + 256;           // 256: global - tile position per bucket
  static constexpr int kWarp = kDelta + 256;          // 32: scan scratch
  static constexpr int kWords = kWarp + 32;
};

template <int NW, int ITEMS, bool SMALLM, bool PAIRS>
constexpr size_t postscan_smem_bytes() {
  using Lay = SmemLayout<NW, SMALLM>;
  constexpr int T = NW * 32 * ITEMS;
  return sizeof(uint32_t) * (Lay::kWords + T * (PAIRS ? 2 : 1)) + T;  // + one byte per key
}

template <int NW, bool SMALLM>
constexpr size_t prescan_smem_bytes() {
  return sizeof(uint32_t) * SmemLayout<NW, SMALLM>::kWords;
}

// ---------------------------------------------------------------------------
// Pre-scan (Alg. 1, first stage; Section 5.5.1 and 5.5.3): every CTA counts
// the keys of its chunk per bucket and writes column c of H.
template <int KIND, int NW, int ITEMS, bool SMALLM>
__global__ void __launch_bounds__(NW * 32, 2) k_prescan(PrescanArgs a) {
  using Lay = SmemLayout<NW, SMALLM>;
  constexpr int T = NW * 32 * ITEMS;
  extern __shared__ uint32_t smem[];
  uint32_t* s_tbl = smem + Lay::kTbl;
  uint32_t* s_cnt = smem + Lay::kCnt;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const DevSpec& sp = a.sp;

  if constexpr (KIND == kRange) load_splitter_table(sp, s_tbl);
  uint32_t* wcnt = s_cnt + w * Lay::kStride;
  if constexpr (!SMALLM)
    for (uint32_t b = lane; b < sp.m; b += 32) wcnt[b] = 0;
  __syncthreads();

  uint32_t run = 0;  // SMALLM: count of bucket `lane` in this warp's share of the chunk
  const uint32_t c = blockIdx.x;
  const uint32_t t0 = c * a.tiles_per_cta;
  const uint32_t t1 = min(t0 + a.tiles_per_cta, a.num_tiles);
  for (uint32_t tile = t0; tile < t1; ++tile) {
    const size_t base = (size_t)tile * T + (size_t)w * (32 * ITEMS) + lane;
    uint32_t key[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const size_t idx = base + (size_t)i * 32;
      key[i] = (idx < a.n) ? __ldcs(a.keys + idx) : 0u;
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = (base + (size_t)i * 32) < a.n;
      const uint32_t b = bucket_of<KIND>(key[i], sp, s_tbl);
      if constexpr (SMALLM) {
        uint32_t own, lane_bm;
        window_vote<5>(b, valid, sp.nbits, own, lane_bm);
        run += __popc(lane_bm);
      } else {
        const uint32_t peers = __match_any_sync(kFull, valid ? b : 0xffffffffu);
        if (valid && (peers & lanemask_lt()) == 0) wcnt[b] += __popc(peers);
        __syncwarp();
      }
    }
  }
  if constexpr (SMALLM) wcnt[lane] = run;
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < sp.m; b += NW * 32) {
    uint32_t s = 0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) s += s_cnt[ww * Lay::kStride + b];
    a.H[(size_t)b * a.G + c] = s;
  }
}

// ---------------------------------------------------------------------------
// Post-scan (Alg. 1, third stage, with the block-level reordering of Section
// 5.6.2): per tile, recompute buckets, rank every key among the earlier keys
// of its bucket in the tile (window offset + earlier windows of the warp +
// earlier warps, Section 5.5.4), reorder the tile in shared memory by bucket,
// then write each bucket run to its global position
//   Gx[b][c] + (keys of b in earlier tiles of the chunk) + (rank in tile).
template <int KIND, int NW, int ITEMS, bool SMALLM, bool PAIRS>
__global__ void __launch_bounds__(NW * 32, 2) k_postscan(PostscanArgs a) {
  using Lay = SmemLayout<NW, SMALLM>;
  constexpr int THREADS = NW * 32;
  constexpr int T = THREADS * ITEMS;
  extern __shared__ uint32_t smem[];
  uint32_t* s_tbl = smem + Lay::kTbl;
  uint32_t* s_cnt = smem + Lay::kCnt;
  uint32_t* s_run = smem + Lay::kRun;
  uint32_t* s_delta = smem + Lay::kDelta;
  uint32_t* s_warp = smem + Lay::kWarp;
  uint32_t* s_keys = smem + Lay::kWords;
  uint32_t* s_vals = s_keys + T;  // PAIRS only
  uint8_t* s_bkt = reinterpret_cast<uint8_t*>(s_keys + T * (PAIRS ? 2 : 1));

  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const DevSpec& sp = a.sp;
  const uint32_t m = sp.m;
  const uint32_t c = blockIdx.x;

  if constexpr (KIND == kRange) load_splitter_table(sp, s_tbl);
  for (uint32_t b = threadIdx.x; b < m; b += THREADS) s_run[b] = a.Gx[(size_t)b * a.G + c];
  uint32_t* wcnt = s_cnt + w * Lay::kStride;
  __syncthreads();

  const uint32_t t0 = c * a.tiles_per_cta;
  const uint32_t t1 = min(t0 + a.tiles_per_cta, a.num_tiles);
  for (uint32_t tile = t0; tile < t1; ++tile) {
    const size_t tile_base = (size_t)tile * T;
    const uint32_t tile_n = (uint32_t)min((size_t)T, (size_t)a.n - tile_base);
    const size_t base = tile_base + (size_t)w * (32 * ITEMS) + lane;
    uint32_t key[ITEMS], val[ITEMS], bkt[ITEMS], rank[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const size_t idx = base + (size_t)i * 32;
      const bool valid = idx < a.n;
      key[i] = valid ? __ldcs(a.keys_in + idx) : 0u;
      if constexpr (PAIRS) val[i] = valid ? __ldcs(a.vals_in + idx) : 0u;
    }
    if constexpr (!SMALLM) {
      for (uint32_t b = lane; b < m; b += 32) wcnt[b] = 0;
      __syncwarp();
    }
    uint32_t run = 0;  // SMALLM: keys of bucket `lane` in earlier windows of this warp
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = (base + (size_t)i * 32) < a.n;
      const uint32_t b = valid ? bucket_of<KIND>(key[i], sp, s_tbl) : 0u;
      bkt[i] = b;
      if constexpr (SMALLM) {
        uint32_t own, lane_bm;
        window_vote<5>(b, valid, sp.nbits, own, lane_bm);
        const uint32_t before = __shfl_sync(kFull, run, b & 31u);
        rank[i] = before + __popc(own & lanemask_lt());
        run += __popc(lane_bm);
      } else {
        const uint32_t peers = __match_any_sync(kFull, valid ? b : 0xffffffffu);
        const uint32_t lt = peers & lanemask_lt();
        const uint32_t leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && lt == 0) {
          before = wcnt[b];
          wcnt[b] = before + __popc(peers);
        }
        before = __shfl_sync(kFull, before, leader);
        rank[i] = before + __popc(lt);
        __syncwarp();
      }
    }
    if constexpr (SMALLM) {
      wcnt[lane] = run;
    }
    __syncthreads();

    // Per bucket: exclusive scan over warps (Section 5.5.4, third term) and
    // the tile histogram; then an exclusive scan over buckets (Section 5.6.2,
    // item 2) gives where each bucket starts in the reordered tile.
    uint32_t hist = 0;
    const uint32_t b_me = threadIdx.x;
    if (b_me < m) {
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) {
        const uint32_t v = s_cnt[ww * Lay::kStride + b_me];
        s_cnt[ww * Lay::kStride + b_me] = hist;
        hist += v;
      }
    }
    uint32_t total;
    const uint32_t tstart = block_exclusive_scan<NW>(hist, s_warp, &total);
    if (b_me < m) {
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) s_cnt[ww * Lay::kStride + b_me] += tstart;
      const uint32_t g = s_run[b_me];
      s_delta[b_me] = g - tstart;
      s_run[b_me] = g + hist;
    }
    __syncthreads();

    // Reorder the tile in shared memory (a local stable multisplit).
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = (base + (size_t)i * 32) < a.n;
      if (valid) {
        const uint32_t p = wcnt[bkt[i]] + rank[i];
        if (p < (uint32_t)T) {
          s_keys[p] = key[i];
          if constexpr (PAIRS) s_vals[p] = val[i];
          s_bkt[p] = (uint8_t)bkt[i];
        } else {
          atomicOr(a.err, kDevErrBounds);
        }
      }
    }
    __syncthreads();

    // Consecutive threads now hold consecutive keys of one bucket run: the
    // global writes are coalesced per run.
#pragma unroll 4
    for (uint32_t p = threadIdx.x; p < tile_n; p += THREADS) {
      const uint32_t g = s_delta[s_bkt[p]] + p;
      if (g < a.n) {
        a.keys_out[g] = s_keys[p];
        if constexpr (PAIRS) a.vals_out[g] = s_vals[p];
      } else {
        atomicOr(a.err, kDevErrBounds);
      }
    }
    __syncthreads();
  }
}

}  // namespace ms
