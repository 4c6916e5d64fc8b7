// ms_kernels.cuh -- the local stages of the multisplit (Section 4.6 / 5.3):
// pre-scan (per-chunk bucket histograms) and post-scan (stable local offsets,
// block-level reordering in shared memory, coalesced scatter).  The global
// stage between them is ms_scan.cuh.
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
// window of 32 keys may cost only ~11 ALU instructions in the pre-scan and ~22
// in the post-scan.  Hence:
//  * pre-scan: every lane keeps private 8-bit counters per bucket in shared
//    memory (a load and a store per key, no voting); warps flush them into
//    32-bit totals before any can overflow;
//  * post-scan ranks: for m <= 4 the ballot voting of Section 5.4 (Alg. 2 and
//    the corrected Alg. 3: one ballot per bucket bit); for larger m a per-warp
//    "peer table" in shared memory: each lane ORs its lane bit into the entry
//    of its bucket, reads back the mask of its peers, and the lowest peer
//    advances the warp's counter of that bucket (the same information the
//    ballots give, at a cost that does not grow with log m).
#pragma once

#include "ms_bucket.cuh"

namespace ms {

enum RankMode : int { kRankBallot = 0, kRankTable = 1 };

struct PrescanArgs {
  const uint32_t* keys;
  uint32_t n;
  DevSpec sp;
  uint32_t tiles_per_cta;  // K: tiles of one chunk
  uint32_t num_tiles;      // L = ceil(n / T)
  uint32_t G;              // chunks (CTAs)
  uint32_t* H;             // m * G, bucket-major
  uint32_t prefetch;       // 1: bulk-prefetch the next tiles into L2
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
  const uint32_t* Gx;  // exclusive scan of row-vectorised H (m*G entries)
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

// Adds one warp's per-lane byte counters into its 32-bit totals and clears
// them: lane l handles buckets l, l+32, ...; a row of 32 bytes is summed with
// four-way byte dot products.
__device__ __forceinline__ void prescan_flush(uint8_t* wbytes, uint32_t* wtot, uint32_t m_pad, uint32_t lane) {
  __syncwarp();
  for (uint32_t b = lane; b < m_pad; b += 32) {
    uint4* row = reinterpret_cast<uint4*>(wbytes + b * 32);
    const uint4 x = row[0], y = row[1];
    uint32_t s = 0;
    s = __dp4a(x.x, 0x01010101u, s);
    s = __dp4a(x.y, 0x01010101u, s);
    s = __dp4a(x.z, 0x01010101u, s);
    s = __dp4a(x.w, 0x01010101u, s);
    s = __dp4a(y.x, 0x01010101u, s);
    s = __dp4a(y.y, 0x01010101u, s);
    s = __dp4a(y.z, 0x01010101u, s);
    s = __dp4a(y.w, 0x01010101u, s);
    wtot[b] += s;
    row[0] = make_uint4(0u, 0u, 0u, 0u);
    row[1] = make_uint4(0u, 0u, 0u, 0u);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Pre-scan.  Dynamic shared memory (words): splitter table (256), LUT, then
// per warp m_pad x 32 byte counters (m_pad * 8 words), then per warp m_pad
// 32-bit totals.
template <int KIND, int NB, int NW, int ITEMS>
__global__ void __launch_bounds__(NW * 32, 3) k_prescan(PrescanArgs a) {
  constexpr int T = NW * 32 * ITEMS;
  extern __shared__ __align__(16) uint32_t smem[];
  const DevSpec& sp = a.sp;
  const uint32_t m_pad = sp.m_pad;
  uint32_t* s_tbl = smem;
  uint2* s_lut = reinterpret_cast<uint2*>(smem + 256);
  uint32_t* s_bytes = smem + 256 + lut_words<KIND>(sp.lut_bits);  // NW * m_pad * 8 words
  uint32_t* s_tot = s_bytes + NW * m_pad * 8;                      // NW * m_pad words

  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint8_t* wbytes = reinterpret_cast<uint8_t*>(s_bytes + w * m_pad * 8);  // [b][lane]
  uint32_t* wtot = s_tot + w * m_pad;
  for (uint32_t i = threadIdx.x; i < NW * m_pad * 9; i += NW * 32) s_bytes[i] = 0u;  // bytes + totals
  build_bucket_tables<KIND, NB>(sp, s_tbl, s_lut);  // ends with a barrier

  const uint32_t c = blockIdx.x;
  const uint32_t t0 = c * a.tiles_per_cta;
  const uint32_t t1 = min(t0 + a.tiles_per_cta, a.num_tiles);
  uint32_t since_flush = 0;  // keys counted per lane since the last flush
  for (uint32_t tile = t0; tile < t1; ++tile) {
    if (a.prefetch && threadIdx.x == 0 && tile + 2 < t1 && (size_t)(tile + 3) * T <= a.n)
      prefetch_l2(a.keys + (size_t)(tile + 2) * T, T * 4u);  // a full tile only
    const uint32_t* src = a.keys + (size_t)tile * T;
    const uint32_t rem = (uint32_t)min((size_t)T, (size_t)a.n - (size_t)tile * T);
    const uint32_t off0 = w * (32 * ITEMS) + lane;
    uint32_t key[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) key[i] = (off0 + i * 32 < rem) ? src[off0 + i * 32] : 0u;
    if (since_flush + ITEMS > 255u) {
      prescan_flush(wbytes, wtot, m_pad, lane);
      since_flush = 0;
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (off0 + i * 32 < rem) {
        const uint32_t b = bucket_of<KIND, NB>(key[i], sp, s_tbl, s_lut);
        uint8_t* p = wbytes + b * 32 + lane;
        *p = (uint8_t)(*p + 1u);
      }
    }
    since_flush += ITEMS;
  }
  prescan_flush(wbytes, wtot, m_pad, lane);
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < sp.m; b += NW * 32) {
    uint32_t s = 0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) s += s_tot[ww * m_pad + b];
    a.H[(size_t)b * a.G + c] = s;
  }
}

template <int KIND, int NW>
__host__ size_t prescan_smem_bytes(uint32_t m_pad, uint32_t lut_bits) {
  return 4u * (256u + lut_words<KIND>(lut_bits) + NW * m_pad * 9u);
}

// ---------------------------------------------------------------------------
// Post-scan.  Dynamic shared memory (words): splitter table (256), LUT,
// s_run / s_delta (256 each), s_warp (32), counters NW*(m_pad+1), peer tables
// NW*m_pad (table mode), then the reorder buffers: T keys, T values (pairs),
// T bucket bytes.
template <int KIND, int NB, int NW, int ITEMS, bool PAIRS, int RANK>
__global__ void __launch_bounds__(NW * 32, PAIRS ? 2 : 3) k_postscan(PostscanArgs a) {
  constexpr int THREADS = NW * 32;
  constexpr int T = THREADS * ITEMS;
  static_assert(NW >= 8, "the per-bucket phase needs >= 256 threads");
  static_assert(NW == 8 || NW == 16 || NW == 32, "NW must be 8, 16 or 32");
  constexpr int LOGNW = NW == 8 ? 3 : NW == 16 ? 4 : 5;
  extern __shared__ __align__(16) uint32_t smem[];
  const DevSpec& sp = a.sp;
  const uint32_t m = sp.m, m_pad = sp.m_pad, S = m_pad + 1;
  uint32_t* s_tbl = smem;
  uint2* s_lut = reinterpret_cast<uint2*>(smem + 256);
  uint32_t* s_run = smem + 256 + lut_words<KIND>(sp.lut_bits);
  uint32_t* s_delta = s_run + 256;
  uint32_t* s_warp = s_delta + 256;
  uint32_t* s_cnt = s_warp + 32;                                       // [w * S + b]
  uint32_t* s_peer = s_cnt + NW * S;                                   // [w * m_pad + b]
  uint32_t* s_keys = s_peer + (RANK == kRankTable ? NW * m_pad : 0u);  // T
  uint32_t* s_vals = s_keys + T;                                       // T (pairs)
  uint8_t* s_bkt = reinterpret_cast<uint8_t*>(s_keys + T * (PAIRS ? 2 : 1));

  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t c = blockIdx.x;
  const uint32_t len = m * a.G;
  if (RANK == kRankTable)
    for (uint32_t i = threadIdx.x; i < NW * m_pad; i += THREADS) s_peer[i] = 0u;
  // next global position of each bucket: chunk start (forward) or chunk end (reverse)
  for (uint32_t b = threadIdx.x; b < m; b += THREADS) {
    const uint32_t e = b * a.G + c;
    s_run[b] = a.reverse ? ((e + 1 < len) ? a.Gx[e + 1] : a.n) : a.Gx[e];
  }
  build_bucket_tables<KIND, NB>(sp, s_tbl, s_lut);  // ends with a barrier

  uint32_t* wc = s_cnt + w * S;
  uint32_t* wpeer = s_peer + w * m_pad;
  const uint32_t lt_mask = lanemask_lt();
  // Alg. 2: per ballot, the mask that keeps the lanes whose bucket bit equals
  // the same bit of this lane's id
  uint32_t lane_x[NB > 0 ? NB : 1];
#pragma unroll
  for (int k = 0; k < NB; ++k) lane_x[k] = ((lane >> k) & 1u) ? 0u : 0xffffffffu;

  const uint32_t t0 = c * a.tiles_per_cta;
  const uint32_t t1 = min(t0 + a.tiles_per_cta, a.num_tiles);
  const uint32_t ntiles = t1 > t0 ? t1 - t0 : 0u;
  for (uint32_t j = 0; j < ntiles; ++j) {
    const uint32_t tile = a.reverse ? t1 - 1 - j : t0 + j;
    if (a.prefetch && threadIdx.x == 0 && j + 2 < ntiles) {
      const uint32_t pt = a.reverse ? t1 - 3 - j : t0 + j + 2;
      if ((size_t)(pt + 1) * T <= a.n) {  // a full tile only
        prefetch_l2(a.keys_in + (size_t)pt * T, T * 4u);
        if constexpr (PAIRS) prefetch_l2(a.vals_in + (size_t)pt * T, T * 4u);
      }
    }
    const size_t tbase = (size_t)tile * T;
    const uint32_t tile_n = (uint32_t)min((size_t)T, (size_t)a.n - tbase);
    const uint32_t off0 = w * (32 * ITEMS) + lane;
    const uint32_t* ksrc = a.keys_in + tbase;
    const uint32_t* vsrc = PAIRS ? a.vals_in + tbase : nullptr;
    uint32_t key[ITEMS], val[ITEMS], rb[ITEMS];  // rb: rank in warp (low 16 bits) | bucket << 16
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = off0 + i * 32 < tile_n;
      key[i] = valid ? __ldcs(ksrc + off0 + i * 32) : 0u;
      if constexpr (PAIRS) val[i] = valid ? __ldcs(vsrc + off0 + i * 32) : 0u;
    }
    for (uint32_t b = lane; b < m_pad; b += 32) wc[b] = 0u;
    __syncwarp();
    uint32_t run = 0;  // ballot mode: keys of bucket `lane` in earlier windows of this warp
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool valid = off0 + i * 32 < tile_n;
      const uint32_t b = valid ? bucket_of<KIND, NB>(key[i], sp, s_tbl, s_lut) : 0u;
      if constexpr (RANK == kRankBallot) {
        // Section 5.4 / Alg. 2 / Alg. 3: NB ballots give every lane the
        // bucket of every lane of the window.
        const uint32_t vb = __ballot_sync(kFull, valid);
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
      } else {
        // peer table: OR the lane bit into the bucket's entry, read the peers
        if (valid) atomicOr(wpeer + b, 1u << lane);
        __syncwarp();
        const uint32_t own = valid ? wpeer[b] : 0u;
        __syncwarp();
        const uint32_t lt = own & lt_mask;
        uint32_t before = 0;
        if (valid && lt == 0u) {  // lowest peer: advance the counter, clear the entry
          before = wc[b];
          wc[b] = before + __popc(own);
          wpeer[b] = 0u;
        }
        __syncwarp();
        before = __shfl_sync(kFull, before, (__ffs(own) - 1) & 31);
        rb[i] = (before + __popc(lt)) | (b << 16);
      }
    }
    if constexpr (RANK == kRankBallot) wc[lane] = (lane < m) ? run : 0u;
    __syncthreads();

    // One exclusive scan over the (bucket, warp) counters in bucket-major
    // order gives, for every warp and bucket, where its keys start in the
    // reordered tile: earlier buckets of the tile (Section 5.6.2, item 2) plus
    // earlier warps of the same bucket (Section 5.5.4, third term).
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

    // Reorder the tile (a local stable multisplit) and compute, per bucket,
    // global position minus tile position.
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
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (off0 + i * 32 < tile_n) {
        const uint32_t b = rb[i] >> 16;
        const uint32_t p = wc[b] + (rb[i] & 0xffffu);
        if (p < (uint32_t)T) {
          s_keys[p] = key[i];
          if constexpr (PAIRS) s_vals[p] = val[i];
          s_bkt[p] = (uint8_t)b;
        } else {
          atomicOr(a.err, kDevErrBounds);
        }
      }
    }
    __syncthreads();

    // Consecutive threads hold consecutive keys of one bucket run: the global
    // writes are coalesced per run.
#pragma unroll 4
    for (uint32_t p = threadIdx.x; p < tile_n; p += THREADS) {
      const uint32_t g = s_delta[s_bkt[p]] + p;
      if (g < a.n) {
        __stcs(a.keys_out + g, s_keys[p]);
        if constexpr (PAIRS) __stcs(a.vals_out + g, s_vals[p]);
      } else {
        atomicOr(a.err, kDevErrBounds);
      }
    }
    __syncthreads();
  }
}

template <int KIND, int NW, int ITEMS, bool PAIRS, int RANK>
__host__ size_t postscan_smem_bytes(uint32_t m_pad, uint32_t lut_bits) {
  constexpr uint32_t T = NW * 32 * ITEMS;
  return 4u * (256u + lut_words<KIND>(lut_bits) + 256u + 256u + 32u + NW * (m_pad + 1u) +
               (RANK == kRankTable ? NW * m_pad : 0u) + T * (PAIRS ? 2u : 1u)) +
         T;
}

}  // namespace ms
