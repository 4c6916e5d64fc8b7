// ms_batch_tc.cuh -- the persistent batched multisplit (ms_batch.cu) for up to
// 32 buckets, solving each tile with the per-thread bucket counters of
// ms_tc.cuh.
//
// Same work list and protocol as k_batch, with items of up to K tiles:
// histogram items of multi-tile segments first (chunk histogram -> column of
// the segment's H; the CTA that finishes a segment's last histogram scans its
// H and raises the ready flag), then the post-scan items.  Differences: a
// histogram item only counts (one shared atomic per key, no ranks), reading
// its keys straight from global memory with 16-byte loads at any segment
// phase; a post-scan item walks its tiles in order, each CTA copying the next
// tile -- of the same item, or the next item's first -- into the other of two
// shared-memory slots with asynchronous copies while it works on the current
// one (16-byte copies for the chunks of any segment phase, see
// copy_tile_shifted).  Items are taken by ticket, three tickets ahead of the
// current item; a waiting post-scan item only waits for histogram items of
// smaller tickets, which never wait, so every wait ends.
#pragma once

#include "ms_tc.cuh"

namespace ms {

__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t* dst, const uint32_t* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies the n <= T words at src (4-byte aligned, any phase) into a slot
// region: word p lands at tc_swz(p + r), r = the word phase of src modulo 4,
// so that src's 16-byte chunks land on 16-byte chunks of the region and go
// by 16-byte copies; the at most 3 words before the first chunk and after the
// last go by 4-byte copies.  The region needs T + 32 words.  All threads of
// the block call it.
__device__ __forceinline__ void copy_tile_shifted(uint32_t* dst, const uint32_t* src, uint32_t n) {
  const uint32_t t = threadIdx.x;
  const uint32_t r = (uint32_t)(reinterpret_cast<uintptr_t>(src) >> 2) & 3u;
  const uint32_t h = min(n, (4u - r) & 3u);  // head words
  const uint32_t nch = (n - h) >> 2;         // whole 16-byte chunks after the head
  for (uint32_t k = t; k < nch; k += kTcThreads) {
    const uint32_t p = h + 4u * k;
    cp_async16(dst + tc_swz(p + r), src + p);
  }
  const uint32_t tail0 = h + 4u * nch;
  if (t < h) cp_async4(dst + tc_swz(t + r), src + t);
  if (t >= 4u && t - 4u < n - tail0) cp_async4(dst + tc_swz(tail0 + (t - 4u) + r), src + tail0 + (t - 4u));
}

// The 16 words of positions [16t, 16t+16) of a region filled by
// copy_tile_shifted with phase r (uniform over the block): five 16-byte
// loads and a shift by r.
__device__ __forceinline__ void read16_shifted(const uint32_t* region, uint32_t r, uint32_t (&out)[16]) {
  uint32_t w[20];
  const uint32_t t = threadIdx.x;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const uint4 v = *reinterpret_cast<const uint4*>(region + tc_swz(16u * t + 4u * c));
    w[4 * c + 0] = v.x;
    w[4 * c + 1] = v.y;
    w[4 * c + 2] = v.z;
    w[4 * c + 3] = v.w;
  }
  switch (r) {
#define MS_SHIFT_CASE(R)                                 \
  case R:                                                \
    _Pragma("unroll") for (int e = 0; e < 16; ++e) out[e] = w[e + R]; \
    break;
    MS_SHIFT_CASE(0)
    MS_SHIFT_CASE(1)
    MS_SHIFT_CASE(2)
    default:
      _Pragma("unroll") for (int e = 0; e < 16; ++e) out[e] = w[e + 3];
#undef MS_SHIFT_CASE
  }
}

// Dynamic shared memory (words): two slots (keys T + 32, then values T + 32
// for pairs), counters R * 288, bucket bytes (T), splitter table 32, lookup
// table.
template <int KIND, bool PAIRS>
struct BatchTcLayout {
  static constexpr uint32_t T = kTcTile;
  static constexpr uint32_t kRegion = T + 32;
  static constexpr uint32_t kSlotWords = kRegion * (PAIRS ? 2 : 1);
  static __host__ __device__ uint32_t cnt() { return 2 * kSlotWords; }
  static __host__ __device__ uint32_t bkt(uint32_t R) { return cnt() + R * kTcRow; }
  static __host__ __device__ uint32_t tbl(uint32_t R) { return bkt(R) + T / 4; }
  static __host__ __device__ uint32_t lut(uint32_t R) { return tbl(R) + 32; }
  static __host__ size_t bytes(uint32_t m, uint32_t lb, uint32_t lw) {
    return 4u * (size_t)(lut(tc_rows(m)) + tc_lut_words(KIND, lb, lw));
  }
};

template <int KIND, bool PAIRS>
__global__ void __launch_bounds__(kTcThreads, 2) k_batch_tc(BatchArgs a, uint32_t lb, uint32_t lw) {
  using Lay = BatchTcLayout<KIND, PAIRS>;
  constexpr uint32_t T = Lay::T;
  constexpr uint32_t SW = Lay::kSlotWords;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_tk[4], s_flag;
  __shared__ uint32_t s_delta[kTcMaxM], s_start[kTcMaxM];
  __shared__ __align__(16) uint32_t s_warp[8];
  const DevSpec& sp = a.sp;
  const uint32_t m = sp.m, R = tc_rows(m);
  uint32_t* s_cnt = smem + Lay::cnt();
  uint8_t* s_bkt = reinterpret_cast<uint8_t*>(smem + Lay::bkt(R));
  uint32_t* s_tbl = smem + Lay::tbl(R);
  uint32_t* s_lut = smem + Lay::lut(R);
  const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5;
  const TcLut L{s_lut, 32u - lb, lw, lane & ((1u << lw) - 1u), (1u << (32u - lb)) - 1u, s_tbl};
  uint32_t* my = s_cnt + t + ((t >> 5) << 2);  // counter (bucket 0, thread t)

  for (uint32_t i = t; i < R * kTcRow; i += kTcThreads) s_cnt[i] = 0u;
  tc_build_tables<KIND>(sp, lb, lw, s_tbl, s_lut);  // ends with a barrier
  const uint2 counts = a.items[0];  // read from memory so a captured graph follows later updates
  const uint32_t n_items = counts.y;
  const uint64_t pol_last = policy_evict_last();

  // all threads: copy tile t0 + j of post-scan item `it` (keys, and values
  // for pairs) into `slot`, laid out as ms_tc.cuh's swizzled tiles; one
  // commit group per call, empty or not (histogram items read their keys
  // straight from global memory)
  auto fetch = [&](uint32_t it, uint32_t j, uint32_t slot) {
    if (it < n_items) {
      const uint2 item = a.items[1 + it];
      if (item.y & kBatchPost) {
        const DevSeg sg = a.segs[item.x];
        const size_t tb = (size_t)((item.y & ~kBatchPost) + j) * T;
        const uint32_t tile_n = (size_t)sg.n > tb ? (uint32_t)min((size_t)T, (size_t)sg.n - tb) : 0u;
        uint32_t* sk = smem + slot * SW;
        copy_tile_shifted(sk, sg.kin + tb, tile_n);
        if constexpr (PAIRS) copy_tile_shifted(sk + Lay::kRegion, sg.vin + tb, tile_n);
      }
    }
    cp_async_commit();
  };

  // histogram item: the n keys at src (any 4-byte phase) into this thread's
  // (bucket, thread) counters -- the 16-byte chunks inside the tile by
  // 16-byte loads, the at most 3 words before the first chunk and after the
  // last by 4-byte loads (measured on GB300: the next tile's loads in flight
  // while one is counted made the batched run 1.6% slower)
  auto count_tile = [&](const uint32_t* src, uint32_t n) {
    const uint32_t r = (uint32_t)(reinterpret_cast<uintptr_t>(src) >> 2) & 3u;
    const uint32_t h = min(n, (4u - r) & 3u);
    const uint32_t nch = (n - h) >> 2;  // at most T / 4 = 4 * kTcThreads
    uint32_t key[16], bk[16];
    uint32_t valid = 0;  // bit i: key[i] is a key of the tile
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t k = t + kTcThreads * j;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (k < nch) {
        v = ldg_v4_policy(src + h + 4u * k, pol_last);
        valid |= 0xfu << (4 * j);
      }
      key[4 * j + 0] = v.x;
      key[4 * j + 1] = v.y;
      key[4 * j + 2] = v.z;
      key[4 * j + 3] = v.w;
    }
    uint32_t flag = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) bk[i] = tc_bucket<KIND>(key[i], sp, L, flag);
    if constexpr (KIND == kRange)
      if (flag & kTcLutFlag) tc_fixup<16>(key, bk, L, s_tbl, m);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if ((valid >> i) & 1u) atomicAdd(my + bk[i] * kTcRow, 1u);
    const uint32_t tail0 = h + 4u * nch;
    const bool head = t < h, tail = t >= 4u && t - 4u < n - tail0;
    if (head || tail) {
      const uint32_t u = src[head ? t : tail0 + (t - 4u)];
      uint32_t f = 0;
      uint32_t b = tc_bucket<KIND>(u, sp, L, f);
      if constexpr (KIND == kRange)
        if (f & kTcLutFlag) b = range_search<5>(u, s_tbl, m);
      atomicAdd(my + b * kTcRow, 1u);
    }
  };

  // Tickets are taken three items ahead, and the descriptors of the later
  // items are pulled into L1 in two steps (the item entry, then the segment
  // it names) while the current item is worked on, so that the copy of the
  // next item's first tile starts without waiting on their loads.  (Holding
  // unstarted tickets is safe: a blocked CTA's current item waits only for
  // histogram items of smaller tickets, and the CTA holding one of those is
  // either working on it or blocked on a still smaller ticket, so the CTA
  // with the smallest blocked ticket can always proceed.)
  auto prefetch_l1 = [](const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); };
  if (t == 0) {
    s_tk[0] = atomicAdd(a.ticket, 1u);
    s_tk[1] = atomicAdd(a.ticket, 1u);
    s_tk[2] = atomicAdd(a.ticket, 1u);
    for (int k = 1; k < 3; ++k)
      if (s_tk[k] < n_items) prefetch_l1(a.items + 1 + s_tk[k]);
  }
  __syncthreads();
  uint32_t cur = s_tk[0], nxt = s_tk[1], nxt2 = s_tk[2];
  uint32_t slot = 0;  // where the next post-scan tile is (being) copied
  fetch(cur, 0, 0);

  while (cur < n_items) {
    const uint2 item = a.items[1 + cur];
    const uint32_t seg = item.x, t0 = item.y & ~kBatchPost;
    const DevSeg sg = a.segs[seg];
    const uint32_t t1 = min(t0 + a.K, sg.L), chunk = t0 / a.K;
    const bool hist = (item.y & kBatchPost) == 0u;
    uint32_t nn = 0;    // the ticket taken during this item
    uint32_t grun = 0;  // post-scan, thread b < m: global position of bucket b's next key of this chunk

    for (uint32_t tile = t0; tile < t1; ++tile) {
      const bool last = tile + 1u == t1;
      if (hist) {
        // (A) this tile's keys into the chunk's per-thread counts; at the
        // chunk's last tile, the next item's first tile into `slot`, free
        // since the last post-scan tile (in the other slot) was written out
        if (last) {
          __syncthreads();  // everyone read s_tk[3]
          if (t == 0) {
            if (nxt2 < n_items) prefetch_l1(a.segs + a.items[1 + nxt2].x);
            const uint32_t tk = atomicAdd(a.ticket, 1u);
            s_tk[3] = tk;
            if (tk < n_items) prefetch_l1(a.items + 1 + tk);
          }
          fetch(nxt, 0, slot);
          __syncthreads();
          nn = s_tk[3];
        }
        const size_t tb = (size_t)tile * T;
        count_tile(sg.kin + tb, (uint32_t)min((size_t)T, (size_t)sg.n - tb));
        continue;
      }
      __syncthreads();  // the other slot's tile is written out; everyone read s_tk[3]
      if (last) {
        if (t == 0) {
          if (nxt2 < n_items) prefetch_l1(a.segs + a.items[1 + nxt2].x);  // its entry came in an item ago
          const uint32_t tk = atomicAdd(a.ticket, 1u);
          s_tk[3] = tk;
          if (tk < n_items) prefetch_l1(a.items + 1 + tk);
        }
        fetch(nxt, 0, slot ^ 1u);
      } else {
        fetch(cur, tile + 1u - t0, slot ^ 1u);
      }
      cp_async_wait<1>();  // this thread's copies of the current tile landed
      __syncthreads();     // everyone's
      if (last) nn = s_tk[3];

      const size_t tb = (size_t)tile * T;
      const uint32_t tile_n = (size_t)sg.n > tb ? (uint32_t)min((size_t)T, (size_t)sg.n - tb) : 0u;
      uint32_t* sk = smem + slot * SW;
      uint32_t* sv = sk + Lay::kRegion;
      (void)sv;

      uint32_t key[16], bk[16];
      read16_shifted(sk, (uint32_t)(reinterpret_cast<uintptr_t>(sg.kin + tb) >> 2) & 3u, key);
      uint32_t flag = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) bk[i] = tc_bucket<KIND>(key[i], sp, L, flag);
      if constexpr (KIND == kRange)
        if (flag & kTcLutFlag) tc_fixup<16>(key, bk, L, s_tbl, m);

      {
        // (B) post-scan of one tile
        uint32_t val[PAIRS ? 16 : 1], pos[16];
        if constexpr (PAIRS)
          read16_shifted(sv, (uint32_t)(reinterpret_cast<uintptr_t>(sg.vin + tb) >> 2) & 3u, val);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (16u * t + i < tile_n) pos[i] = atomicAdd(my + bk[i] * kTcRow, 1u);
        __syncthreads();
        {
          uint4* segc = reinterpret_cast<uint4*>(s_cnt + tc_pad(t * R));
          uint32_t sum = 0;
          for (uint32_t g = 0; g < R / 4u; ++g) {
            const uint4 v = segc[g];
            sum += v.x + v.y + v.z + v.w;
          }
          uint32_t total;
          uint32_t run = tc_block_scan(sum, s_warp, &total);
          if (((t * R) & 255u) == 0u) {
            const uint32_t b = (t * R) >> 8;
            if (b < m) s_start[b] = run;
          }
          for (uint32_t g = 0; t * R < m * 256u && g < R / 4u; ++g) {
            const uint4 v = segc[g];
            uint4 o;
            o.x = run;
            run += v.x;
            o.y = run;
            run += v.y;
            o.z = run;
            run += v.z;
            o.w = run;
            run += v.w;
            segc[g] = o;
          }
        }
        __syncthreads();
        // global base of each bucket for this tile
        if (t < m) {
          const uint32_t start = s_start[t];
          if (sg.L == 1u) {
            s_delta[t] = 0u;  // the tile is the segment
            if (sg.offsets != nullptr) {
              sg.offsets[t] = start;
              if (t == 0) sg.offsets[m] = tile_n;
            }
          } else {
            if (tile == t0) {
              uint32_t spins = 0;
              while (ld_acquire_u32(a.ready + seg) == 0u) {
                // give up at the bound, or at once when another wait has already given up
                if (++spins > kSpinLimit || (spins > 64 && (*(volatile uint32_t*)a.err & kDevErrTimeout))) {
                  atomicOr(a.err, kDevErrTimeout);
                  break;
                }
                __nanosleep(spins < 64 ? 64 : 512);
              }
              grun = __ldcg(a.H + sg.hoff + t * sg.C + chunk);
            }
            const uint32_t end = (t + 1u < m) ? s_start[t + 1u] : tile_n;
            s_delta[t] = grun - start;
            grun += end - start;
          }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (16u * t + i < tile_n) pos[i] += my[bk[i] * kTcRow];
        for (uint32_t b = 0; b < m; ++b) my[b * kTcRow] = 0u;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (16u * t + i < tile_n) {
            const uint32_t p = pos[i];
            if (p < T) {
              sk[tc_rswz(p)] = key[i];
              if constexpr (PAIRS) sv[tc_rswz(p)] = val[i];
              s_bkt[tc_rswz(p)] = (uint8_t)bk[i];
            } else {
              atomicOr(a.err, kDevErrBounds);
            }
          }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const uint32_t p = t + k * kTcThreads;
          if (p < tile_n) {
            const uint32_t q = tc_rswz(p);
            const uint32_t g = s_delta[s_bkt[q]] + p;
            if (g < sg.n) {
              __stcs(sg.kout + g, sk[q]);
              if constexpr (PAIRS) __stcs(sg.vout + g, sv[q]);
            } else {
              atomicOr(a.err, kDevErrBounds);
            }
          }
        }
      }
      slot ^= 1u;
    }

    if (hist) {
      // the chunk's counts -> column `chunk` of the segment's H
      __syncthreads();
      for (uint32_t b = w; b < m; b += kTcThreads / 32) {
        uint32_t* row = s_cnt + b * kTcRow + lane;
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          s += row[36 * k];
          row[36 * k] = 0u;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
        if (lane == 0) a.H[sg.hoff + b * sg.C + chunk] = s;
      }
      __threadfence();
      __syncthreads();
      if (t == 0) s_flag = (atomicAdd(a.done + seg, 1u) == sg.C - 1u) ? 1u : 0u;
      __syncthreads();
      if (s_flag) {
        // last histogram of the segment: exclusive scan of its H (m * C
        // words, bucket-major), bucket offsets, then the ready flag
        __threadfence();
        const uint32_t len = m * sg.C;
        uint32_t* Hs = a.H + sg.hoff;
        uint32_t carry = 0;
        for (uint32_t base = 0; base < len; base += kTcTile) {
          uint32_t v[16];
          uint32_t sum = 0;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const uint32_t idx = base + 16u * t + i;
            v[i] = idx < len ? __ldcg(Hs + idx) : 0u;
            sum += v[i];
          }
          uint32_t total;
          uint32_t run = carry + tc_block_scan(sum, s_warp, &total);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const uint32_t idx = base + 16u * t + i;
            if (idx < len) {
              Hs[idx] = run;
              if (sg.offsets != nullptr && idx % sg.C == 0u) sg.offsets[idx / sg.C] = run;
            }
            run += v[i];
          }
          carry += total;
          __syncthreads();  // s_warp is rewritten by the next round
        }
        if (sg.offsets != nullptr && t == 0) sg.offsets[m] = carry;
        __threadfence();
        __syncthreads();
        if (t == 0) st_release_u32(a.ready + seg, 1u);
      }
    }
    cur = nxt;
    nxt = nxt2;
    nxt2 = nn;
  }
  cp_async_wait<0>();  // nothing may be in flight into shared memory at exit
}

}  // namespace ms
