// ms_onesweep.cu -- the LSD radix sort of Section 7.1 with one sweep per digit.
//
// Section 7.1 builds the sort from ceil(32/r) multisplits with the radix digit
// f_k(u) = (u >> kr) & (2^r - 1) as bucket identifier; each of those is the
// three-stage multisplit (pre-scan, scan, post-scan), reading the keys twice
// per digit.  On GB300 the per-digit pre-scan is replaced as in the
// "single-sweep" LSD sorts (Adinets and Merrill, "Onesweep", 2022): one kernel
// reads the keys once and counts the digits of every pass (the first term of
// Eq. 2 for every pass, since a histogram does not depend on the order of the
// keys), and each pass is then a single kernel whose tiles obtain the second
// term of Eq. 2 -- the count of their digit in all earlier tiles -- by a
// decoupled look-back over per-tile, per-digit status words, instead of a
// separate scan of a histogram matrix.  The ranking, the scan over (digit,
// warp) counters and the reordered, coalesced writes are the multisplit's own
// (ms_kernels.cuh).  Result: 4 + 8 bytes per key per pass instead of 12.
//
// Status words are 32-bit: bits 31..30 a flag (1: tile aggregate, 2:
// inclusive prefix), bits 29..0 a count, so this path takes n < 2^30.  Two
// status arrays alternate between passes; every tile clears its words of the
// array the next pass will use.  All waits are bounded.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "ms.h"
#include "ms_host.h"
#include "ms_kernels.cuh"
#include "ms_scan.cuh"

namespace ms {

constexpr uint32_t kOsAggregate = 1u << 30;
constexpr uint32_t kOsPrefix = 2u << 30;
constexpr uint32_t kOsValue = (1u << 30) - 1u;
constexpr int kOsNW = 8, kOsItems = 16;
constexpr int kOsLookback = 8;  // predecessors read per look-back step
constexpr uint32_t kOsTile = kOsNW * 32 * kOsItems;  // 4096 keys
constexpr int kHistNW = 8, kHistItems = 16;

__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct RadixHistArgs {
  const uint32_t* keys;
  uint32_t n;
  uint32_t begin_bit, end_bit, passes;
  uint32_t* hist;  // passes * 256, zeroed
};

// Digit histograms of every pass in one read of the keys.  Per warp, 32-bit
// counters [pass][digit] in shared memory; at the end the CTA adds its counts
// into the global histograms.  The passes (at most four) are unrolled with
// their shifts and masks kept in registers: the kernel is bound by its
// instruction issue, not by the bytes it reads.
__global__ void __launch_bounds__(kHistNW * 32) k_radix_hist(RadixHistArgs a) {
  constexpr uint32_t T = kHistNW * 32 * kHistItems;
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t* wh = smem + w * 4 * 256;
  for (uint32_t i = threadIdx.x; i < kHistNW * 4 * 256; i += kHistNW * 32) smem[i] = 0u;
  __syncthreads();
  uint32_t sh[4], mk[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    sh[p] = a.begin_bit + 8u * p;
    const uint32_t bits = (uint32_t)p < a.passes ? min(8u, a.end_bit - sh[p]) : 0u;
    mk[p] = (1u << bits) - 1u;
    sh[p] = min(sh[p], 31u);
  }
  const uint32_t passes = a.passes;
  for (size_t tb = (size_t)blockIdx.x * T; tb < a.n; tb += (size_t)gridDim.x * T) {
    const uint32_t rem = (uint32_t)min((size_t)T, (size_t)a.n - tb);
    const uint32_t off0 = w * (32 * kHistItems) + lane;
    uint32_t key[kHistItems];
#pragma unroll
    for (int i = 0; i < kHistItems; ++i) key[i] = (off0 + i * 32 < rem) ? __ldcs(a.keys + tb + off0 + i * 32) : 0u;
#pragma unroll
    for (int i = 0; i < kHistItems; ++i) {
      if (off0 + i * 32 < rem) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
          if ((uint32_t)p < passes) atomicAdd(wh + p * 256 + ((key[i] >> sh[p]) & mk[p]), 1u);
      }
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < a.passes * 256; i += kHistNW * 32) {
    uint32_t s = 0;
#pragma unroll
    for (int ww = 0; ww < kHistNW; ++ww) s += smem[ww * 4 * 256 + i];
    if (s) atomicAdd(a.hist + i, s);
  }
}

struct OnesweepArgs {
  const uint32_t* keys_in;
  const uint32_t* vals_in;
  uint32_t* keys_out;
  uint32_t* vals_out;
  uint32_t n;
  DevSpec sp;              // radix digit of this pass (kRadix)
  const uint32_t* hist;    // this pass's digit histogram (m entries)
  uint32_t* status;        // this pass: num_tiles * 256 words, zero
  uint32_t* status_next;   // the next pass's array: cleared here
  uint32_t* ticket;        // zero
  uint32_t* err;
  uint32_t aligned;        // inputs 16-byte aligned: full tiles arrive by TMA
};

// Shared memory (words): a ring of two slots (keys T, then values T for
// pairs), s_goff 256, s_delta 256, s_warp 32, s_cnt NW*257, s_peer
// 2*NW*256.  The tile is permuted in place in its slot; the write-out takes
// each key's digit from the key again.
template <bool PAIRS>
struct OsLayout {
  static constexpr uint32_t T = kOsTile;
  static constexpr uint32_t kSlotWords = T * (PAIRS ? 2 : 1);
  static constexpr uint32_t kGoff = 2 * kSlotWords;
  static constexpr uint32_t kDelta = kGoff + 256;
  static constexpr uint32_t kWarp = kDelta + 256;
  static constexpr uint32_t kCnt = kWarp + 32;
  static constexpr uint32_t kPeer = kCnt + kOsNW * 257;
  static constexpr size_t kBytes = 4u * (size_t)(kPeer + 2 * kOsNW * 256);
};

// One digit pass, persistent: every CTA takes tiles by ticket (so every
// earlier tile belongs to a CTA that already started, and the look-back below
// always ends); once a tile's prefixes are published, the CTA takes its next
// ticket and copies that tile into the other slot while it reorders and
// writes the current one.
template <bool PAIRS, int RANK>
__global__ void __launch_bounds__(kOsNW * 32, PAIRS ? 2 : 3) k_onesweep_pass(OnesweepArgs a) {
  using Lay = OsLayout<PAIRS>;
  constexpr uint32_t T = Lay::T;
  constexpr int THREADS = kOsNW * 32;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tile[2], s_pend[2];
  uint32_t* s_goff = smem + Lay::kGoff;
  uint32_t* s_delta = smem + Lay::kDelta;
  uint32_t* s_warp = smem + Lay::kWarp;
  uint32_t* s_cnt = smem + Lay::kCnt;
  uint32_t* s_peer = smem + Lay::kPeer;
  const DevSpec& sp = a.sp;
  const uint32_t m = sp.m, m_pad = sp.m_pad, S = m_pad + 1;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t L = (uint32_t)(((size_t)a.n + T - 1) / T);

  // thread 0: start the copy of `tile` into `slot` (full tiles of aligned inputs)
  auto issue = [&](uint32_t tile, uint32_t slot) {
    const size_t tbase = (size_t)tile * T;
    if (tile >= L || !a.aligned || tbase + T > a.n) return;
    uint32_t* sk = smem + slot * Lay::kSlotWords;
    mbar_arrive_expect_tx(s_bar + slot, T * 4u * (PAIRS ? 2u : 1u));
    bulk_g2s(sk, a.keys_in + tbase, T * 4u, s_bar + slot);
    if constexpr (PAIRS) bulk_g2s(sk + T, a.vals_in + tbase, T * 4u, s_bar + slot);
    s_pend[slot] = 1u;
  };

  if (threadIdx.x == 0) {
    mbar_init(s_bar, 1);
    mbar_init(s_bar + 1, 1);
    s_pend[0] = s_pend[1] = 0u;
    fence_mbar_init();
    s_tile[0] = atomicAdd(a.ticket, 1u);
    issue(s_tile[0], 0);
  }
  // digit offsets of this pass (first term of Eq. 2): exclusive scan of the histogram
  {
    const uint32_t v = threadIdx.x < m ? a.hist[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<kOsNW>(v, s_warp, &tot);
    if (threadIdx.x < m) s_goff[threadIdx.x] = ex;
  }
  for (uint32_t i = threadIdx.x; i < 2 * kOsNW * m_pad; i += THREADS) s_peer[i] = 0u;
  __syncthreads();

  uint32_t* wc = s_cnt + w * S;
  uint32_t* wpeer = s_peer + w * 2 * m_pad;
  const uint32_t off0 = w * (32 * kOsItems) + lane;
  const uint32_t lane_x[1] = {0u};
  uint32_t phase = 0;  // bit k: parity of slot k's next completion

  for (uint32_t k = 0;; ++k) {
    const uint32_t slot = k & 1u;
    const uint32_t tile = s_tile[slot];
    if (tile >= L) break;
    uint32_t* sk = smem + slot * Lay::kSlotWords;
    uint32_t* sv = sk + T;
    (void)sv;
    const size_t tbase = (size_t)tile * T;
    const uint32_t tile_n = (uint32_t)min((size_t)T, (size_t)a.n - tbase);
    const bool tma = a.aligned && tile_n == T;
    if (a.status_next != nullptr)
      for (uint32_t d = threadIdx.x; d < 256; d += THREADS) a.status_next[(size_t)tile * 256 + d] = 0u;
    bool ok = true;
    if (tma) {
      ok = mbar_wait(s_bar + slot, (phase >> slot) & 1u, a.err);
      if (ok) phase ^= 1u << slot;
    } else {
      for (uint32_t p = threadIdx.x; p < tile_n; p += THREADS) {
        sk[p] = __ldcs(a.keys_in + tbase + p);
        if constexpr (PAIRS) sv[p] = __ldcs(a.vals_in + tbase + p);
      }
      __syncthreads();
    }

    const uint32_t avail = tile_n - min(tile_n, w * (32u * kOsItems));
    uint32_t rb[kOsItems];
    if (tile_n == T)
      rank_windows<kRadix, 8, kOsItems, RANK, true>(sk + off0, avail, sp, nullptr, nullptr, wc, wpeer, m_pad, m,
                                                   lane_x, lanemask_lt(), lane, rb);
    else
      rank_windows<kRadix, 8, kOsItems, RANK, false>(sk + off0, avail, sp, nullptr, nullptr, wc, wpeer, m_pad,
                                                    m, lane_x, lanemask_lt(), lane, rb);
    if (__syncthreads_or(!ok)) {
      // a copy never arrived (the error bit is set): drain the copies in flight, stop
      if (threadIdx.x == 0)
        for (uint32_t q = 0; q < 2; ++q)
          if (s_pend[q] != 0u && !(q == slot && ok)) mbar_drain(s_bar + q, (phase >> q) & 1u);
      __syncthreads();
      return;
    }
    if (threadIdx.x == 0) s_pend[slot] = 0u;
    const uint32_t total = scan_tile_counters<kOsNW>(s_cnt, S, m_pad, s_warp);

    // Decoupled look-back per digit: publish this tile's count, add up the
    // earlier tiles' counts until one carries an inclusive prefix.
    if (threadIdx.x < m) {
      const uint32_t d = threadIdx.x;
      const uint32_t tstart = s_cnt[d];
      const uint32_t hist = ((d + 1 < m_pad) ? s_cnt[d + 1] : total) - tstart;
      uint32_t* st = a.status + (size_t)tile * 256 + d;
      uint32_t excl = 0;
      if (tile == 0) {
        st_relaxed_u32(st, kOsPrefix | hist);
      } else {
        st_relaxed_u32(st, kOsAggregate | hist);
        // Walk back kOsLookback predecessors per step, their status words
        // read at once: hundreds of tiles are in flight, most with only an
        // aggregate published, so a walk spans many tiles (measured on GB300:
        // 8 per step beats 1 and 32).  Before tile 0 counts as an inclusive
        // prefix of 0.
        bool found = false;
        for (int64_t p0 = (int64_t)tile - 1; !found; p0 -= kOsLookback) {
          uint32_t v[kOsLookback];
#pragma unroll
          for (int j = 0; j < kOsLookback; ++j)
            v[j] = (p0 - j >= 0) ? ld_relaxed_u32(a.status + (size_t)(p0 - j) * 256 + d) : kOsPrefix;
#pragma unroll
          for (int j = 0; j < kOsLookback; ++j) {
            if (found) continue;
            const uint32_t* q = a.status + (size_t)(p0 - j) * 256 + d;
            uint32_t spins = 0;
            while ((v[j] & ~kOsValue) == 0u) {
              // give up at the bound, or at once when another wait has already given up
              if (++spins > kSpinLimit || (spins > 64 && (*(volatile uint32_t*)a.err & kDevErrTimeout))) {
                atomicOr(a.err, kDevErrTimeout);
                v[j] = kOsPrefix;
                break;
              }
              __nanosleep(spins < 64 ? 32 : 256);
              v[j] = ld_relaxed_u32(q);
            }
            excl += v[j] & kOsValue;
            if ((v[j] & ~kOsValue) == kOsPrefix) found = true;
          }
        }
        st_relaxed_u32(st, kOsPrefix | ((excl + hist) & kOsValue));
      }
      s_delta[d] = s_goff[d] + excl - tstart;
    }
    if (threadIdx.x == 0) {
      // This tile's prefixes are published: take the next ticket now (a
      // ticket taken earlier would sit unstarted while later tiles wait on
      // it) and start its copy into the other slot, emptied before the last
      // barrier, to overlap the reorder and writes below.
      const uint32_t nx = atomicAdd(a.ticket, 1u);
      s_tile[slot ^ 1u] = nx;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(nx, slot ^ 1u);
    }
    // this thread's keys (and values) into registers before the in-place permutation
    uint32_t kr[kOsItems];
    uint32_t vr[PAIRS ? kOsItems : 1];
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) {
      if (off0 + i * 32 < tile_n) {
        kr[i] = sk[off0 + i * 32];
        if constexpr (PAIRS) vr[i] = sv[off0 + i * 32];
      }
    }
    __syncthreads();
    // reorder the tile by digit in place, then coalesced writes
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) {
      if (off0 + i * 32 < tile_n) {
        const uint32_t b = rb[i] >> 16;
        const uint32_t p = wc[b] + (rb[i] & 0xffffu);
        if (p < T) {
          sk[p] = kr[i];
          if constexpr (PAIRS) sv[p] = vr[i];
        } else {
          atomicOr(a.err, kDevErrBounds);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kOsItems; ++q) {
      const uint32_t p = threadIdx.x + q * THREADS;
      if (p < tile_n) {
        const uint32_t kq = sk[p];
        const uint32_t g = s_delta[(kq >> a.sp.shift) & a.sp.mask] + p;  // the digit again: two instructions
        if (g < a.n) {
          __stcs(a.keys_out + g, kq);
          if constexpr (PAIRS) __stcs(a.vals_out + g, sv[p]);
        } else {
          atomicOr(a.err, kDevErrBounds);
        }
      }
    }
    __syncthreads();  // the slot and s_delta are free again
  }
}

// Whole sort on `stream`: 2 <= passes, n < 2^30.  Scratch from the pool:
// histograms, two status arrays, tickets, one ping-pong buffer per array.
cudaError_t run_onesweep_sort(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t n, int begin_bit, int end_bit,
                              uint32_t* keys_out, uint32_t* vals_out, cudaStream_t s, DeviceCtx& ctx) {
  const bool pairs = vals_in != nullptr;
  const uint32_t passes = (uint32_t)((end_bit - begin_bit + 7) / 8);
  const uint32_t L = (n + kOsTile - 1) / kOsTile;
  const size_t hist_b = 4u * 256u * 4u;
  const size_t status_b = (size_t)L * 256u * 4u;
  const size_t tick_b = 64;
  const size_t buf_b = passes > 1 ? (size_t)n * 4u * (pairs ? 2u : 1u) : 0u;
  const size_t buf_off = (hist_b + 2 * status_b + tick_b + 255) & ~(size_t)255;
  void* ws = nullptr;
  cudaError_t e = scratch_alloc(ctx, &ws, buf_off + buf_b, s);
  if (e != cudaSuccess) return e;
  char* base = static_cast<char*>(ws);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base);
  uint32_t* status[2] = {reinterpret_cast<uint32_t*>(base + hist_b),
                         reinterpret_cast<uint32_t*>(base + hist_b + status_b)};
  uint32_t* tickets = reinterpret_cast<uint32_t*>(base + hist_b + 2 * status_b);
  uint32_t* tmp_k = reinterpret_cast<uint32_t*>(base + buf_off);
  uint32_t* tmp_v = pairs ? tmp_k + n : nullptr;
  e = cudaMemsetAsync(ws, 0, hist_b + 2 * status_b + tick_b, s);

  int occ_keys = 1, occ_pairs = 1;  // CTAs of the pass kernel resident per SM
  {
    // dynamic shared memory opt-in and occupancy, once per device
    static std::mutex mu;
    static uint64_t ready = 0;
    static int g_occ[64][2];
    std::lock_guard<std::mutex> lock(mu);
    const int d = ctx.device & 63;
    if (!((ready >> d) & 1ull)) {
      cudaFuncSetAttribute(k_radix_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, kHistNW * 4 * 256 * 4);
      for (auto k : {k_onesweep_pass<false, kRankTable>, k_onesweep_pass<false, kRankVote>})
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OsLayout<false>::kBytes);
      for (auto k : {k_onesweep_pass<true, kRankTable>, k_onesweep_pass<true, kRankVote>})
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OsLayout<true>::kBytes);
      int v = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_onesweep_pass<false, kRankTable>, kOsNW * 32,
                                                        OsLayout<false>::kBytes) == cudaSuccess && v > 0)
        g_occ[d][0] = v;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_onesweep_pass<true, kRankTable>, kOsNW * 32,
                                                        OsLayout<true>::kBytes) == cudaSuccess && v > 0)
        g_occ[d][1] = v;
      ready |= 1ull << d;
    }
    occ_keys = g_occ[d][0];
    occ_pairs = g_occ[d][1];
  }
  if (e == cudaSuccess) {
    RadixHistArgs ha{keys_in, n, (uint32_t)begin_bit, (uint32_t)end_bit, passes, hist};
    const uint32_t grid = std::min<uint32_t>((n + kHistNW * 32 * kHistItems - 1) / (kHistNW * 32 * kHistItems),
                                             (uint32_t)ctx.sm_count * 4u);
    k_radix_hist<<<std::max(grid, 1u), kHistNW * 32, kHistNW * 4 * 256 * 4, s>>>(ha);
    e = cudaGetLastError();
  }
  const uint32_t aligned = ((reinterpret_cast<uintptr_t>(keys_in) | reinterpret_cast<uintptr_t>(vals_in) |
                             reinterpret_cast<uintptr_t>(keys_out) | reinterpret_cast<uintptr_t>(vals_out) |
                             reinterpret_cast<uintptr_t>(tmp_k) | reinterpret_cast<uintptr_t>(tmp_v)) & 15u) == 0;
  // ranks of the 8-bit digits: peer tables or ballot peers, as the tuning
  // table says for radix-digit multisplits with 256 buckets at this size
  Call probe;
  std::memset(&probe, 0, sizeof probe);
  probe.kind = kRadix;
  probe.sp.nbits = 8;
  probe.n = n;
  probe.vals_in = vals_in;
  const bool vote = choose_variant(probe).rank == kRankVote;
  const uint32_t* src_k = keys_in;
  const uint32_t* src_v = vals_in;
  for (uint32_t p = 0; p < passes && e == cudaSuccess; ++p) {
    const uint32_t shift = (uint32_t)begin_bit + 8 * p;
    const uint32_t bits = std::min(8u, (uint32_t)end_bit - shift);
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    uint32_t* dst_k = to_out ? keys_out : tmp_k;
    uint32_t* dst_v = to_out ? vals_out : tmp_v;
    OnesweepArgs oa;
    std::memset(&oa, 0, sizeof oa);
    oa.keys_in = src_k;
    oa.vals_in = pairs ? src_v : nullptr;
    oa.keys_out = dst_k;
    oa.vals_out = pairs ? dst_v : nullptr;
    oa.n = n;
    oa.sp.m = 1u << bits;
    oa.sp.nbits = bits;
    oa.sp.shift = shift;
    oa.sp.mask = (1u << bits) - 1u;
    oa.sp.m_pad = oa.sp.m <= 32 ? 32u : oa.sp.m;
    oa.hist = hist + p * 256;
    oa.status = status[p & 1];
    oa.status_next = (p + 1 < passes) ? status[(p + 1) & 1] : nullptr;
    oa.ticket = tickets + p;
    oa.err = ctx.d_err;
    oa.aligned = aligned;
    const uint32_t grid = std::max(1u, std::min(L, (uint32_t)ctx.sm_count * (uint32_t)(pairs ? occ_pairs : occ_keys)));
    if (pairs && vote)
      k_onesweep_pass<true, kRankVote><<<grid, kOsNW * 32, OsLayout<true>::kBytes, s>>>(oa);
    else if (pairs)
      k_onesweep_pass<true, kRankTable><<<grid, kOsNW * 32, OsLayout<true>::kBytes, s>>>(oa);
    else if (vote)
      k_onesweep_pass<false, kRankVote><<<grid, kOsNW * 32, OsLayout<false>::kBytes, s>>>(oa);
    else
      k_onesweep_pass<false, kRankTable><<<grid, kOsNW * 32, OsLayout<false>::kBytes, s>>>(oa);
    e = cudaGetLastError();
    src_k = dst_k;
    src_v = dst_v;
  }
  const cudaError_t e2 = scratch_free(ws, s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace ms
