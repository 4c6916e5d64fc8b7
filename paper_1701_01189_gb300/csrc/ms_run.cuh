// ms_run.cuh -- host launcher of the three multisplit stages for one bucket
// kind; included once per kind by ms_kind_<kind>.cu so the kinds compile in
// parallel.
#pragma once

#include <algorithm>
#include <map>
#include <mutex>

#include "ms_host.h"
#include "ms_kernels.cuh"
#include "ms_scan.cuh"

namespace ms {

// Per-device, per-instantiation launch set-up: the dynamic shared memory
// opt-in (once, for the largest size the instantiation can use) and the
// number of CTAs resident per SM for each shared-memory size seen.
struct LaunchInfo {
  std::mutex mu;
  uint64_t ready = 0;  // bit d: opt-in done on device d
  std::map<std::pair<int, size_t>, int> resident;
};

template <typename K>
static int setup_kernel(LaunchInfo& li, K kernel, int threads, size_t smem_max, size_t smem, int device) {
  std::lock_guard<std::mutex> lock(li.mu);
  const int d = device & 63;
  if (!((li.ready >> d) & 1ull)) {
    if (smem_max > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    // these kernels read through TMA or no-allocate loads: give the SM's
    // L1/shared storage to shared memory, so occupancy is not capped by the carveout
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    li.ready |= 1ull << d;
  }
  auto key = std::make_pair(d, smem);
  auto it = li.resident.find(key);
  if (it != li.resident.end()) return it->second;
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem) != cudaSuccess || v < 1) v = 1;
  li.resident[key] = v;
  return v;
}

// Chunking of L tiles over at most `max_ctas` CTAs: K tiles per chunk, G chunks.
struct Chunking {
  uint32_t L, K, G;
};
static inline Chunking make_chunking(uint32_t n, uint32_t T, uint32_t max_ctas) {
  Chunking ch;
  ch.L = (uint32_t)(((uint64_t)n + T - 1) / T);
  const uint32_t g0 = std::max(1u, std::min(ch.L, max_ctas));
  ch.K = (ch.L + g0 - 1) / g0;
  ch.G = (ch.L + ch.K - 1) / ch.K;
  return ch;
}

}  // namespace ms

#include "ms_run_tc.cuh"

namespace ms {

template <int KIND, int NB, int NW, int ITEMS, bool PAIRS, int RANK, int REORDER, int MINB, int STAGES = 2>
static cudaError_t run_ms_cfg(const Call& c, DeviceCtx& ctx) {
  constexpr int THREADS = NW * 32;
  constexpr uint32_t T = THREADS * ITEMS;
  static_assert(kTcTile % T == 0, "post-scan tiles divide the pre-scan's");
  auto kpost = k_postscan<KIND, NB, NW, ITEMS, PAIRS, RANK, REORDER, MINB, STAGES>;
  const uint32_t m_pad = c.sp.m_pad, lb = c.sp.lut_bits;
  const uint32_t mp_max = RANK == kRankBallot ? 32u : 256u;  // peer tables and vote counters: any m
  const size_t smem_post_max = postscan_smem_bytes<KIND, NW, ITEMS, PAIRS, RANK, REORDER, STAGES>(mp_max, 11);
  const size_t smem_post = postscan_smem_bytes<KIND, NW, ITEMS, PAIRS, RANK, REORDER, STAGES>(m_pad, lb);
  static LaunchInfo li_post;
  const int nb_post = setup_kernel(li_post, kpost, THREADS, smem_post_max, smem_post, ctx.device);

  // One chunk per CTA in both kernels: whole 4096-key pre-scan tiles, walked
  // by the post-scan in its own tiles.
  const Chunking ch = make_chunking(c.n, kTcTile, (uint32_t)(ctx.sm_count * nb_post));
  const uint32_t post_k = ch.K * (kTcTile / T);
  const uint32_t post_l = (uint32_t)(((uint64_t)c.n + T - 1) / T);
  const uint32_t m = c.sp.m;
  // Up to 32 buckets every post-scan CTA reads the chunk-major H whole and
  // reduces its own offsets; beyond, H is longer and the look-back scan turns
  // the bucket-major H into the offsets in parallel tiles.
  const bool small = m <= kTcMaxM;
  const uint32_t len = (small ? tc_rows(m) : m) * ch.G;  // small: chunk-major rows of tc_rows(m) words
  const uint32_t nscan = small ? 0u : (len + kScanTile - 1) / kScanTile;

  // scratch: H (m * G words, 16-byte aligned) | scan status (nscan u64) | ticket
  const size_t h_bytes = ((size_t)len * 4 + 15) & ~(size_t)15;
  const size_t st_bytes = (size_t)nscan * 8;
  const size_t bytes = h_bytes + st_bytes + 16;
  void* ws = nullptr;
  cudaError_t e = cudaSuccess;
  if (c.ws_fixed != nullptr) {
    if (bytes > c.ws_capacity) return cudaErrorMemoryAllocation;
    ws = c.ws_fixed;
  } else {
    e = scratch_alloc(ctx, &ws, bytes, c.stream);
    if (e != cudaSuccess) return e;
  }
  uint32_t* H = static_cast<uint32_t*>(ws);
  auto* status = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + h_bytes);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + h_bytes + st_bytes);
  e = cudaMemsetAsync(ws, 0, h_bytes + st_bytes + 16, c.stream);  // H (the pre-scan adds into it), status, ticket

  const uint32_t aligned =
      ((reinterpret_cast<uintptr_t>(c.keys_in) | reinterpret_cast<uintptr_t>(c.vals_in)) & 15u) == 0;
  const int slot = c.ws_fixed != nullptr ? -1 : trace_begin(c.stream);
  if (e == cudaSuccess) {
    e = launch_prescan<KIND>(c, ctx, ch, H, small ? 1u : ch.G, small ? tc_rows(m) : 1u, nullptr);
    trace_mark(slot, 1, c.stream);
  }
  if (e == cudaSuccess && !small) {
    ScanArgs sa{H, len, ch.G, c.offsets, m, status, ticket, ctx.d_err};
    e = launch_scan_lookback(sa, c.stream);
  }
  trace_mark(slot, 2, c.stream);
  if (e == cudaSuccess) {
    PostscanArgs qa{c.keys_in, c.vals_in, c.keys_out, c.vals_out, c.n, c.sp, post_k, post_l, ch.G, H,
                    small ? c.offsets : nullptr, ctx.d_err, aligned, 1u};
    // stage timing records events between the kernels: then a plain launch
    e = launch_dependent(kpost, ch.G, THREADS, smem_post, c.stream, slot >= 0, qa);
    trace_mark(slot, 3, c.stream);
  }
  const cudaError_t e2 = c.ws_fixed != nullptr ? cudaSuccess : scratch_free(ws, c.stream);
  return e != cudaSuccess ? e : e2;
}

// Tile shapes of the post-scan the tuner chooses from (warps x keys per lane):
// 0: 8 x 16 (4096 keys), 1: 16 x 8 (4096 keys), 2: 8 x 8 (2048 keys).
template <int KIND, int NB, bool PAIRS, int RANK, int REORDER>
static cudaError_t run_ms_shape(const Call& c, DeviceCtx& ctx, int shape) {
  switch (shape) {
    case 1: return run_ms_cfg<KIND, NB, 16, 8, PAIRS, RANK, REORDER, PAIRS ? 1 : 2>(c, ctx);
    case 2: return run_ms_cfg<KIND, NB, 8, 8, PAIRS, RANK, REORDER, PAIRS ? 3 : 4>(c, ctx);
    default: return run_ms_cfg<KIND, NB, 8, 16, PAIRS, RANK, REORDER, PAIRS ? 2 : 3>(c, ctx);
  }
}

template <int KIND, int NB, int RANK, int REORDER>
static cudaError_t run_ms_pairs(const Call& c, DeviceCtx& ctx, int shape) {
  if (c.vals_in != nullptr) return run_ms_shape<KIND, NB, true, RANK, REORDER>(c, ctx, shape);
  return run_ms_shape<KIND, NB, false, RANK, REORDER>(c, ctx, shape);
}

template <int KIND, int NB>
static cudaError_t run_ms_ballot(const Call& c, DeviceCtx& ctx, const Variant& v) {
  if (v.reorder || NB > 3) return run_ms_pairs<KIND, NB, kRankBallot, 1>(c, ctx, v.shape);
  return run_ms_pairs<KIND, (NB > 3 ? 3 : NB), kRankBallot, 0>(c, ctx, v.shape);
}

// Ballot ranks are built for m <= 32 (NB <= 5; direct writes only for m <= 8);
// every m runs with peer tables (NB = 8 sizes the range-splitter search for
// any m).
template <int KIND>
static cudaError_t run_ms_kind(const Call& c, DeviceCtx& ctx) {
  if (c.counts != nullptr) return run_histogram<KIND>(c, ctx);
  const Variant v = choose_variant(c);
  if (v.rank == kRankThread && c.sp.m <= kTcMaxM) return run_tc<KIND>(c, ctx, v.shape);
  if (v.rank == kRankVote) return run_ms_pairs<KIND, 8, kRankVote, 1>(c, ctx, v.shape);
  if (v.rank == kRankBallot && c.sp.nbits <= 5) {
    switch (c.sp.nbits) {
      case 0: return run_ms_ballot<KIND, 0>(c, ctx, v);
      case 1: return run_ms_ballot<KIND, 1>(c, ctx, v);
      case 2: return run_ms_ballot<KIND, 2>(c, ctx, v);
      case 3: return run_ms_ballot<KIND, 3>(c, ctx, v);
      case 4: return run_ms_ballot<KIND, 4>(c, ctx, v);
      default: return run_ms_ballot<KIND, 5>(c, ctx, v);
    }
  }
  return run_ms_pairs<KIND, 8, kRankTable, 1>(c, ctx, v.shape);
}

}  // namespace ms
