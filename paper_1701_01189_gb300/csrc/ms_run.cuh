// ms_run.cuh -- host launcher of the three multisplit stages for one bucket
// kind; included once per kind by ms_kind_<kind>.cu so the kinds compile in
// parallel.
#pragma once

#include <algorithm>
#include <mutex>

#include "ms_host.h"
#include "ms_kernels.cuh"
#include "ms_scan.cuh"

namespace ms {

// Per-device, per-instantiation launch set-up: the dynamic shared memory
// opt-in and the number of CTAs resident per SM.
struct LaunchInfo {
  std::mutex mu;
  uint64_t ready = 0;  // bit d: set up on device d
  int resident[64] = {};
};

template <typename K>
static int setup_kernel(LaunchInfo& li, K kernel, int threads, size_t smem, int device) {
  std::lock_guard<std::mutex> lock(li.mu);
  const int d = device & 63;
  if (!((li.ready >> d) & 1ull)) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem) != cudaSuccess || v < 1) v = 1;
    li.resident[d] = v;
    li.ready |= 1ull << d;
  }
  return li.resident[d];
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

template <int KIND, int NW, int ITEMS, bool SMALLM, bool PAIRS>
static cudaError_t run_ms_cfg(const Call& c, DeviceCtx& ctx) {
  constexpr int THREADS = NW * 32;
  constexpr uint32_t T = THREADS * ITEMS;
  static_assert(NW >= 8, "the per-bucket block phase needs >= 256 threads");
  auto kpre = k_prescan<KIND, NW, ITEMS, SMALLM>;
  auto kpost = k_postscan<KIND, NW, ITEMS, SMALLM, PAIRS>;
  const size_t smem_pre = prescan_smem_bytes<NW, SMALLM>();
  const size_t smem_post = postscan_smem_bytes<NW, ITEMS, SMALLM, PAIRS>();
  static LaunchInfo li_pre, li_post;
  const int nb_post = setup_kernel(li_post, kpost, THREADS, smem_post, ctx.device);
  setup_kernel(li_pre, kpre, THREADS, smem_pre, ctx.device);

  const Chunking ch = make_chunking(c.n, T, (uint32_t)(ctx.sm_count * nb_post));
  const uint32_t m = c.sp.m;
  const uint32_t len = m * ch.G;
  const uint32_t nscan = (len + kScanTile - 1) / kScanTile;

  // scratch: H (len words, 16-byte aligned) | scan status (nscan u64) | ticket
  const size_t h_bytes = ((size_t)len * 4 + 15) & ~(size_t)15;
  const size_t st_bytes = (size_t)nscan * 8;
  const size_t bytes = h_bytes + st_bytes + 16;
  void* ws = nullptr;
  cudaError_t e = scratch_alloc(ctx, &ws, bytes, c.stream);
  if (e != cudaSuccess) return e;
  uint32_t* H = static_cast<uint32_t*>(ws);
  auto* status = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + h_bytes);
  auto* ticket = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + h_bytes + st_bytes);
  e = cudaMemsetAsync(status, 0, st_bytes + 16, c.stream);

  const int slot = trace_begin(c.stream);
  if (e == cudaSuccess) {
    PrescanArgs pa{c.keys_in, c.n, c.sp, ch.K, ch.L, ch.G, H};
    kpre<<<ch.G, THREADS, smem_pre, c.stream>>>(pa);
    e = cudaGetLastError();
    trace_mark(slot, 1, c.stream);
  }
  if (e == cudaSuccess) {
    ScanArgs sa{H, len, ch.G, c.offsets, m, status, ticket, ctx.d_err};
    e = launch_scan_lookback(sa, c.stream);
    trace_mark(slot, 2, c.stream);
  }
  if (e == cudaSuccess) {
    PostscanArgs qa{c.keys_in, c.vals_in, c.keys_out, c.vals_out, c.n, c.sp, ch.K, ch.L, ch.G, H, ctx.d_err};
    kpost<<<ch.G, THREADS, smem_post, c.stream>>>(qa);
    e = cudaGetLastError();
    trace_mark(slot, 3, c.stream);
  }
  const cudaError_t e2 = scratch_free(ws, c.stream);
  return e != cudaSuccess ? e : e2;
}

template <int KIND>
static cudaError_t run_ms_kind(const Call& c, DeviceCtx& ctx) {
  const bool pairs = c.vals_in != nullptr;
  const bool smallm = c.sp.m <= 32;
  if (smallm) {
    return pairs ? run_ms_cfg<KIND, 16, 8, true, true>(c, ctx) : run_ms_cfg<KIND, 16, 8, true, false>(c, ctx);
  }
  return pairs ? run_ms_cfg<KIND, 16, 8, false, true>(c, ctx) : run_ms_cfg<KIND, 16, 8, false, false>(c, ctx);
}

}  // namespace ms
