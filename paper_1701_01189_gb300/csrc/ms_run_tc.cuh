// ms_run_tc.cuh -- host launcher of the per-thread-counter multisplit kernels
// (ms_tc.cuh) for m <= 32: one small memset, the pre-scan (whose last CTA
// scans H), and the post-scan launched as a programmatic dependent of the
// pre-scan.
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ms_host.h"
#include "ms_tc.cuh"

namespace ms {

// cuTensorMapEncodeTiled from the driver, looked up once (nullptr if missing:
// the kernels then copy tiles with plain loads).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of a uint32 array seen as rows of 32 words (floor(n / 32) rows),
// box 32 x (tile / 32) (one tile), 128-byte swizzle.  False if it cannot be
// made (then the caller copies tiles with plain loads).
inline bool make_tile_map(CUtensorMap* map, const uint32_t* base, uint32_t n, uint32_t tile) {
  auto enc = tensor_map_encoder();
  if (enc == nullptr || n < tile || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  const cuuint64_t dims[2] = {32, n / 32u};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {32, tile / 32u};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(base), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Launches `kernel` on `s` as a programmatic dependent of the kernel before it
// (it may start while that one drains; it waits with griddepcontrol.wait
// before reading that kernel's results), unless `plain`.
template <typename K, typename... Args>
static cudaError_t launch_dependent(K kernel, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t s,
                                    bool plain, Args... args) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = plain ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Bytes of L2 the pre-scan asks to keep (evict_last) for the post-scan: the
// last tiles of every chunk, about half of the 126 MB L2.
constexpr size_t kTcL2KeepBytes = (size_t)64 << 20;

// The pre-scan of every design: `k_prescan_tc` (ms_tc.cuh) counting in
// registers (m <= 8), per-thread counters (m <= 32) or per-lane byte counters
// (m <= 256), into H (strides hsb, hsc; nullptr: none) and/or the bucket
// totals `tot`.  Chunks are whole 4096-key tiles.
template <int KIND>
static cudaError_t launch_prescan(const Call& c, DeviceCtx& ctx, const Chunking& ch, uint32_t* H, uint32_t hsb,
                                  uint32_t hsc, uint32_t* tot) {
  const uint32_t m = c.sp.m;
  const int mode = m <= 8 ? kCountReg : m <= 32 ? kCountThread : kCountLaneBytes;
  // splitter lookup tables: 1024 cells x 8 copies (m <= 32), 4096 cells x 1 copy beyond
  // (with random cells two copies barely thin the bank conflicts; twice the
  // cells halve the flagged ones)
  const uint32_t lb = mode == kCountLaneBytes ? 12u : 10u, lw = mode == kCountLaneBytes ? 0u : 3u;
  const bool vec = ((reinterpret_cast<uintptr_t>(c.keys_in)) & 15u) == 0;
  const size_t keep_tiles = kTcL2KeepBytes / ((size_t)kTcTile * 4);
  const uint32_t keep = (uint32_t)std::min<size_t>(ch.K, (keep_tiles + ch.G - 1) / ch.G);
  TcPreArgs pa{c.keys_in, c.n, ch.K, ch.L, ch.G, ch.K - keep, vec ? 1u : 0u, H, hsb, hsc, tot, lb, lw, c.sp};
  static LaunchInfo li[3];
  // one CTA per chunk; or, when the chunks outnumber the CTAs the SMs hold at
  // once, or number at most half of them (a post-scan of one CTA per SM),
  // one wave of those CTAs, each an equal run of tiles whose pieces add into
  // their chunks' columns of H (measured on GB300: key-value multisplits of
  // 2^26 elements with 256 buckets had their pre-scan at one CTA per SM,
  // 26-47% slower than for the same keys alone)
  auto launch = [&](auto k, size_t smem, size_t smem_max, LaunchInfo& info) {
    const int resident = setup_kernel(info, k, kTcThreads, smem_max, smem, ctx.device);
    const uint32_t cap = (uint32_t)(ctx.sm_count * resident);
    uint32_t grid = std::min(ch.G, cap);
    if (2u * ch.G <= cap) grid = std::min(cap, ch.L);
    k<<<std::max(1u, grid), kTcThreads, smem, c.stream>>>(pa);
  };
  if (mode == kCountLaneBytes)
    launch(k_prescan_tc<KIND, kCountLaneBytes>, tc_prescan_smem<KIND, kCountLaneBytes>(m, lb, lw),
           tc_prescan_smem<KIND, kCountLaneBytes>(kMaxM, lb, lw), li[2]);
  else if (mode == kCountThread)
    launch(k_prescan_tc<KIND, kCountThread>, tc_prescan_smem<KIND, kCountThread>(m, lb, lw),
           tc_prescan_smem<KIND, kCountThread>(kTcMaxM, lb, lw), li[0]);
  else
    launch(k_prescan_tc<KIND, kCountReg>, tc_prescan_smem<KIND, kCountReg>(m, lb, lw),
           tc_prescan_smem<KIND, kCountReg>(kTcMaxM, lb, lw), li[1]);
  return cudaGetLastError();
}

template <int KIND, bool PAIRS, int STAGES, int KPT, bool BULK>
static cudaError_t run_tc_cfg(const Call& c, DeviceCtx& ctx) {
  constexpr uint32_t T = kTcThreads * KPT;  // post-scan tile; the pre-scan works in 4096-key tiles
  auto kpost = k_postscan_tc<KIND, PAIRS, STAGES, KPT, BULK>;
  using Lay = TcPostLayout<KIND, PAIRS, STAGES, KPT, BULK>;
  const DevSpec& sp = c.sp;
  // splitter lookup table of the post-scan: 512 cells x 4 copies (x 2 for
  // key-value pairs with more than 16 buckets, which keeps two CTAs per SM)
  const uint32_t post_lb = 9, post_lw = (PAIRS && sp.m > 16) ? 1u : 2u;
  const size_t smem_post = Lay::bytes(sp.m, post_lb, post_lw);
  static LaunchInfo li_post;
  const int nb_post = setup_kernel(li_post, kpost, kTcThreads, Lay::bytes(kTcMaxM, post_lb, 2), smem_post, ctx.device);

  // chunks are whole 4096-key pre-scan tiles; the post-scan walks them in its own tiles
  const Chunking ch = make_chunking(c.n, kTcTile, (uint32_t)(ctx.sm_count * nb_post));
  const uint32_t post_k = ch.K * (kTcTile / T);
  const uint32_t post_l = (uint32_t)(((uint64_t)c.n + T - 1) / T);
  const uint32_t m = sp.m;
  // scratch: H (chunk-major, rows of tc_rows(m) words; the pre-scan adds into it)
  const size_t h_bytes = ((size_t)tc_rows(m) * ch.G * 4 + 15) & ~(size_t)15;
  const size_t bytes = h_bytes;
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
  e = cudaMemsetAsync(ws, 0, h_bytes, c.stream);

  CUtensorMap tmk, tmv;
  std::memset(&tmk, 0, sizeof tmk);
  std::memset(&tmv, 0, sizeof tmv);
  bool tma = make_tile_map(&tmk, c.keys_in, c.n, T);
  if (tma && PAIRS) tma = make_tile_map(&tmv, c.vals_in, c.n, T);

  const int slot = c.ws_fixed != nullptr ? -1 : trace_begin(c.stream);
  if (e == cudaSuccess) {
    e = launch_prescan<KIND>(c, ctx, ch, H, 1u, tc_rows(m), nullptr);
    trace_mark(slot, 1, c.stream);
    trace_mark(slot, 2, c.stream);  // the global scan is folded into the post-scan's set-up
  }
  if (e == cudaSuccess) {
    TcPostArgs qa{c.keys_in, c.vals_in, c.keys_out, c.vals_out, c.n, post_k, post_l, ch.G, H, c.offsets, ctx.d_err,
                  tma ? 1u : 0u, post_lb, post_lw, sp};
    // stage timing records events between the kernels: then a plain launch
    e = launch_dependent(kpost, ch.G, kTcThreads, smem_post, c.stream, slot >= 0, tmk, tmv, qa);
    trace_mark(slot, 3, c.stream);
  }
  const cudaError_t e2 = c.ws_fixed != nullptr ? cudaSuccess : scratch_free(ws, c.stream);
  return e != cudaSuccess ? e : e2;
}

// Device histogram (Section 7.3): the pre-scan alone, its CTAs adding their
// counts into c.counts (zeroed first).  Any m <= 256.
template <int KIND>
static cudaError_t run_histogram(const Call& c, DeviceCtx& ctx) {
  const Chunking ch = make_chunking(c.n, kTcTile, (uint32_t)(ctx.sm_count * 3));
  cudaError_t e = cudaMemsetAsync(c.counts, 0, (size_t)c.sp.m * 4, c.stream);
  const int slot = trace_begin(c.stream);
  if (e == cudaSuccess) e = launch_prescan<KIND>(c, ctx, ch, nullptr, 0u, 0u, c.counts);
  trace_mark(slot, 1, c.stream);
  trace_mark(slot, 2, c.stream);
  trace_mark(slot, 3, c.stream);
  return e;
}

// Variant shape 2 selects 8 keys per thread, any other 16; shape 1 a
// 3-slot ring for keys only (key-value pairs keep 2 slots).  Up to
// kTcBulkMaxM buckets the write-out goes by bulk copies per bucket run.
template <int KIND, bool BULK>
static cudaError_t run_tc_bulk(const Call& c, DeviceCtx& ctx, int shape) {
  if (shape == 2) {
    if (c.vals_in != nullptr) return run_tc_cfg<KIND, true, 2, 8, BULK>(c, ctx);
    return run_tc_cfg<KIND, false, 2, 8, BULK>(c, ctx);
  }
  if (c.vals_in != nullptr) return run_tc_cfg<KIND, true, 2, 16, BULK>(c, ctx);
  if (shape == 1) return run_tc_cfg<KIND, false, 3, 16, BULK>(c, ctx);
  return run_tc_cfg<KIND, false, 2, 16, BULK>(c, ctx);
}

template <int KIND>
static cudaError_t run_tc(const Call& c, DeviceCtx& ctx, int shape) {
  if (c.sp.m <= kTcBulkMaxM) return run_tc_bulk<KIND, true>(c, ctx, shape);
  return run_tc_bulk<KIND, false>(c, ctx, shape);
}

}  // namespace ms
