// ms_batch.cu -- many independent multisplits in one persistent launch.
//
// Not in the paper (which sizes one problem per launch); this is the batching
// form of the same method for many small and uneven arrays, where launching
// the three stages once per array is dominated by launch latency (cf. the
// small-frontier overhead the paper notes for SSSP, Section 7.2).
//
// A plan flattens every segment into a list of work items, each a run of up
// to K consecutive 4096-key tiles of one segment (a chunk; K = 1 for the
// peer-table kernel, kBatchChunkTiles for the per-thread-counter kernel), of
// two kinds: (A) the histogram of each chunk of every segment that spans more
// than one tile, and (B) the post-scan of every chunk of every segment, where
// a segment of a single tile is done in one item from start to finish (its
// own tile histogram is the whole H, so no global scan is needed).  The list
// holds the histogram items first, then the post-scan items (build_work).
// CTAs of one persistent grid take
// items in ticket order.  The CTA that finishes the last histogram of a
// segment scans that segment's histogram matrix (bucket-major, one column per
// chunk: Eq. 2 with the segment's chunks as subproblems) and raises the
// segment's ready flag; post-scan items of the segment wait for that flag
// (bounded).  Every item a post-scan item waits for has an earlier ticket and
// never waits itself, so the waits always end (the argument is at
// build_work).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "ms.h"
#include "ms_host.h"
#include "ms_kernels.cuh"
#include "ms_scan.cuh"

struct ms_batch_plan;  // defined below (outside the namespace, as declared in ms.h)

namespace ms {

constexpr int kBatchNW = 8, kBatchItems = 16;
constexpr uint32_t kBatchTile = kBatchNW * 32 * kBatchItems;  // 4096
// tiles per work item of the per-thread-counter kernel: a post-scan item
// pays its ready-flag wait and descriptor loads, and a histogram item its
// fence, done-counter atomic and H write, once per chunk instead of per tile
constexpr uint32_t kBatchChunkTiles = 8;
// bit of an item's second word that marks a post-scan item (the rest is the
// item's first tile)
constexpr uint32_t kBatchPost = 1u << 31;

struct DevSeg {
  const uint32_t* kin;
  const uint32_t* vin;
  uint32_t* kout;
  uint32_t* vout;
  uint32_t* offsets;  // m+1 words or nullptr
  uint32_t n;
  uint32_t L;         // tiles
  uint32_t hoff;      // first word of the segment's H in the plan's pool (multi-tile only)
  uint32_t C;         // chunks of K tiles: the columns of the segment's H (m x C words)
};

struct BatchArgs {
  const DevSeg* segs;
  const uint2* items;    // items[0] = (n_hist, n_items); then (segment, first tile | kBatchPost for a post-scan)
  uint32_t* H;           // histogram pool
  uint32_t* done;        // per segment: histogram items finished (zeroed per run)
  uint32_t* ready;       // per segment: scan finished (zeroed per run)
  uint32_t* ticket;      // zeroed per run
  uint32_t* err;
  uint32_t K;            // tiles per item (the last item of a segment may hold fewer)
  DevSpec sp;
};

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Shared memory (words): splitter table 256, LUT, s_base 256, s_delta 256,
// s_warp 32, counters NW*257, peer tables 2*NW*256, tile keys T, tile values T
// (pairs), reorder keys T, values T (pairs), bucket bytes T.
template <int KIND, bool PAIRS, int NW>
struct BatchLayout {
  static constexpr uint32_t T = kBatchTile;
  static __host__ __device__ uint32_t lut() { return 256; }
  static __host__ __device__ uint32_t base(uint32_t lb) { return lut() + lut_words<KIND>(lb); }
  static __host__ __device__ uint32_t cnt(uint32_t lb) { return base(lb) + 256 + 256 + 32; }
  static __host__ __device__ uint32_t peer(uint32_t lb) { return cnt(lb) + NW * 257; }
  static __host__ __device__ uint32_t tile(uint32_t lb) { return (peer(lb) + 2 * NW * 256 + 3) & ~3u; }
  static __host__ __device__ uint32_t reorder(uint32_t lb) { return tile(lb) + T * (PAIRS ? 2 : 1); }
  static __host__ size_t bytes(uint32_t lb) { return 4u * (size_t)(reorder(lb) + T * (PAIRS ? 2 : 1)) + T; }
};

// NW warps of ITEMS windows each (NW * 32 * ITEMS = 4096 keys a tile); ranks
// by per-warp peer tables (RANK = kRankTable) or by ballot peers with
// per-warp counters (kRankVote).
template <int KIND, bool PAIRS, int NW, int ITEMS, int RANK>
__global__ void __launch_bounds__(NW * 32, (PAIRS ? 2 : 3) * 8 / NW) k_batch(BatchArgs a) {
  static_assert(NW * 32 * ITEMS == (int)kBatchTile, "a tile is 4096 keys");
  using Lay = BatchLayout<KIND, PAIRS, NW>;
  constexpr uint32_t T = Lay::T;
  constexpr int THREADS = NW * 32;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_item, s_flag;
  const DevSpec& sp = a.sp;
  const uint32_t m = sp.m, m_pad = sp.m_pad, S = m_pad + 1, lb = sp.lut_bits;
  uint32_t* s_tbl = smem;
  uint32_t* s_lut = smem + Lay::lut();
  uint32_t* s_base = smem + Lay::base(lb);
  uint32_t* s_delta = s_base + 256;
  uint32_t* s_warp = s_delta + 256;
  uint32_t* s_cnt = smem + Lay::cnt(lb);
  uint32_t* s_peer = smem + Lay::peer(lb);
  uint32_t* t_keys = smem + Lay::tile(lb);
  uint32_t* t_vals = t_keys + T;
  uint32_t* s_keys = smem + Lay::reorder(lb);
  uint32_t* s_vals = s_keys + T;
  uint8_t* s_bkt = reinterpret_cast<uint8_t*>(s_keys + T * (PAIRS ? 2 : 1));
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t* wc = s_cnt + w * S;
  uint32_t* wpeer = s_peer + w * 2 * m_pad;
  const uint32_t off0 = w * (32 * ITEMS) + lane;
  const uint32_t lane_x[1] = {0u};

  for (uint32_t i = threadIdx.x; i < 2 * NW * m_pad; i += THREADS) s_peer[i] = 0u;
  build_bucket_tables<KIND, 8>(sp, s_tbl, s_lut);  // ends with a barrier
  const uint2 counts = a.items[0];  // read from memory so a captured graph follows later updates
  const uint32_t n_items = counts.y;

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= n_items) break;
    const uint2 item = a.items[1 + it];
    const DevSeg sg = a.segs[item.x];
    const uint32_t tile = item.y & ~kBatchPost;
    const bool post = (item.y & kBatchPost) != 0u;
    const size_t tbase = (size_t)tile * T;
    const uint32_t tile_n = (uint32_t)min((size_t)T, (size_t)sg.n - tbase);

    // the tile's keys (and values) into shared memory
    for (uint32_t p = threadIdx.x; p < tile_n; p += THREADS) {
      t_keys[p] = __ldcs(sg.kin + tbase + p);
      if constexpr (PAIRS)
        if (post) t_vals[p] = __ldcs(sg.vin + tbase + p);
    }
    __syncthreads();
    const uint32_t avail = tile_n - min(tile_n, w * (32u * ITEMS));
    uint32_t rb[ITEMS];
    if (tile_n == T)
      rank_windows<KIND, 8, ITEMS, RANK, true>(t_keys + off0, avail, sp, s_tbl, s_lut, wc, wpeer, m_pad,
                                                          m, lane_x, lanemask_lt(), lane, rb);
    else
      rank_windows<KIND, 8, ITEMS, RANK, false>(t_keys + off0, avail, sp, s_tbl, s_lut, wc, wpeer,
                                                           m_pad, m, lane_x, lanemask_lt(), lane, rb);
    __syncthreads();
    const uint32_t total = scan_tile_counters<NW>(s_cnt, S, m_pad, s_warp);

    if (!post) {
      // (A) tile histogram -> column `tile` of the segment's H
      if (threadIdx.x < m) {
        const uint32_t b = threadIdx.x;
        const uint32_t hist = ((b + 1 < m_pad) ? s_cnt[b + 1] : total) - s_cnt[b];
        a.H[sg.hoff + b * sg.C + tile] = hist;
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_flag = (atomicAdd(a.done + item.x, 1u) == sg.C - 1) ? 1u : 0u;
      __syncthreads();
      if (s_flag) {
        // last histogram of the segment: exclusive scan of its H (m*L words,
        // bucket-major), bucket offsets, then the ready flag
        __threadfence();
        const uint32_t len = m * sg.C;
        uint32_t* Hs = a.H + sg.hoff;
        uint32_t carry = 0;
        for (uint32_t base = 0; base < len; base += THREADS) {
          const uint32_t e = base + threadIdx.x;
          const uint32_t v = e < len ? __ldcg(Hs + e) : 0u;
          uint32_t tot;
          const uint32_t ex = block_exclusive_scan<NW>(v, s_warp, &tot);
          if (e < len) {
            Hs[e] = carry + ex;
            if (sg.offsets != nullptr && e % sg.C == 0u) sg.offsets[e / sg.C] = carry + ex;
          }
          carry += tot;
        }
        if (sg.offsets != nullptr && threadIdx.x == 0) sg.offsets[m] = carry;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release_u32(a.ready + item.x, 1u);
      }
      __syncthreads();
      continue;
    }

    // (B) post-scan of one tile: global base of each bucket for this tile
    if (sg.L == 1) {
      if (threadIdx.x < m) s_base[threadIdx.x] = s_cnt[threadIdx.x];  // the tile is the segment
      if (sg.offsets != nullptr) {
        if (threadIdx.x < m) sg.offsets[threadIdx.x] = s_cnt[threadIdx.x];
        if (threadIdx.x == 0) sg.offsets[m] = total;
      }
    } else {
      if (threadIdx.x == 0) {
        uint32_t spins = 0;
        while (ld_acquire_u32(a.ready + item.x) == 0u) {
          // give up at the bound, or at once when another wait has already given up
          if (++spins > kSpinLimit || (spins > 64 && (*(volatile uint32_t*)a.err & kDevErrTimeout))) {
            atomicOr(a.err, kDevErrTimeout);
            break;
          }
          __nanosleep(spins < 64 ? 64 : 512);
        }
      }
      __syncthreads();
      if (threadIdx.x < m) s_base[threadIdx.x] = __ldcg(a.H + sg.hoff + threadIdx.x * sg.C + tile);
    }
    if (threadIdx.x < m) s_delta[threadIdx.x] = s_base[threadIdx.x] - s_cnt[threadIdx.x];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (off0 + i * 32 < tile_n) {
        const uint32_t b = rb[i] >> 16;
        const uint32_t p = wc[b] + (rb[i] & 0xffffu);
        if (p < T) {
          s_keys[p] = t_keys[off0 + i * 32];
          if constexpr (PAIRS) s_vals[p] = t_vals[off0 + i * 32];
          s_bkt[p] = (uint8_t)b;
        } else {
          atomicOr(a.err, kDevErrBounds);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t p = threadIdx.x + k * THREADS;
      if (p < tile_n) {
        const uint32_t g = s_delta[s_bkt[p]] + p;
        if (g < sg.n) {
          __stcs(sg.kout + g, s_keys[p]);
          if constexpr (PAIRS) __stcs(sg.vout + g, s_vals[p]);
        } else {
          atomicOr(a.err, kDevErrBounds);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace ms

#include "ms_batch_tc.cuh"

using namespace ms;

struct ms_batch_plan {
  int device = -1;
  int kind = 0;
  bool pairs = false;
  DevSpec sp;
  // capacities (fixed at creation) and the current work
  uint32_t max_segments = 0, max_items = 0;
  uint64_t max_hwords = 0;
  uint32_t num_segments = 0, n_items = 0;
  uint32_t grid = 0;
  size_t smem = 0;
  uint32_t lb = 0, lw = 0;  // m <= 32: splitter lookup table of k_batch_tc
  int shape = 0, rank = 0;  // the kernel (from the batched variant table, see choose_batch_variant)
  uint32_t K = 1;           // tiles per work item
  DevSeg* d_segs = nullptr;
  uint2* d_items = nullptr;  // [0] = (n_hist, n_items), then the items
  uint32_t* d_H = nullptr;
  uint32_t* d_flags = nullptr;  // done[max_segments] | ready[max_segments] | ticket
  size_t flags_bytes = 0;
  uint32_t* d_err = nullptr;
  cudaGraphExec_t graph = nullptr;
  // dynamic plans: two pinned staging areas for segment tables and items
  void* h_stage[2] = {nullptr, nullptr};
  cudaEvent_t stage_done[2] = {nullptr, nullptr};
  int stage_next = 0;
};

namespace ms {

template <typename K>
static cudaError_t batch_occupancy(ms_batch_plan& p, K k, int threads, int sm_count) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, p.smem);
  if (e != cudaSuccess) return e;
  p.grid = (uint32_t)std::max(1, nb) * (uint32_t)sm_count;
  return cudaSuccess;
}

template <int KIND, bool PAIRS>
static cudaError_t batch_setup(ms_batch_plan& p, int sm_count) {
  if (p.rank == kRankThread) {
    p.lb = 9;
    p.lw = (PAIRS && p.sp.m > 16) ? 1u : 2u;
    p.smem = BatchTcLayout<KIND, PAIRS>::bytes(p.sp.m, p.lb, p.lw);
    return batch_occupancy(p, k_batch_tc<KIND, PAIRS>, kTcThreads, sm_count);
  }
  if (p.shape == 1) {
    p.smem = BatchLayout<KIND, PAIRS, 16>::bytes(p.sp.lut_bits);
    if (p.rank == kRankVote) return batch_occupancy(p, k_batch<KIND, PAIRS, 16, 8, kRankVote>, 512, sm_count);
    return batch_occupancy(p, k_batch<KIND, PAIRS, 16, 8, kRankTable>, 512, sm_count);
  }
  p.smem = BatchLayout<KIND, PAIRS, 8>::bytes(p.sp.lut_bits);
  if (p.rank == kRankVote) return batch_occupancy(p, k_batch<KIND, PAIRS, 8, 16, kRankVote>, 256, sm_count);
  return batch_occupancy(p, k_batch<KIND, PAIRS, 8, 16, kRankTable>, 256, sm_count);
}

template <int KIND, bool PAIRS>
static cudaError_t batch_launch(const ms_batch_plan& p, cudaStream_t s) {
  BatchArgs a;
  a.segs = p.d_segs;
  a.items = p.d_items;
  a.H = p.d_H;
  a.done = p.d_flags;
  a.ready = p.d_flags + p.max_segments;
  a.ticket = p.d_flags + 2 * p.max_segments;
  a.err = p.d_err;
  a.K = p.K;
  a.sp = p.sp;
  if (p.rank == kRankThread)
    k_batch_tc<KIND, PAIRS><<<p.grid, kTcThreads, p.smem, s>>>(a, p.lb, p.lw);
  else if (p.shape == 1 && p.rank == kRankVote)
    k_batch<KIND, PAIRS, 16, 8, kRankVote><<<p.grid, 512, p.smem, s>>>(a);
  else if (p.shape == 1)
    k_batch<KIND, PAIRS, 16, 8, kRankTable><<<p.grid, 512, p.smem, s>>>(a);
  else if (p.rank == kRankVote)
    k_batch<KIND, PAIRS, 8, 16, kRankVote><<<p.grid, 256, p.smem, s>>>(a);
  else
    k_batch<KIND, PAIRS, 8, 16, kRankTable><<<p.grid, 256, p.smem, s>>>(a);
  return cudaGetLastError();
}

template <int KIND>
static cudaError_t batch_dispatch(ms_batch_plan& p, int sm_count, cudaStream_t s, bool setup) {
  if (p.pairs) return setup ? batch_setup<KIND, true>(p, sm_count) : batch_launch<KIND, true>(p, s);
  return setup ? batch_setup<KIND, false>(p, sm_count) : batch_launch<KIND, false>(p, s);
}

static cudaError_t batch_call(ms_batch_plan& p, int sm_count, cudaStream_t s, bool setup) {
  switch (p.kind) {
    case kRange: return batch_dispatch<kRange>(p, sm_count, s, setup);
    case kDelta: return batch_dispatch<kDelta>(p, sm_count, s, setup);
    case kRadix: return batch_dispatch<kRadix>(p, sm_count, s, setup);
    default: return batch_dispatch<kMod>(p, sm_count, s, setup);
  }
}

// Plans alive per device (ms_shutdown refuses to run while a caller's plan
// still refers to the device's status word).
static std::atomic<int> g_live_plans[64];

static void plan_free(ms_batch_plan* p) {
  if (p == nullptr) return;
  if (p->device >= 0 && p->device < 64) g_live_plans[p->device].fetch_sub(1);
  if (p->graph) cudaGraphExecDestroy(p->graph);
  for (int k = 0; k < 2; ++k) {
    if (p->stage_done[k]) cudaEventDestroy(p->stage_done[k]);
    if (p->h_stage[k]) cudaFreeHost(p->h_stage[k]);
  }
  cudaFree(p->d_segs);
  cudaFree(p->d_items);
  cudaFree(p->d_H);
  cudaFree(p->d_flags);
  delete p;
}

}  // namespace ms

namespace ms {

// The kernel a plan runs and its tiles per work item.
static void plan_kernel(int kind, bool pairs, const DevSpec& sp, uint64_t mean_n, int* rank, int* shape,
                        uint32_t* K) {
  const Variant v = choose_batch_variant(kind, pairs, sp.nbits, mean_n);
  *rank = (v.rank == kRankThread && sp.m > kTcMaxM) ? kRankTable : v.rank;
  *shape = *rank == kRankThread ? 0 : v.shape;
  *K = *rank == kRankThread ? kBatchChunkTiles : 1u;
}

// Validates segs and builds the segment table and the work list of items of
// up to K tiles: the histogram items, then the post-scan items (measured on
// GB300: interleaving waves of segments' histograms and post-scans, for the
// post-scans to find their keys in L2, was slower -- post-scans waiting on
// histograms still in progress -- and post-scans in reverse segment order no
// faster).  Every post-scan item comes after all histogram items of its
// segment, which is all the protocol needs:
// if every running CTA were blocked, the one whose current item has the
// smallest ticket would wait for a histogram item of a smaller ticket, held
// by a CTA that is either working on it (histogram items never wait) or
// blocked on an item of a still smaller ticket -- a contradiction.  Returns
// the histogram words needed in *hwords.
static ms_status build_work(const ms_segment* segs, uint32_t num, const DevSpec& sp, bool pairs, uint32_t K,
                            DevSeg* hs, std::vector<uint2>& items, uint64_t* hwords) {
  std::vector<uint2> post;
  items.clear();
  items.push_back(make_uint2(0u, 0u));  // counts, filled below
  uint64_t hw = 0;
  for (uint32_t i = 0; i < num; ++i) {
    const ms_segment& g = segs[i];
    if (g.n >= ((size_t)1 << 32)) return MS_ERR_INVALID_ARG;
    // an empty segment may leave every pointer NULL
    if (g.n > 0 && ((g.vals_in != nullptr) != pairs || (g.vals_out != nullptr) != pairs)) return MS_ERR_INVALID_ARG;
    const size_t bytes = g.n * 4;
    if (g.n > 0 && (g.keys_in == nullptr || g.keys_out == nullptr || overlap(g.keys_in, g.keys_out, bytes)))
      return MS_ERR_INVALID_ARG;
    if (pairs && g.n > 0 &&
        (overlap(g.vals_in, g.vals_out, bytes) || overlap(g.vals_out, g.keys_out, bytes) ||
         overlap(g.vals_out, g.keys_in, bytes) || overlap(g.keys_out, g.vals_in, bytes)))
      return MS_ERR_INVALID_ARG;
    DevSeg d;
    std::memset(&d, 0, sizeof d);
    d.kin = g.keys_in;
    d.vin = g.vals_in;
    d.kout = g.keys_out;
    d.vout = g.vals_out;
    d.offsets = g.offsets;
    d.n = (uint32_t)g.n;
    // an empty segment still gets one (empty) item: it writes zero offsets
    d.L = std::max<uint32_t>(1u, (uint32_t)((g.n + kBatchTile - 1) / kBatchTile));
    d.C = (d.L + K - 1) / K;
    if (d.L > 1) {
      d.hoff = (uint32_t)hw;
      hw += (uint64_t)sp.m * d.C;
      for (uint32_t t = 0; t < d.L; t += K) items.push_back(make_uint2(i, t));
    }
    for (uint32_t t = 0; t < d.L; t += K) post.push_back(make_uint2(i, t | kBatchPost));
    hs[i] = d;
  }
  const uint32_t n_hist = (uint32_t)(items.size() - 1);
  items.insert(items.end(), post.begin(), post.end());
  items[0] = make_uint2(n_hist, (uint32_t)(items.size() - 1));
  if (hw >= ((uint64_t)1 << 32)) return MS_ERR_UNSUPPORTED;
  *hwords = hw;
  return MS_OK;
}

// Allocates a plan's device memory for the given capacities.
static ms_status plan_alloc(ms_batch_plan* p, DeviceCtx* ctx, int kind, bool pairs, const DevSpec& sp,
                            uint32_t max_segments, uint32_t max_items, uint64_t max_hwords, uint64_t mean_n) {
  p->device = ctx->device;
  if (p->device >= 0 && p->device < 64) g_live_plans[p->device].fetch_add(1);
  p->kind = kind;
  p->pairs = pairs;
  p->sp = sp;
  p->d_err = ctx->d_err;
  p->max_segments = max_segments;
  p->max_items = max_items;
  plan_kernel(kind, pairs, sp, mean_n, &p->rank, &p->shape, &p->K);
  p->max_hwords = max_hwords;
  p->flags_bytes = ((size_t)2 * max_segments + 4) * 4;
  cudaError_t e = cudaMalloc(&p->d_segs, std::max<size_t>(1, max_segments) * sizeof(DevSeg));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_items, ((size_t)max_items + 1) * sizeof(uint2));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_H, std::max<uint64_t>(1, max_hwords) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_flags, p->flags_bytes);
  if (e == cudaSuccess) e = cudaMemset(p->d_items, 0, sizeof(uint2));
  if (e == cudaSuccess) e = batch_call(*p, ctx->sm_count, nullptr, true);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MS_ERR_OUT_OF_MEMORY : MS_ERR_CUDA;
  }
  return MS_OK;
}

}  // namespace ms

extern "C" ms_status ms_batch_plan_create(const ms_segment* segs, uint32_t num_segments, const ms_bucket_spec* spec,
                                          ms_batch_plan** plan) {
  if (plan == nullptr) return MS_ERR_INVALID_ARG;
  *plan = nullptr;
  if (num_segments > 0 && segs == nullptr) return MS_ERR_INVALID_ARG;
  DevSpec sp;
  int kind = 0;
  ms_status st = make_devspec(spec, &sp, &kind);
  if (st != MS_OK) return st;
  bool pairs = false;  // key-value if any segment carries values
  for (uint32_t i = 0; i < num_segments; ++i) pairs = pairs || segs[i].vals_in != nullptr;
  uint64_t total = 0;
  for (uint32_t i = 0; i < num_segments; ++i) total += segs[i].n;
  const uint64_t mean_n = num_segments ? total / num_segments : 0;
  int rank = 0, shape = 0;
  uint32_t K = 1;
  plan_kernel(kind, pairs, sp, mean_n, &rank, &shape, &K);
  std::vector<DevSeg> hs(num_segments);
  std::vector<uint2> items;
  uint64_t hwords = 0;
  st = build_work(segs, num_segments, sp, pairs, K, hs.data(), items, &hwords);
  if (st != MS_OK) return st;
  DeviceCtx* ctx = nullptr;
  st = current_device_ctx(&ctx);
  if (st != MS_OK) return st;
  auto* p = new ms_batch_plan();
  st = plan_alloc(p, ctx, kind, pairs, sp, num_segments, (uint32_t)(items.size() - 1), hwords, mean_n);
  p->num_segments = num_segments;
  p->n_items = items[0].y;
  cudaError_t e = cudaSuccess;
  if (st == MS_OK && !hs.empty())
    e = cudaMemcpy(p->d_segs, hs.data(), hs.size() * sizeof(DevSeg), cudaMemcpyHostToDevice);
  if (st == MS_OK && e == cudaSuccess)
    e = cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(uint2), cudaMemcpyHostToDevice);
  if (st == MS_OK && e != cudaSuccess) st = to_status(e);
  if (st != MS_OK) {
    plan_free(p);
    return st;
  }
  *plan = p;
  return MS_OK;
}

extern "C" ms_status ms_batch_plan_create_dynamic(uint32_t max_segments, uint64_t max_elements, int pairs,
                                                  const ms_bucket_spec* spec, ms_batch_plan** plan) {
  if (plan == nullptr) return MS_ERR_INVALID_ARG;
  *plan = nullptr;
  if (max_segments == 0) return MS_ERR_INVALID_ARG;
  DevSpec sp;
  int kind = 0;
  ms_status st = make_devspec(spec, &sp, &kind);
  if (st != MS_OK) return st;
  // every segment adds at most one partial tile
  const uint64_t tiles = max_elements / kBatchTile + max_segments;
  if (2 * tiles >= ((uint64_t)1 << 31)) return MS_ERR_INVALID_ARG;
  DeviceCtx* ctx = nullptr;
  st = current_device_ctx(&ctx);
  if (st != MS_OK) return st;
  auto* p = new ms_batch_plan();
  st = plan_alloc(p, ctx, kind, pairs != 0, sp, max_segments, (uint32_t)(2 * tiles), (uint64_t)sp.m * tiles,
                  max_elements / max_segments);
  const size_t stage_bytes = (size_t)max_segments * sizeof(DevSeg) + ((size_t)2 * tiles + 1) * sizeof(uint2);
  for (int k = 0; k < 2 && st == MS_OK; ++k) {
    if (cudaMallocHost(&p->h_stage[k], stage_bytes) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->stage_done[k], cudaEventDisableTiming) != cudaSuccess)
      st = MS_ERR_OUT_OF_MEMORY;
  }
  if (st != MS_OK) {
    cudaGetLastError();
    plan_free(p);
    return st;
  }
  *plan = p;
  return MS_OK;
}

extern "C" ms_status ms_batch_plan_set_segments(ms_batch_plan* plan, const ms_segment* segs, uint32_t num_segments,
                                                void* stream) {
  if (plan == nullptr || plan->h_stage[0] == nullptr) return MS_ERR_INVALID_ARG;
  if (num_segments > plan->max_segments || (num_segments > 0 && segs == nullptr)) return MS_ERR_INVALID_ARG;
  const int k = plan->stage_next;
  // the staging area is free once its previous upload has been read
  if (cudaEventSynchronize(plan->stage_done[k]) != cudaSuccess) return MS_ERR_CUDA;
  DevSeg* hs = static_cast<DevSeg*>(plan->h_stage[k]);
  std::vector<uint2> items;
  uint64_t hwords = 0;
  ms_status st = build_work(segs, num_segments, plan->sp, plan->pairs, plan->K, hs, items, &hwords);
  if (st != MS_OK) return st;
  if (items.size() - 1 > plan->max_items || hwords > plan->max_hwords) return MS_ERR_INVALID_ARG;
  uint2* hi = reinterpret_cast<uint2*>(static_cast<char*>(plan->h_stage[k]) +
                                       (size_t)plan->max_segments * sizeof(DevSeg));
  std::memcpy(hi, items.data(), items.size() * sizeof(uint2));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (num_segments > 0) e = cudaMemcpyAsync(plan->d_segs, hs, num_segments * sizeof(DevSeg), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_items, hi, items.size() * sizeof(uint2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(plan->stage_done[k], s);
  if (e != cudaSuccess) return to_status(e);
  plan->num_segments = num_segments;
  plan->n_items = items[0].y;
  plan->stage_next = k ^ 1;
  return MS_OK;
}

extern "C" ms_status ms_batch_run(ms_batch_plan* plan, void* stream) {
  if (plan == nullptr) return MS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MS_ERR_CUDA;
  if (dev != plan->device) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(plan->d_flags, 0, plan->flags_bytes, s);
  if (e == cudaSuccess) e = batch_call(*plan, 0, s, false);
  return to_status(e);
}

extern "C" ms_status ms_batch_run_graph(ms_batch_plan* plan, void* stream) {
  if (plan == nullptr) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (plan->graph == nullptr) {
    // capture the memset and the launch once, on a private stream
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MS_ERR_CUDA;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    ms_status st = MS_OK;
    if (e == cudaSuccess) {
      st = ms_batch_run(plan, cs);
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess && st == MS_OK) e = cudaGraphInstantiate(&plan->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != MS_OK) return st;
    if (e != cudaSuccess) return to_status(e);
  }
  return to_status(cudaGraphLaunch(plan->graph, s));
}

extern "C" ms_status ms_batch_plan_destroy(ms_batch_plan* plan) {
  if (plan == nullptr) return MS_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
  }
  plan_free(plan);
  return MS_OK;
}

// ---------------------------------------------------------------------------
// One call over device-resident segment descriptors.  The descriptors are
// read back to the host (the work list is built there, as for the plans
// above), then the work runs through a dynamic plan kept in a small
// per-process cache keyed by device, bucket spec and keys-only / key-value,
// and grown when a call needs more segments or elements than it holds.
namespace ms {
namespace {
struct CachedPlan {
  int device;
  bool pairs;
  ms_bucket_spec spec;
  uint32_t max_segments;
  uint64_t max_elements;
  ms_batch_plan* plan;
  cudaEvent_t last_run;  // recorded after the plan's latest run
  uint64_t stamp;        // least recently used is evicted first
};
std::mutex g_cache_mu;
std::vector<CachedPlan> g_cache;
uint64_t g_cache_clock = 0;
constexpr size_t kCacheEntries = 8;

bool same_spec(const ms_bucket_spec& a, const ms_bucket_spec& b) {
  return a.kind == b.kind && a.m == b.m && a.splitters == b.splitters && a.x0 == b.x0 && a.delta == b.delta &&
         a.shift == b.shift && a.bits == b.bits;
}

void release_entry(CachedPlan& c) {
  if (c.last_run) {
    cudaEventSynchronize(c.last_run);
    cudaEventDestroy(c.last_run);
  }
  plan_free(c.plan);
  c.plan = nullptr;
  c.last_run = nullptr;
}

uint64_t round_up_pow2(uint64_t v, uint64_t floor_v) {
  uint64_t r = floor_v;
  while (r < v) r <<= 1;
  return r;
}
}  // namespace

int batch_live_plans(int dev) {
  if (dev < 0 || dev >= 64) return 0;
  int cached = 0;
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (const auto& c : g_cache) cached += c.device == dev ? 1 : 0;
  }
  return g_live_plans[dev].load() - cached;
}

void batch_cache_release(int dev) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  for (auto& c : g_cache)
    if (c.device == dev) release_entry(c);
  g_cache.erase(std::remove_if(g_cache.begin(), g_cache.end(), [](const CachedPlan& c) { return c.plan == nullptr; }),
                g_cache.end());
}

}  // namespace ms

extern "C" ms_status ms_multisplit_pairs_batched(const ms_segment* segs_dev, uint32_t num_segments,
                                                 const ms_bucket_spec* spec, uint32_t* offsets, void* stream) {
  DevSpec sp;
  int kind = 0;
  ms_status st = make_devspec(spec, &sp, &kind);
  if (st != MS_OK) return st;
  if (num_segments == 0) return MS_OK;
  if (segs_dev == nullptr) return MS_ERR_INVALID_ARG;
  DeviceCtx* ctx = nullptr;
  st = current_device_ctx(&ctx);
  if (st != MS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<ms_segment> segs(num_segments);
  cudaError_t e = cudaMemcpyAsync(segs.data(), segs_dev, num_segments * sizeof(ms_segment), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return to_status(e);
  bool pairs = false;
  uint64_t total = 0;
  for (uint32_t i = 0; i < num_segments; ++i) {
    if (offsets != nullptr) segs[i].offsets = offsets + (size_t)i * (sp.m + 1);
    if (segs[i].n >= ((size_t)1 << 32)) return MS_ERR_INVALID_ARG;
    pairs = pairs || (segs[i].n > 0 && segs[i].vals_in != nullptr);
    total += segs[i].n;
  }
  std::lock_guard<std::mutex> lock(g_cache_mu);
  CachedPlan* hit = nullptr;
  for (auto& c : g_cache)
    if (c.device == ctx->device && c.pairs == pairs && same_spec(c.spec, *spec) && c.max_segments >= num_segments &&
        c.max_elements >= total)
      hit = &c;
  if (hit == nullptr) {
    // a new plan, a little larger than needed so that nearby calls reuse it;
    // replaces a smaller one for the same spec, else the least recently used
    CachedPlan c;
    std::memset(&c, 0, sizeof c);
    c.device = ctx->device;
    c.pairs = pairs;
    c.spec = *spec;
    c.max_segments = (uint32_t)round_up_pow2(num_segments, 64);
    c.max_elements = round_up_pow2(total, (uint64_t)1 << 20);
    st = ms_batch_plan_create_dynamic(c.max_segments, c.max_elements, pairs ? 1 : 0, spec, &c.plan);
    if (st != MS_OK) return st;
    if (cudaEventCreateWithFlags(&c.last_run, cudaEventDisableTiming) != cudaSuccess) {
      plan_free(c.plan);
      return to_status(cudaGetLastError());
    }
    size_t victim = g_cache.size();
    for (size_t i = 0; i < g_cache.size(); ++i)
      if (g_cache[i].device == c.device && g_cache[i].pairs == pairs && same_spec(g_cache[i].spec, *spec)) victim = i;
    if (victim == g_cache.size() && g_cache.size() >= kCacheEntries) {
      victim = 0;
      for (size_t i = 1; i < g_cache.size(); ++i)
        if (g_cache[i].stamp < g_cache[victim].stamp) victim = i;
    }
    if (victim < g_cache.size()) {
      release_entry(g_cache[victim]);
      g_cache[victim] = c;
      hit = &g_cache[victim];
    } else {
      g_cache.push_back(c);
      hit = &g_cache.back();
    }
  }
  hit->stamp = ++g_cache_clock;
  // the plan's previous run (possibly on another stream) reads the segment
  // table and work list that the upload below replaces
  e = cudaStreamWaitEvent(s, hit->last_run, 0);
  if (e != cudaSuccess) return to_status(e);
  st = ms_batch_plan_set_segments(hit->plan, segs.data(), num_segments, stream);
  if (st != MS_OK) return st;
  st = ms_batch_run(hit->plan, stream);
  if (st != MS_OK) return st;
  return to_status(cudaEventRecord(hit->last_run, s));
}
