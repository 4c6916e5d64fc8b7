// ms_scan.cu -- the single-pass look-back scan kernel of the global stage (see
// ms_scan.cuh for what it computes).
#include "ms_scan.cuh"

namespace ms {

__global__ void __launch_bounds__(kScanThreads) k_scan_lookback(ScanArgs a) {
  __shared__ uint32_t s_tile, s_excl;
  __shared__ uint32_t s_warp[kScanThreads / 32];
  if (threadIdx.x == 0) s_tile = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const size_t i0 = (size_t)tile * kScanTile + (size_t)threadIdx.x * kScanItems;

  uint32_t v[kScanItems];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (i0 + k < a.len) ? a.data[i0 + k] : 0u;
    sum += v[k];
  }
  uint32_t agg;
  const uint32_t tpre = block_exclusive_scan<kScanThreads / 32>(sum, s_warp, &agg);

  if (threadIdx.x == 0) {
    uint32_t excl = 0;
    if (tile == 0) {
      st_relaxed_u64(a.status, kFlagPrefix | agg);
    } else {
      st_relaxed_u64(a.status + tile, kFlagAggregate | agg);
      for (int p = (int)tile - 1; p >= 0; --p) {
        const unsigned long long st = wait_status(a.status + p, a.err);
        excl += (uint32_t)st;
        if ((st >> 32) == (kFlagPrefix >> 32)) break;
      }
      st_relaxed_u64(a.status + tile, kFlagPrefix | (uint32_t)(excl + agg));
    }
    s_excl = excl;
    if (a.offsets != nullptr && (size_t)(tile + 1) * kScanTile >= a.len) a.offsets[a.m] = excl + agg;
  }
  __syncthreads();

  uint32_t run = s_excl + tpre;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const size_t i = i0 + k;
    if (i < a.len) {
      a.data[i] = run;
      if (a.offsets != nullptr && (uint32_t)(i % a.G) == 0u) a.offsets[i / a.G] = run;
    }
    run += v[k];
  }
}

cudaError_t launch_scan_lookback(const ScanArgs& a, cudaStream_t stream) {
  const uint32_t tiles = (a.len + kScanTile - 1) / kScanTile;
  k_scan_lookback<<<tiles, kScanThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scan_tiles(const ScanArgs& a, uint32_t ctas, cudaStream_t stream) {
  k_scan_lookback<<<ctas, kScanThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace ms
