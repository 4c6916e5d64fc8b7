// ms_noalloc.cu -- a keys-only multisplit that allocates no memory.
//
// Why it exists: some callers of this library cannot let it allocate device
// memory at call time.  Examples: latency-critical loops that forbid
// allocator calls on their hot path, and hosts whose device memory is entirely
// handed out by another allocator (a framework's caching pool), where a
// second allocator would fragment or oversubscribe it.  For them,
// ms_multisplit_keys_noalloc runs the same kernels as ms_multisplit_keys, with
// the scratch (histogram matrix, arrival counter or look-back status words and
// ticket) taken from a fixed array in device memory that is part of the loaded
// library instead of from the library's memory pool.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library is loaded holds kStaticScratchBytes of it until the process exits.
// In host code its name is only a host-side handle, not a device address, so
// the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and remembers it.  The first
// call that uses a given kernel variant (bucket kind, m and the size class of
// n pick it) also sets that kernel's attributes and queries its occupancy;
// later calls skip these host-side steps.  All calls share the
// array: calls that overlap on the GPU (concurrent streams, or several
// devices' worth of work racing on one device) race on it and corrupt each
// other; serialize them.  Each call clears the words that must start at zero
// (arrival counter, status words, ticket).
//
// Device-side failures: the first 256 bytes of the array are a header.  Word
// 0 is the status word of the call in flight -- its kernels set a bit there
// when a bounded wait expires or an index check fails, and once the timeout
// bit is set the other waits of that call give up early.  Word 1 keeps the
// bits of earlier calls: every call starts with a one-thread kernel that moves
// word 0 into word 1 and clears word 0, so one expired wait never shortens the
// waits of a later call.  ms_noalloc_status() reads both words and clears them.
#include <cstring>
#include <mutex>

#include "ms.h"
#include "ms_host.h"
#include "ms_scan.cuh"

namespace ms {

// 1 MiB: the first 256 bytes are the header (word 0: status of the call in
// flight, word 1: status bits of earlier calls), the rest the scratch.  The
// scratch needs 4*m*G bytes for the histogram matrix (G = CTAs of the launch,
// at most SMs x resident CTAs per SM) plus 16 bytes, and for m > 32 8 bytes per
// 4096 matrix entries of look-back status; on a 152-SM GB300 (G <= 4 * 152)
// that is at most about 610 KiB.
constexpr size_t kStaticScratchBytes = (size_t)1 << 20;
constexpr size_t kStaticHeader = 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_mu;
void* g_scratch_ptr[64] = {};
int g_sm_count[64] = {};
}  // namespace

// Device address of the static scratch on the current device (looked up once
// per device, with that device current).
static ms_status static_scratch(int dev, void** ptr, int* sms) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return MS_ERR_CUDA;
    }
    int s = 0;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MS_ERR_CUDA;
    g_scratch_ptr[dev] = p;
    g_sm_count[dev] = s;
  }
  *ptr = g_scratch_ptr[dev];
  *sms = g_sm_count[dev];
  return MS_OK;
}

// Moves the status bits of the previous call (word 0) into word 1 and clears
// word 0 for the call that follows on the stream.
__global__ void k_noalloc_fold_status(uint32_t* hdr) {
  hdr[1] |= hdr[0];
  hdr[0] = 0u;
}

// The fixed array on the current device: its address and the SM count.
static ms_status current_static_scratch(void** base, int* sms, int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MS_ERR_CUDA;
  if (dev < 0 || dev >= 64) return MS_ERR_UNSUPPORTED;
  *dev_out = dev;
  return static_scratch(dev, base, sms);
}

}  // namespace ms

using namespace ms;

extern "C" ms_status ms_multisplit_keys_noalloc(const uint32_t* keys_in, size_t n, const ms_bucket_spec* spec,
                                                uint32_t* keys_out, uint32_t* offsets, void* stream) {
  Call c;
  std::memset(&c, 0, sizeof c);
  ms_status st = make_devspec(spec, &c.sp, &c.kind);
  if (st != MS_OK) return st;
  if (n >= ((size_t)1 << 32)) return MS_ERR_INVALID_ARG;
  if (n > 0 && (keys_in == nullptr || keys_out == nullptr || overlap(keys_in, keys_out, n * sizeof(uint32_t))))
    return MS_ERR_INVALID_ARG;
  int dev = 0;
  void* base = nullptr;
  int sms = 0;
  st = current_static_scratch(&base, &sms, &dev);
  if (st != MS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (offsets != nullptr) return to_status(cudaMemsetAsync(offsets, 0, (size_t)(c.sp.m + 1) * 4, s));
    return MS_OK;
  }
  k_noalloc_fold_status<<<1, 1, 0, s>>>(static_cast<uint32_t*>(base));
  if (cudaPeekAtLastError() != cudaSuccess) return to_status(cudaGetLastError());
  DeviceCtx ctx;  // no pool: nothing is allocated on this path
  ctx.device = dev;
  ctx.sm_count = sms;
  ctx.pool = nullptr;
  ctx.d_err = static_cast<uint32_t*>(base);
  c.keys_in = keys_in;
  c.keys_out = keys_out;
  c.offsets = offsets;
  c.n = (uint32_t)n;
  c.stream = s;
  c.ws_fixed = static_cast<unsigned char*>(base) + kStaticHeader;
  c.ws_capacity = kStaticScratchBytes - kStaticHeader;
  return to_status(run_multisplit(c, ctx));
}

extern "C" ms_status ms_noalloc_status(void* stream) {
  int dev = 0, sms = 0;
  void* base = nullptr;
  ms_status st = current_static_scratch(&base, &sms, &dev);
  if (st != MS_OK) return st;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return to_status(cudaGetLastError());
  uint32_t h[2] = {0u, 0u};
  if (cudaMemcpy(h, base, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return to_status(cudaGetLastError());
  if (cudaMemset(base, 0, sizeof h) != cudaSuccess) return to_status(cudaGetLastError());
  const uint32_t bits = h[0] | h[1];
  if (bits & kDevErrTimeout) return MS_ERR_TIMEOUT;
  return bits == 0u ? MS_OK : MS_ERR_CUDA;
}

// Failure-path test aid for this entry point: the look-back scan kernel runs
// as the second of two scan tiles on the fixed array's scratch, with the
// first tile's status word never published, so its bounded wait runs out and
// sets the timeout bit of header word 0, as an expired wait inside a call
// would.  Enqueued on `stream`; nothing else is touched.
extern "C" ms_status ms_test_expire_lookback_noalloc(void* stream) {
  int dev = 0, sms = 0;
  void* base = nullptr;
  ms_status st = current_static_scratch(&base, &sms, &dev);
  if (st != MS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* hdr = static_cast<uint32_t*>(base);
  // scratch: two scan tiles of data | two status words | ticket
  unsigned char* ws = static_cast<unsigned char*>(base) + kStaticHeader;
  const size_t data_bytes = (size_t)2 * kScanTile * 4;
  auto* status = reinterpret_cast<unsigned long long*>(ws + data_bytes);
  auto* ticket = reinterpret_cast<uint32_t*>(ws + data_bytes + 16);
  k_noalloc_fold_status<<<1, 1, 0, s>>>(hdr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, data_bytes + 16 + 4, s);
  // ticket = 1 (little-endian low byte): the only CTA is tile 1, whose predecessor never runs
  if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 1, 1, s);
  if (e == cudaSuccess) {
    ScanArgs a{reinterpret_cast<uint32_t*>(ws), (uint32_t)(2 * kScanTile), 1u, nullptr, 1u, status, ticket, hdr};
    e = launch_scan_tiles(a, 1, s);
  }
  return to_status(e);
}
