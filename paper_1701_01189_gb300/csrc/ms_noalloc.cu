// ms_noalloc.cu -- a keys-only multisplit that allocates no memory.
//
// Why it exists: some callers of this library cannot let it allocate device
// memory at call time.  Examples: code that enqueues work while a CUDA graph is
// being captured and must not add allocation nodes to it; latency-critical
// loops that forbid allocator calls on their hot path; and hosts whose device
// memory is entirely handed out by another allocator (a framework's caching
// pool), where a second allocator would fragment or oversubscribe it.  For
// them, ms_multisplit_keys_noalloc runs the same kernels as
// ms_multisplit_keys, with the scratch (histogram matrix, arrival counter or
// look-back status words and ticket) taken from a fixed array in device
// memory that is part of the loaded library instead of from the library's
// memory pool.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library is loaded holds kStaticScratchBytes of it until the process exits.
// In host code its name is only a host-side handle, not a device address, so
// the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and remembers it.  That first
// call also sets kernel attributes and queries occupancy; make it before any
// stream capture.  All calls share the array: calls that overlap on the GPU
// (concurrent streams, or several devices' worth of work racing on one device)
// race on it and corrupt each other; serialize them.  Each call clears the
// words that must start at zero (arrival counter, status words, ticket).
#include <cstring>
#include <mutex>

#include "ms.h"
#include "ms_host.h"

namespace ms {

// 1 MiB: the first 256 bytes hold this entry point's device status word, the
// rest the scratch.  The scratch needs 4*m*G bytes for the histogram matrix
// (G = CTAs of the launch, at most SMs x resident CTAs per SM) plus 16 bytes,
// and for m > 32 8 bytes per 4096 matrix entries of look-back status; on a
// 152-SM GB300 (G <= 4 * 152) that is at most about 610 KiB.
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
  if (cudaGetDevice(&dev) != cudaSuccess) return MS_ERR_CUDA;
  if (dev < 0 || dev >= 64) return MS_ERR_UNSUPPORTED;
  void* base = nullptr;
  int sms = 0;
  st = static_scratch(dev, &base, &sms);
  if (st != MS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (offsets != nullptr) return to_status(cudaMemsetAsync(offsets, 0, (size_t)(c.sp.m + 1) * 4, s));
    return MS_OK;
  }
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
