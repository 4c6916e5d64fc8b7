// ms_api.cu -- the C ABI of libms.so (declared in include/ms.h): argument
// validation, per-device state, the scratch pool, dispatch to the per-kind
// multisplit launchers, and the radix sort driver of Section 7.1.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ms.h"
#include "ms_host.h"
#include "ms_scan.cuh"

namespace ms {

static std::mutex g_ctx_mu;
static DeviceCtx g_ctx[64];

ms_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return MS_OK;
  cudaGetLastError();  // clear a sticky launch error of this thread
  return e == cudaErrorMemoryAllocation ? MS_ERR_OUT_OF_MEMORY : MS_ERR_CUDA;
}

// The state of the current device, created on first use (this first call
// allocates and must not run inside a CUDA graph capture).
static ms_status current_ctx(DeviceCtx** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MS_ERR_CUDA;
  if (dev < 0 || dev >= 64) return MS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_ctx_mu);
  DeviceCtx& c = g_ctx[dev];
  if (c.device < 0) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MS_ERR_CUDA;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return MS_ERR_CUDA;
    uint64_t keep = UINT64_MAX;  // keep freed scratch cached in the pool
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    // scratch freed on one stream is not handed to another by making the
    // second wait on the first: concurrent calls on different streams stay
    // concurrent (the pool grows instead)
    int no = 0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    uint32_t* d_err = nullptr;
    if (cudaMalloc(&d_err, sizeof(uint32_t)) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return MS_ERR_OUT_OF_MEMORY;
    }
    if (cudaMemset(d_err, 0, sizeof(uint32_t)) != cudaSuccess) return MS_ERR_CUDA;
    c.sm_count = sms;
    c.pool = pool;
    c.d_err = d_err;
    c.device = dev;
  }
  *out = &c;
  return MS_OK;
}

ms_status current_device_ctx(DeviceCtx** out) { return current_ctx(out); }

cudaError_t scratch_alloc(DeviceCtx& ctx, void** p, size_t bytes, cudaStream_t stream) {
  return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, ctx.pool, stream);
}

cudaError_t scratch_free(void* p, cudaStream_t stream) { return p ? cudaFreeAsync(p, stream) : cudaSuccess; }

cudaError_t run_multisplit(const Call& c, DeviceCtx& ctx) {
  switch (c.kind) {
    case kRange: return run_multisplit_range(c, ctx);
    case kDelta: return run_multisplit_delta(c, ctx);
    case kRadix: return run_multisplit_radix(c, ctx);
    case kMod: return run_multisplit_mod(c, ctx);
  }
  return cudaErrorInvalidValue;
}

static uint32_t ceil_log2(uint32_t m) {
  uint32_t l = 0;
  while ((1u << l) < m) ++l;
  return l;
}

// Validates a bucket spec and converts it to kernel terms.
ms_status make_devspec(const ms_bucket_spec* spec, DevSpec* out, int* kind) {
  if (spec == nullptr) return MS_ERR_INVALID_ARG;
  const uint32_t m = spec->m;
  if (m < 1 || m > (uint32_t)kMaxM) return MS_ERR_INVALID_ARG;
  DevSpec d;
  std::memset(&d, 0, sizeof d);
  d.m = m;
  d.nbits = ceil_log2(m);
  d.m_pad = m <= 32 ? 32u : ((m + 31u) & ~31u);
  d.lut_bits = m <= 64 ? 10u : 11u;
  if (m == 1) {
    // every key is in bucket 0: any identifier reduces to the empty radix digit
    if (spec->kind < MS_BUCKET_RANGE_U32 || spec->kind > MS_BUCKET_MOD) return MS_ERR_INVALID_ARG;
    if (spec->kind == MS_BUCKET_DELTA_F32 &&
        (!std::isfinite(spec->x0) || !std::isfinite(spec->delta) || !(spec->delta > 0.0f)))
      return MS_ERR_INVALID_ARG;
    if (spec->kind == MS_BUCKET_RADIX && (spec->bits != 0 || spec->shift > 32)) return MS_ERR_INVALID_ARG;
    d.shift = 0;
    d.mask = 0;
    *kind = kRadix;
    *out = d;
    return MS_OK;
  }
  switch (spec->kind) {
    case MS_BUCKET_RANGE_U32:
      if (m > 1 && spec->splitters == nullptr) return MS_ERR_INVALID_ARG;
      d.splitters = spec->splitters;
      *kind = kRange;
      break;
    case MS_BUCKET_DELTA_F32:
      if (!std::isfinite(spec->x0) || !std::isfinite(spec->delta) || !(spec->delta > 0.0f))
        return MS_ERR_INVALID_ARG;
      d.x0 = spec->x0;
      d.delta = spec->delta;
      d.rdelta = 1.0f / spec->delta;
      *kind = kDelta;
      break;
    case MS_BUCKET_RADIX:
      if (spec->bits > 8 || m != (1u << spec->bits) || spec->shift + spec->bits > 32) return MS_ERR_INVALID_ARG;
      d.shift = spec->bits == 0 ? 0u : spec->shift;
      d.mask = (1u << spec->bits) - 1u;
      *kind = kRadix;
      break;
    case MS_BUCKET_MOD: {
      // Granlund-Montgomery constants for unsigned division by m:
      // l = ceil(log2 m), M = floor(2^32 (2^l - m) / m) + 1, sh1 = min(l, 1),
      // sh2 = max(l - 1, 0).
      const uint32_t l = d.nbits;
      const uint64_t M = (((uint64_t)1 << 32) * (((uint64_t)1 << l) - m)) / m + 1;
      d.mod_magic = (uint32_t)M;
      d.mod_sh1 = l < 1 ? l : 1u;
      d.mod_sh2 = l > 0 ? l - 1 : 0u;
      *kind = kMod;
      break;
    }
    default:
      return MS_ERR_INVALID_ARG;
  }
  *out = d;
  return MS_OK;
}

bool overlap(const void* a, const void* b, size_t bytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes && y < x + bytes;
}

static ms_status multisplit_impl(const uint32_t* keys_in, const uint32_t* vals_in, size_t n,
                                 const ms_bucket_spec* spec, uint32_t* keys_out, uint32_t* vals_out,
                                 uint32_t* offsets, void* stream, bool pairs) {
  Call c;
  std::memset(&c, 0, sizeof c);
  WideSpec w;
  std::memset(&w, 0, sizeof w);
  const bool wide = spec != nullptr && spec->m > (uint32_t)kMaxM;
  ms_status st = wide ? make_wide_spec(spec, &w) : make_devspec(spec, &c.sp, &c.kind);
  if (st != MS_OK) return st;
  const uint32_t m = wide ? w.fm : c.sp.m;
  if (n >= ((size_t)1 << 32)) return MS_ERR_INVALID_ARG;
  const size_t bytes = n * sizeof(uint32_t);
  if (n > 0) {
    if (keys_in == nullptr || keys_out == nullptr) return MS_ERR_INVALID_ARG;
    if (overlap(keys_in, keys_out, bytes)) return MS_ERR_INVALID_ARG;
    if (pairs) {
      if (vals_in == nullptr || vals_out == nullptr) return MS_ERR_INVALID_ARG;
      if (overlap(vals_in, vals_out, bytes) || overlap(vals_out, keys_out, bytes) ||
          overlap(vals_out, keys_in, bytes) || overlap(keys_out, vals_in, bytes))
        return MS_ERR_INVALID_ARG;
    }
  }
  DeviceCtx* ctx = nullptr;
  st = current_ctx(&ctx);
  if (st != MS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (offsets != nullptr) return to_status(cudaMemsetAsync(offsets, 0, (size_t)(m + 1) * 4, s));
    return MS_OK;
  }
  c.keys_in = keys_in;
  c.vals_in = pairs ? vals_in : nullptr;
  c.keys_out = keys_out;
  c.vals_out = pairs ? vals_out : nullptr;
  c.offsets = offsets;
  c.n = (uint32_t)n;
  c.stream = s;
  return to_status(wide ? run_wide(c, w, *ctx) : run_multisplit(c, *ctx));
}

}  // namespace ms

using namespace ms;

extern "C" ms_status ms_multisplit_keys(const uint32_t* keys_in, size_t n, const ms_bucket_spec* spec,
                                        uint32_t* keys_out, uint32_t* offsets, void* stream) {
  return multisplit_impl(keys_in, nullptr, n, spec, keys_out, nullptr, offsets, stream, false);
}

extern "C" ms_status ms_multisplit_pairs(const uint32_t* keys_in, const uint32_t* vals_in, size_t n,
                                         const ms_bucket_spec* spec, uint32_t* keys_out, uint32_t* vals_out,
                                         uint32_t* offsets, void* stream) {
  return multisplit_impl(keys_in, vals_in, n, spec, keys_out, vals_out, offsets, stream, true);
}

// Section 7.3: the device histogram is the multisplit's pre-scan alone --
// per-chunk bucket counts and their scan -- with the bucket sizes as result.
extern "C" ms_status ms_histogram(const uint32_t* keys, size_t n, const ms_bucket_spec* spec, uint32_t* counts,
                                  void* stream) {
  Call c;
  std::memset(&c, 0, sizeof c);
  ms_status st = make_devspec(spec, &c.sp, &c.kind);
  if (st != MS_OK) return st;
  if (n >= ((size_t)1 << 32) || counts == nullptr || (n > 0 && keys == nullptr)) return MS_ERR_INVALID_ARG;
  DeviceCtx* ctx = nullptr;
  st = current_ctx(&ctx);
  if (st != MS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) return to_status(cudaMemsetAsync(counts, 0, (size_t)c.sp.m * 4, s));
  c.keys_in = keys;
  c.counts = counts;
  c.n = (uint32_t)n;
  c.stream = s;
  return to_status(run_multisplit(c, *ctx));
}

// Section 7.1: LSD passes of multisplit with the radix-digit identifier
// f_k(u) = (u >> (begin + rk)) & (2^r - 1), r bits except for a shorter last
// digit.  Each pass is a stable multisplit, so the composition is the stable
// sort by bits [begin_bit, end_bit).  Buffers ping-pong between keys_out and a
// pool buffer so that the last pass lands in keys_out.
static cudaError_t sort_by_multisplit_passes(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t n,
                                             int begin_bit, int end_bit, int r, uint32_t* keys_out,
                                             uint32_t* vals_out, cudaStream_t s, DeviceCtx& ctx) {
  const bool pairs = vals_in != nullptr;
  const size_t bytes = (size_t)n * sizeof(uint32_t);
  const int width = end_bit - begin_bit;
  const int passes = (width + r - 1) / r;
  void* tmp = nullptr;
  uint32_t* tmp_k = nullptr;
  uint32_t* tmp_v = nullptr;
  if (passes > 1) {
    const size_t arr = (bytes + 255) & ~(size_t)255;  // keeps the value array 256-byte aligned
    cudaError_t e = scratch_alloc(ctx, &tmp, arr * (pairs ? 2 : 1), s);
    if (e != cudaSuccess) return e;
    tmp_k = static_cast<uint32_t*>(tmp);
    tmp_v = pairs ? reinterpret_cast<uint32_t*>(static_cast<char*>(tmp) + arr) : nullptr;
  }
  const uint32_t* src_k = keys_in;
  const uint32_t* src_v = vals_in;
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < passes && e == cudaSuccess; ++p) {
    const int shift = begin_bit + r * p;
    const int bits = (end_bit - shift) < r ? (end_bit - shift) : r;
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    uint32_t* dst_k = to_out ? keys_out : tmp_k;
    uint32_t* dst_v = to_out ? vals_out : tmp_v;
    Call c;
    std::memset(&c, 0, sizeof c);
    c.kind = kRadix;
    c.sp.m = 1u << bits;
    c.sp.nbits = (uint32_t)bits;
    c.sp.m_pad = c.sp.m <= 32 ? 32u : c.sp.m;
    c.sp.lut_bits = 10u;
    c.sp.shift = (uint32_t)shift;
    c.sp.mask = (1u << bits) - 1u;
    c.keys_in = src_k;
    c.vals_in = pairs ? src_v : nullptr;
    c.keys_out = dst_k;
    c.vals_out = pairs ? dst_v : nullptr;
    c.offsets = nullptr;
    c.n = n;
    c.stream = s;
    e = run_multisplit(c, ctx);
    src_k = dst_k;
    src_v = dst_v;
  }
  const cudaError_t e2 = scratch_free(tmp, s);
  return e != cudaSuccess ? e : e2;
}

// Shared argument handling of the two sorts; r = 0 picks the tuned method
// with 8-bit digits.
static ms_status radix_sort_impl(const uint32_t* keys_in, const uint32_t* vals_in, size_t n, int begin_bit,
                                 int end_bit, int r, uint32_t* keys_out, uint32_t* vals_out, void* stream) {
  if (begin_bit < 0 || end_bit > 32 || begin_bit > end_bit) return MS_ERR_INVALID_ARG;
  if (n >= ((size_t)1 << 32)) return MS_ERR_INVALID_ARG;
  const bool pairs = vals_in != nullptr || vals_out != nullptr;
  const size_t bytes = n * sizeof(uint32_t);
  if (n > 0) {
    if (keys_in == nullptr || keys_out == nullptr || overlap(keys_in, keys_out, bytes)) return MS_ERR_INVALID_ARG;
    if (pairs && (vals_in == nullptr || vals_out == nullptr || overlap(vals_in, vals_out, bytes) ||
                  overlap(vals_out, keys_out, bytes) || overlap(vals_out, keys_in, bytes) ||
                  overlap(keys_out, vals_in, bytes)))
      return MS_ERR_INVALID_ARG;
  }
  DeviceCtx* ctx = nullptr;
  ms_status st = current_ctx(&ctx);
  if (st != MS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) return MS_OK;
  const int width = end_bit - begin_bit;
  if (width == 0) {
    cudaError_t e = cudaMemcpyAsync(keys_out, keys_in, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && pairs) e = cudaMemcpyAsync(vals_out, vals_in, bytes, cudaMemcpyDeviceToDevice, s);
    return to_status(e);
  }
  if (r == 0 && n < ((size_t)1 << 30) && choose_sort_method((uint32_t)n, pairs) == 0)
    return to_status(run_onesweep_sort(keys_in, pairs ? vals_in : nullptr, (uint32_t)n, begin_bit, end_bit, keys_out,
                                       pairs ? vals_out : nullptr, s, *ctx));
  // one three-stage multisplit per digit (tuned; other digit widths; or
  // n >= 2^30, beyond the one-sweep kernels' 30-bit status counts)
  return to_status(sort_by_multisplit_passes(keys_in, pairs ? vals_in : nullptr, (uint32_t)n, begin_bit, end_bit,
                                             r == 0 ? 8 : r, keys_out, pairs ? vals_out : nullptr, s, *ctx));
}

extern "C" ms_status ms_radix_sort(const uint32_t* keys_in, const uint32_t* vals_in, size_t n, int begin_bit,
                                   int end_bit, uint32_t* keys_out, uint32_t* vals_out, void* stream) {
  return radix_sort_impl(keys_in, vals_in, n, begin_bit, end_bit, 0, keys_out, vals_out, stream);
}

// Section 6.3 / Table 8: the same sort with r-bit digits (1 <= r <= 8), each
// pass a multisplit into 2^r buckets.
extern "C" ms_status ms_radix_sort_r(const uint32_t* keys_in, const uint32_t* vals_in, size_t n, int begin_bit,
                                     int end_bit, int r, uint32_t* keys_out, uint32_t* vals_out, void* stream) {
  if (r < 1 || r > 8) return MS_ERR_INVALID_ARG;
  return radix_sort_impl(keys_in, vals_in, n, begin_bit, end_bit, r, keys_out, vals_out, stream);
}

extern "C" ms_status ms_test_expire_lookback(void* stream) {
  DeviceCtx* ctx = nullptr;
  ms_status st = current_ctx(&ctx);
  if (st != MS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // scratch: two scan tiles of data | two status words | ticket
  const size_t data_bytes = (size_t)2 * kScanTile * 4;
  void* ws = nullptr;
  cudaError_t e = scratch_alloc(*ctx, &ws, data_bytes + 16 + 16, s);
  if (e != cudaSuccess) return to_status(e);
  auto* status = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + data_bytes);
  auto* ticket = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + data_bytes + 16);
  e = cudaMemsetAsync(ws, 0, data_bytes + 16, s);
  const uint32_t one = 1;  // the only CTA takes ticket 1: its predecessor never runs
  if (e == cudaSuccess) e = cudaMemcpyAsync(ticket, &one, sizeof one, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // `one` lives on this stack frame
  if (e == cudaSuccess) {
    ScanArgs a{static_cast<uint32_t*>(ws), (uint32_t)(2 * kScanTile), 1u, nullptr, 1u, status, ticket, ctx->d_err};
    e = launch_scan_tiles(a, 1, s);
  }
  const cudaError_t e2 = scratch_free(ws, s);
  return to_status(e != cudaSuccess ? e : e2);
}

extern "C" ms_status ms_shutdown(void) {
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return MS_ERR_CUDA;
  // a caller's batch plan refers to its device's status word: refuse while one is alive
  for (int dev = 0; dev < 64; ++dev)
    if (batch_live_plans(dev) > 0) return MS_ERR_INVALID_ARG;
  for (int dev = 0; dev < 64; ++dev) batch_cache_release(dev);
  ms_status st = MS_OK;
  {
    std::lock_guard<std::mutex> lock(g_ctx_mu);
    for (int dev = 0; dev < 64; ++dev) {
      DeviceCtx& c = g_ctx[dev];
      if (c.device < 0) continue;
      if (cudaSetDevice(dev) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) st = MS_ERR_CUDA;
      if (c.d_err != nullptr && cudaFree(c.d_err) != cudaSuccess) st = MS_ERR_CUDA;
      if (c.pool != nullptr && cudaMemPoolDestroy(c.pool) != cudaSuccess) st = MS_ERR_CUDA;
      c = DeviceCtx();
    }
  }
  trace_release();
  if (cudaSetDevice(cur) != cudaSuccess) st = MS_ERR_CUDA;
  if (st != MS_OK) cudaGetLastError();
  return st;
}

extern "C" ms_status ms_device_status(void* stream) {
  DeviceCtx* ctx = nullptr;
  ms_status st = current_ctx(&ctx);
  if (st != MS_OK) return st;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MS_ERR_CUDA;
  uint32_t h = 0;
  if (cudaMemcpy(&h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return MS_ERR_CUDA;
  if (cudaMemset(ctx->d_err, 0, sizeof h) != cudaSuccess) return MS_ERR_CUDA;
  if (h & kDevErrTimeout) return MS_ERR_TIMEOUT;
  return h == 0 ? MS_OK : MS_ERR_CUDA;
}

extern "C" const char* ms_status_string(ms_status s) {
  switch (s) {
    case MS_OK: return "MS_OK";
    case MS_ERR_INVALID_ARG: return "MS_ERR_INVALID_ARG";
    case MS_ERR_UNSUPPORTED: return "MS_ERR_UNSUPPORTED";
    case MS_ERR_OUT_OF_MEMORY: return "MS_ERR_OUT_OF_MEMORY";
    case MS_ERR_CUDA: return "MS_ERR_CUDA";
    case MS_ERR_TIMEOUT: return "MS_ERR_TIMEOUT";
  }
  return "MS_ERR_UNKNOWN";
}

extern "C" const char* ms_version(void) { return "ms 0.1 (sm_103a)"; }
