// ms_wide.cu -- multisplit into more than 256 buckets (Section 6.3, "Solutions
// for larger multisplits").
//
// The paper iterates multisplit over super-buckets of at most 256 buckets,
// most significant group first, which restricts it to identifiers whose
// adjacent bucket ids cover adjacent key ranges.  Here the iteration runs over the
// 8-bit digits of the bucket id b = f(u), least significant digit first: pass
// 0 is a stable multisplit by b mod 256, pass 1 a stable multisplit by
// floor(b / 256).  Each pass is stable, so the pair of passes orders the
// elements by b and keeps the input order inside each bucket: the stable
// multisplit by b (Eq. 1), for any identifier the kernels can evaluate (also
// key mod m, which the super-bucket scheme cannot split).  Every pass is the
// three-stage multisplit of the m <= 256 path; the bucket offsets come from
// the last pass's offsets (one per super-bucket) refined by a bisection per
// bucket over the output, which is ordered by bucket.
#include <cmath>
#include <cstring>

#include "ms_run.cuh"

namespace ms {

// One pass: the multisplit of the kernel identifier kWide (a digit of the
// wide identifier), with the tuned variant of the base identifier: per-thread
// counters up to 32 buckets, peer tables beyond.
static cudaError_t run_wide_pass(const Call& c, DeviceCtx& ctx) {
  Call q = c;
  q.kind = (int)c.sp.base;
  const Variant v = choose_variant(q);
  if (c.sp.m <= kTcMaxM && (v.rank == kRankThread || v.rank == kRankBallot)) return run_tc<kWide>(c, ctx, v.shape);
  return run_ms_pairs<kWide, 8, kRankTable, 1>(c, ctx, v.shape);
}

static cudaError_t run_pass(const Call& c, DeviceCtx& ctx) {
  return c.kind == kWide ? run_wide_pass(c, ctx) : run_multisplit(c, ctx);
}

// offsets[j] for j < fm: the first output position whose bucket is >= j.
// Bucket j lies in super-bucket j >> 8, whose run in the output is
// [coff[j >> 8], coff[(j >> 8) + 1]) (the last pass's offsets); the search
// stays inside it.  offsets[fm] = n.  One thread per entry.
template <int KIND>
__global__ void __launch_bounds__(256) k_wide_offsets(const uint32_t* out, uint32_t n, DevSpec sp, uint32_t fm,
                                                      const uint32_t* coff, uint32_t* offsets) {
  __shared__ uint32_t s_tbl[256];
  if constexpr (KIND == kWide) build_wide_table<8>(sp, s_tbl);
  __syncthreads();
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > fm) return;
  if (j == fm) {
    offsets[j] = n;
    return;
  }
  uint32_t lo = coff[j >> 8], hi = coff[(j >> 8) + 1];
  if ((j & 255u) != 0u) {
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if (bucket_of<KIND, 8>(out[mid], sp, s_tbl, nullptr) < j)
        lo = mid + 1u;
      else
        hi = mid;
    }
  }
  offsets[j] = lo;
}

// Number of the fm - 1 splitters <= x (bisection in global memory).
__device__ __forceinline__ uint32_t count_le(const uint32_t* s, uint32_t cnt, uint32_t x) {
  uint32_t lo = 0, hi = cnt;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(s + mid) <= x)
      lo = mid + 1u;
    else
      hi = mid;
  }
  return lo;
}

// The global lookup table of a wide range identifier (layout beside
// kWideLutFlag in ms_bucket.cuh): cell c covers keys [c << (32 - wlb),
// ((c + 1) << (32 - wlb)) - 1]; lo = splitters below its first key, hi =
// splitters up to its last key; the keys of the cell have buckets lo .. hi.
__global__ void __launch_bounds__(256) k_wide_lut(const uint32_t* splitters, uint32_t fm, uint32_t wlb,
                                                  uint32_t* lut) {
  const uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= (1u << wlb)) return;
  const uint32_t sh = 32u - wlb, fmask = (1u << sh) - 1u;
  const uint32_t first = cell << sh, last = first | fmask;
  const uint32_t lo = first == 0u ? 0u : count_le(splitters, fm - 1u, first - 1u);
  const uint32_t hi = count_le(splitters, fm - 1u, last);
  uint32_t e;
  if (hi == lo)
    e = lo | ((fmask + 1u) << 17);
  else if (hi == lo + 1u)
    e = lo | ((__ldg(splitters + lo) & fmask) << 17);
  else
    e = lo | kWideLutFlag | (min(hi - lo, 255u) << 17);
  lut[cell] = e;
}

static uint32_t log2_ceil(uint32_t m) {
  uint32_t l = 0;
  while ((1u << l) < m) ++l;
  return l;
}

// Kernel spec of a digit pass of a wide identifier (kWide) with m buckets.
static DevSpec wide_pass_spec(const WideSpec& w, uint32_t dshift, uint32_t m) {
  DevSpec d = w.full;
  d.m = m;
  d.nbits = log2_ceil(m);
  d.m_pad = m <= 32 ? 32u : ((m + 31u) & ~31u);
  d.lut_bits = m <= 64 ? 10u : 11u;
  d.dshift = dshift;
  d.dmask = 255u;
  return d;
}

ms_status make_wide_spec(const ms_bucket_spec* spec, WideSpec* out) {
  if (spec == nullptr) return MS_ERR_INVALID_ARG;
  const uint32_t m = spec->m;
  if (m <= (uint32_t)kMaxM || m > kMaxWideM) return MS_ERR_INVALID_ARG;
  WideSpec w;
  std::memset(&w, 0, sizeof w);
  w.fm = m;
  w.mc = (m + 255u) >> 8;
  DevSpec& d = w.full;
  d.fm = m;
  d.mc = w.mc;
  d.dshift = 0;
  d.dmask = 0xffffffffu;
  d.m = m;
  switch (spec->kind) {
    case MS_BUCKET_RANGE_U32:
      if (spec->splitters == nullptr) return MS_ERR_INVALID_ARG;
      d.splitters = spec->splitters;
      d.base = kRange;
      w.kind = kWide;
      break;
    case MS_BUCKET_DELTA_F32:
      if (!std::isfinite(spec->x0) || !std::isfinite(spec->delta) || !(spec->delta > 0.0f)) return MS_ERR_INVALID_ARG;
      d.x0 = spec->x0;
      d.delta = spec->delta;
      d.rdelta = 1.0f / spec->delta;
      d.base = kDelta;
      w.kind = kWide;
      break;
    case MS_BUCKET_MOD: {
      // Granlund-Montgomery constants for unsigned division by fm (as for
      // m <= 256): l = ceil(log2 fm), M = floor(2^32 (2^l - fm) / fm) + 1.
      const uint32_t l = log2_ceil(m);
      d.mod_magic = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << l) - m)) / m + 1);
      d.mod_sh1 = 1u;
      d.mod_sh2 = l - 1u;
      d.base = kMod;
      w.kind = kWide;
      break;
    }
    case MS_BUCKET_RADIX:
      // bits 9..16: the two digits are plain radix digits of the key
      if (spec->bits > 16 || m != (1u << spec->bits) || spec->shift + spec->bits > 32) return MS_ERR_INVALID_ARG;
      d.shift = spec->shift;
      d.mask = m - 1u;
      w.kind = kRadix;
      break;
    default:
      return MS_ERR_INVALID_ARG;
  }
  *out = w;
  return MS_OK;
}

// The two passes and the offsets.  c carries the request (keys, values,
// outputs, offsets, n > 0, stream); its spec fields are unused.
cudaError_t run_wide(const Call& c, const WideSpec& w, DeviceCtx& ctx) {
  const bool pairs = c.vals_in != nullptr;
  const size_t arr = (((size_t)c.n * 4) + 255) & ~(size_t)255;  // 256-byte aligned arrays
  const size_t coff_bytes = (((size_t)w.mc + 1) * 4 + 15) & ~(size_t)15;
  // range: a cell per 16 buckets or more (few cells hold two splitters), 2^18 .. 2^20 cells
  const uint32_t wlb = std::min(20u, std::max(18u, log2_ceil(w.fm) + 4u));
  const size_t lut_bytes = w.full.base == kRange && w.kind == kWide ? ((size_t)4 << wlb) : 0;
  const size_t mc_bytes = ((size_t)w.mc * 4 + 15) & ~(size_t)15;
  const size_t bytes = arr * (pairs ? 2 : 1) + coff_bytes + mc_bytes + lut_bytes;
  void* ws = nullptr;
  cudaError_t e = scratch_alloc(ctx, &ws, bytes, c.stream);
  if (e != cudaSuccess) return e;
  char* base = static_cast<char*>(ws);
  uint32_t* tmp_k = reinterpret_cast<uint32_t*>(base);
  uint32_t* tmp_v = pairs ? reinterpret_cast<uint32_t*>(base + arr) : nullptr;
  uint32_t* coff = reinterpret_cast<uint32_t*>(base + arr * (pairs ? 2 : 1));
  uint32_t* coarse = reinterpret_cast<uint32_t*>(base + arr * (pairs ? 2 : 1) + coff_bytes);
  uint32_t* wlut = reinterpret_cast<uint32_t*>(base + arr * (pairs ? 2 : 1) + coff_bytes + mc_bytes);
  WideSpec wf = w;  // the full spec with the lookup table in place (range)
  if (lut_bytes) {
    wf.full.wlut = wlut;
    wf.full.wlb = wlb;
    k_wide_lut<<<(1u << wlb) / 256u, 256, 0, c.stream>>>(w.full.splitters, w.fm, wlb, wlut);
    e = cudaGetLastError();
  }

  Call p0 = c, p1 = c;
  p0.keys_out = tmp_k;
  p0.vals_out = tmp_v;
  p0.offsets = nullptr;
  p1.keys_in = tmp_k;
  p1.vals_in = tmp_v;
  p1.offsets = coff;
  p0.kind = p1.kind = w.kind;
  if (w.kind == kRadix) {
    ms_bucket_spec s0{MS_BUCKET_RADIX, 256u, nullptr, 0.f, 0.f, w.full.shift, 8u};
    ms_bucket_spec s1{MS_BUCKET_RADIX, w.mc, nullptr, 0.f, 0.f, w.full.shift + 8u, log2_ceil(w.mc)};
    int k0 = 0, k1 = 0;
    if (make_devspec(&s0, &p0.sp, &k0) != MS_OK || make_devspec(&s1, &p1.sp, &k1) != MS_OK) {
      scratch_free(ws, c.stream);
      return cudaErrorInvalidValue;
    }
  } else {
    p0.sp = wide_pass_spec(wf, 0u, 256u);
    if (w.full.base == kRange) {
      // the top digit of a range identifier is the range identifier over the
      // super-bucket splitters s_256, s_512, ... (every 256th splitter)
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(coarse, 4, w.full.splitters + 255, 1024, 4, w.mc - 1u, cudaMemcpyDeviceToDevice,
                              c.stream);
      ms_bucket_spec s1{MS_BUCKET_RANGE_U32, w.mc, coarse, 0.f, 0.f, 0u, 0u};
      int k1 = 0;
      if (make_devspec(&s1, &p1.sp, &k1) != MS_OK) e = cudaErrorInvalidValue;
      p1.kind = kRange;
    } else {
      p1.sp = wide_pass_spec(wf, 8u, w.mc);
    }
  }
  if (e == cudaSuccess) e = run_pass(p0, ctx);
  if (e == cudaSuccess) e = run_pass(p1, ctx);
  if (e == cudaSuccess && c.offsets != nullptr) {
    const uint32_t blocks = (w.fm + 1u + 255u) / 256u;
    if (w.kind == kRadix)
      k_wide_offsets<kRadix><<<blocks, 256, 0, c.stream>>>(c.keys_out, c.n, w.full, w.fm, coff, c.offsets);
    else
      k_wide_offsets<kWide><<<blocks, 256, 0, c.stream>>>(c.keys_out, c.n, wf.full, w.fm, coff, c.offsets);
    e = cudaGetLastError();
  }
  const cudaError_t e2 = scratch_free(ws, c.stream);
  return e != cudaSuccess ? e : e2;
}

}  // namespace ms
