/*
 * ms_oracle.c -- plain, slow, single-threaded CPU oracle for stable multisplit.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this file.  The product path (the CUDA library)
 * shares no code, header, table or helper with it.
 *
 * What it computes, from "GPU Multisplit" (Ashkiani et al.):
 *   - Section 3.1: a multisplit permutes n keys (or key-value pairs) so that the
 *     m buckets are contiguous and in ascending bucket-ID order; "stable" keeps
 *     the input order inside each bucket.  The optional bucket-start array is
 *     emitted with m+1 entries (offsets[m] = n).
 *   - Eq. 1 (Section 4.2): p(i) = sum_{k<j} h_k + |{u_r in B_j : r < i}|.
 *     The oracle evaluates that definition literally: a histogram h, its
 *     exclusive prefix sum (global offsets), then one ascending pass over the
 *     input keeping the running count of each bucket (local offsets).
 *   - Bucket identifiers: Section 6 "Bucket identification" (delta buckets,
 *     identity buckets, range splitters) and Section 7.1 (the radix digit
 *     f_k(u) = (u >> kr) & (2^r - 1)); key mod m as a general identifier.
 *
 * Readings where the paper is silent or garbled (each is listed in the design
 * notes of the repository):
 *   - range buckets take m-1 nondecreasing splitters s_1..s_{m-1}; the bucket is
 *     the number of splitters <= u (an upper bound), so u < s_1 -> 0 and
 *     u >= s_{m-1} -> m-1;
 *   - float32 delta buckets: q = (x - x0) / delta in binary32 round-to-nearest,
 *     b = floor(q); b <= 0 (also -0, -inf) -> 0, b >= m (also +inf) -> m-1,
 *     NaN -> m-1;
 *   - m = 1 is a plain copy with offsets [0, n].
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * ORACLE_MUTANT=k (test builds only) plants one deliberate mistake so the
 * tests can show that their pins catch it; a normal build defines nothing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUT(k) (ORACLE_MUTANT == (k))

enum { ORACLE_RANGE_U32 = 0, ORACLE_DELTA_F32 = 1, ORACLE_RADIX = 2, ORACLE_MOD = 3 };

/* Bucket identifier parameters, as plain scalars (no shared struct with the
 * CUDA library). */
typedef struct {
  int32_t kind;
  uint32_t m;
  const uint32_t *splitters; /* RANGE: m-1 nondecreasing values, host memory */
  float x0, delta;           /* DELTA_F32 */
  uint32_t shift, bits;      /* RADIX */
} oracle_spec;

/* Range buckets: number of splitters <= u.  Because the splitters are sorted,
 * that count is the upper-bound position, found by bisection. */
static uint32_t bucket_range(uint32_t u, const uint32_t *s, uint32_t m) {
  uint32_t lo = 0, hi = m - 1; /* answer lies in [lo, hi] */
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2; /* candidate: s[mid] <= u ? */
    if (MUT(6) ? (s[mid] < u) : (s[mid] <= u))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

/* Delta buckets on float32 keys (Section 6 and Section 7.3's even histogram:
 * floor((x - s_0) / delta)), clamped into [0, m-1]. */
static uint32_t bucket_delta(uint32_t bits, float x0, float delta, uint32_t m) {
  float x;
  memcpy(&x, &bits, sizeof x);
  float q = (x - x0) / delta;
  if (isnan(q)) return m - 1;
  float f = floorf(q);
  if (MUT(7)) f = roundf(q);
  if (f <= 0.0f) return 0;
  if (f >= (float)m) return m - 1;
  return (uint32_t)f;
}

static uint32_t bucket_of(uint32_t u, const oracle_spec *sp) {
  switch (sp->kind) {
    case ORACLE_RANGE_U32:
      return bucket_range(u, sp->splitters, sp->m);
    case ORACLE_DELTA_F32:
      return bucket_delta(u, sp->x0, sp->delta, sp->m);
    case ORACLE_RADIX: {
      uint32_t shift = MUT(8) ? sp->shift + 1 : sp->shift;
      uint32_t mask = (sp->bits >= 32) ? 0xffffffffu : ((1u << sp->bits) - 1u);
      return (shift >= 32) ? 0u : ((u >> shift) & mask);
    }
    case ORACLE_MOD:
      return MUT(9) ? (u & (sp->m - 1u)) : (u % sp->m);
  }
  return 0;
}

/* Bucket ID of every key (the vector f(u)). */
void oracle_bucket_ids(const uint32_t *keys, size_t n, const oracle_spec *sp, uint32_t *ids) {
  for (size_t i = 0; i < n; ++i) ids[i] = bucket_of(keys[i], sp);
}

/* Histogram h_j = |{i : f(u_i) = j}| (Section 7.3's device histogram output). */
void oracle_histogram(const uint32_t *keys, size_t n, const oracle_spec *sp, uint64_t *h) {
  for (uint32_t j = 0; j < sp->m; ++j) h[j] = 0;
  for (size_t i = 0; i < n; ++i) h[bucket_of(keys[i], sp)] += 1;
}

/* Stable multisplit by Eq. 1.  vals / vals_out may be NULL (keys only).
 * offsets has m+1 entries.  Returns 0, or -1 if scratch allocation fails. */
int oracle_multisplit(const uint32_t *keys, const uint32_t *vals, size_t n, const oracle_spec *sp,
                      uint32_t *keys_out, uint32_t *vals_out, uint64_t *offsets) {
  const uint32_t m = sp->m;
  uint32_t *ids = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  uint64_t *h = (uint64_t *)calloc(m, sizeof(uint64_t));
  uint64_t *cur = (uint64_t *)calloc(m, sizeof(uint64_t));
  if (!ids || !h || !cur) {
    free(ids);
    free(h);
    free(cur);
    return -1;
  }
  /* bucket of every key, and the histogram h */
  for (size_t i = 0; i < n; ++i) {
    ids[i] = bucket_of(keys[i], sp);
    h[ids[i]] += 1;
  }
  /* global offsets: exclusive prefix sum of h (first term of Eq. 1) */
  offsets[0] = 0;
  for (uint32_t j = 0; j < m; ++j) offsets[j + 1] = offsets[j] + ((MUT(1) && j == 0) ? 0 : h[j]);
  if (MUT(5)) { /* buckets laid out in descending ID order */
    uint64_t acc = 0;
    for (uint32_t j = m; j-- > 0;) {
      offsets[j] = acc;
      acc += h[j];
    }
    offsets[m] = acc;
  }
  /* local offsets: elements r < i of the same bucket placed before element i
   * (second term of Eq. 1), kept as a running count per bucket */
  for (uint32_t j = 0; j < m; ++j) cur[j] = offsets[j] + (MUT(2) ? 1 : 0);
  if (MUT(3)) { /* unstable: later elements first inside each bucket */
    for (size_t r = n; r-- > 0;) {
      uint64_t p = cur[ids[r]]++;
      keys_out[p] = keys[r];
      if (vals && vals_out) vals_out[p] = vals[r];
    }
  } else {
    for (size_t i = 0; i < n; ++i) {
      uint64_t p = cur[ids[i]]++;
      if (p >= n) p = n - 1; /* only reachable in mutant 2 */
      keys_out[p] = keys[i];
      if (vals && vals_out) vals_out[p] = MUT(4) ? keys[i] : vals[i];
    }
  }
  free(ids);
  free(h);
  free(cur);
  return 0;
}

/* Eq. 1 directly for one element: p(i) for the element at index i.  Used to
 * check sampled outputs of large runs one element at a time.  h must be the
 * histogram of the whole input (from oracle_histogram). */
uint64_t oracle_position(const uint32_t *keys, size_t n, const oracle_spec *sp, const uint64_t *h,
                         size_t i) {
  uint32_t j = bucket_of(keys[i], sp);
  uint64_t p = 0;
  for (uint32_t k = 0; k < j; ++k) p += h[k];
  for (size_t r = 0; r < i && r < n; ++r)
    if (bucket_of(keys[r], sp) == j) p += 1;
  return p;
}
