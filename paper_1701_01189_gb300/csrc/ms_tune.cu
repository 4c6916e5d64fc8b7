// ms_tune.cu -- the variant table consulted by every multisplit: which tile
// shape, rank mode and reordering to run for (bucket kind, keys or pairs,
// ceil(log2 m), size class of n).  Defaults come from the rules below; the
// autotuner (paper_1701_01189_gb300/autotune.py) measures the candidates on the
// device and installs the fastest with ms_tune_set().
#include <algorithm>
#include <mutex>

#include "ms.h"
#include "ms_host.h"

namespace ms {

namespace {
constexpr int kKinds = 4, kNbits = 9, kClasses = 4;
std::mutex g_mu;
bool g_set[kKinds][2][kNbits][kClasses] = {};
Variant g_table[kKinds][2][kNbits][kClasses];
// radix sort passes per (pairs, size class): 0 one-sweep, 1 three-stage multisplits
bool g_sort_set[2][kClasses] = {};
int g_sort[2][kClasses];
// batched plans per (kind, pairs, ceil(log2 m), size class of the mean segment)
bool g_batch_set[kKinds][2][kNbits][kClasses] = {};
Variant g_batch[kKinds][2][kNbits][kClasses];

Variant default_batch_variant(int nbits) {
  Variant v;
  v.shape = 0;
  v.rank = nbits <= 5 ? kRankThread : kRankTable;
  v.reorder = 1;
  return v;
}

// Up to 32 buckets: per-thread bucket counters (ms_tc.cuh).  Beyond, peer
// tables with block reordering; key-value pairs prefer the smaller 8 x 8 tile
// (two arrays in flight per tile), except with 256 buckets (16 x 8).
Variant default_variant(int nbits, int pairs) {
  Variant v;
  if (nbits <= 5) {
    v.rank = kRankThread;
    v.reorder = 1;
    v.shape = 0;
  } else {
    v.rank = kRankTable;
    v.reorder = 1;
    v.shape = pairs ? (nbits >= 8 ? 1 : 2) : 0;
  }
  return v;
}
}  // namespace

int size_class(uint32_t n) {
  if (n < (1u << 16)) return 0;
  if (n < (1u << 20)) return 1;
  if (n < (1u << 24)) return 2;
  return 3;
}

int choose_sort_method(uint32_t n, bool pairs) {
  const int sc = size_class(n), p = pairs ? 1 : 0;
  std::lock_guard<std::mutex> lock(g_mu);
  return g_sort_set[p][sc] ? g_sort[p][sc] : 0;
}

Variant choose_variant(const Call& c) {
  const int nb = (int)c.sp.nbits, pairs = c.vals_in != nullptr ? 1 : 0, sc = size_class(c.n);
  std::lock_guard<std::mutex> lock(g_mu);
  if (c.kind >= 0 && c.kind < kKinds && nb < kNbits && g_set[c.kind][pairs][nb][sc]) return g_table[c.kind][pairs][nb][sc];
  return default_variant(nb, pairs);
}

Variant choose_batch_variant(int kind, bool pairs, uint32_t nbits, uint64_t mean_n) {
  const int sc = size_class((uint32_t)std::min<uint64_t>(mean_n, 0xffffffffu)), p = pairs ? 1 : 0;
  std::lock_guard<std::mutex> lock(g_mu);
  if (kind >= 0 && kind < kKinds && nbits < (uint32_t)kNbits && g_batch_set[kind][p][nbits][sc])
    return g_batch[kind][p][nbits][sc];
  return default_batch_variant((int)nbits);
}

}  // namespace ms

using namespace ms;

extern "C" ms_status ms_tune_set_batch(int kind, int pairs, int nbits, int sclass, int shape, int rank) {
  if (kind < 0 || kind >= kKinds || pairs < 0 || pairs > 1 || nbits < 0 || nbits >= kNbits || sclass < 0 ||
      sclass >= kClasses || shape < 0 || shape > 1 || !(rank == kRankTable || rank == kRankThread || rank == kRankVote))
    return MS_ERR_INVALID_ARG;
  if (rank == kRankThread && (nbits > 5 || shape != 0)) return MS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  g_batch[kind][pairs][nbits][sclass] = Variant{shape, rank, 1};
  g_batch_set[kind][pairs][nbits][sclass] = true;
  return MS_OK;
}

extern "C" ms_status ms_tune_get_batch(int kind, int pairs, int nbits, int sclass, int* shape, int* rank) {
  if (kind < 0 || kind >= kKinds || pairs < 0 || pairs > 1 || nbits < 0 || nbits >= kNbits || sclass < 0 ||
      sclass >= kClasses)
    return MS_ERR_INVALID_ARG;
  Variant v;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    v = g_batch_set[kind][pairs][nbits][sclass] ? g_batch[kind][pairs][nbits][sclass] : default_batch_variant(nbits);
  }
  if (shape) *shape = v.shape;
  if (rank) *rank = v.rank;
  return MS_OK;
}

extern "C" int ms_tune_size_class(size_t n) { return n >= ((size_t)1 << 32) ? 3 : size_class((uint32_t)n); }

extern "C" ms_status ms_tune_set(int kind, int pairs, int nbits, int sclass, int shape, int rank, int reorder) {
  if (kind < 0 || kind >= kKinds || pairs < 0 || pairs > 1 || nbits < 0 || nbits >= kNbits || sclass < 0 ||
      sclass >= kClasses || shape < 0 || shape > 2 || rank < 0 || rank > 3 || reorder < 0 || reorder > 1)
    return MS_ERR_INVALID_ARG;
  if ((rank == kRankBallot || rank == kRankThread) && nbits > 5) return MS_ERR_INVALID_ARG;
  if (reorder == 0 && (rank != kRankBallot || nbits > 3)) return MS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  g_table[kind][pairs][nbits][sclass] = Variant{shape, rank, reorder};
  g_set[kind][pairs][nbits][sclass] = true;
  return MS_OK;
}

extern "C" ms_status ms_tune_get(int kind, int pairs, int nbits, int sclass, int* shape, int* rank, int* reorder) {
  if (kind < 0 || kind >= kKinds || pairs < 0 || pairs > 1 || nbits < 0 || nbits >= kNbits || sclass < 0 ||
      sclass >= kClasses)
    return MS_ERR_INVALID_ARG;
  Variant v;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    v = g_set[kind][pairs][nbits][sclass] ? g_table[kind][pairs][nbits][sclass] : default_variant(nbits, pairs);
  }
  if (shape) *shape = v.shape;
  if (rank) *rank = v.rank;
  if (reorder) *reorder = v.reorder;
  return MS_OK;
}

extern "C" ms_status ms_tune_reset(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto& a : g_set)
    for (auto& b : a)
      for (auto& c : b)
        for (auto& d : c) d = false;
  for (auto& a : g_sort_set)
    for (auto& b : a) b = false;
  for (auto& a : g_batch_set)
    for (auto& b : a)
      for (auto& c : b)
        for (auto& d : c) d = false;
  return MS_OK;
}

extern "C" ms_status ms_tune_set_sort(int pairs, int sclass, int method) {
  if (pairs < 0 || pairs > 1 || sclass < 0 || sclass >= kClasses || method < 0 || method > 1)
    return MS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  g_sort[pairs][sclass] = method;
  g_sort_set[pairs][sclass] = true;
  return MS_OK;
}

extern "C" ms_status ms_tune_get_sort(int pairs, int sclass, int* method) {
  if (pairs < 0 || pairs > 1 || sclass < 0 || sclass >= kClasses) return MS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (method) *method = g_sort_set[pairs][sclass] ? g_sort[pairs][sclass] : 0;
  return MS_OK;
}
