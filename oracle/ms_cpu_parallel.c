/*
 * ms_cpu_parallel.c -- the all-core CPU baseline of stable multisplit.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the oracle beside it: only
 * tests/ and the benchmark's CPU-baseline leg load it.  It is not the oracle
 * (ms_oracle.c is); it is the host-side comparison point the benchmark times on
 * every host core, and a test checks it bit for bit against the oracle.  It
 * shares no code with the CUDA library, nor with ms_oracle.c.
 *
 * Method: the paper's localisation (Section 4.4) with one subproblem per
 * thread chunk, on the CPU:
 *   1. the input is cut into T contiguous chunks (T = threads); each thread
 *      computes the bucket of each of its keys and its chunk's histogram
 *      h[c][b];
 *   2. one exclusive scan over the histograms in bucket-major order (Eq. 2:
 *      the start of bucket b in chunk c is the total of all buckets below b
 *      plus bucket b's count in the chunks before c);
 *   3. each thread scatters its chunk in input order from those starts, so
 *      the result is stable (Eq. 1).
 * Threads are POSIX threads (no OpenMP runtime needed on the host).
 *
 * Build: gcc -O3 -std=c11 -ffp-contract=off -fno-fast-math -pthread -shared -fPIC.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { PAR_RANGE_U32 = 0, PAR_DELTA_F32 = 1, PAR_RADIX = 2, PAR_MOD = 3 };

typedef struct {
  int32_t kind;
  uint32_t m;
  const uint32_t *splitters; /* RANGE: m-1 nondecreasing values */
  float x0, delta;           /* DELTA_F32 */
  uint32_t shift, bits;      /* RADIX */
} par_spec;

/* number of splitters <= u (the splitters are sorted: count them by halving
 * the candidate range) */
static inline uint32_t par_range(uint32_t u, const uint32_t *s, uint32_t nspl) {
  uint32_t base = 0, len = nspl;
  while (len > 0) {
    uint32_t half = len >> 1;
    if (s[base + half] <= u) {
      base += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return base;
}

static inline uint32_t par_bucket(uint32_t u, const par_spec *sp) {
  switch (sp->kind) {
    case PAR_RANGE_U32:
      return par_range(u, sp->splitters, sp->m - 1);
    case PAR_DELTA_F32: {
      float x;
      memcpy(&x, &u, sizeof x);
      const float q = (x - sp->x0) / sp->delta;
      if (q != q) return sp->m - 1; /* NaN */
      const float f = floorf(q);
      if (f <= 0.0f) return 0;
      return f >= (float)sp->m ? sp->m - 1 : (uint32_t)f;
    }
    case PAR_RADIX:
      if (sp->bits == 0 || sp->shift >= 32) return 0;
      return (u >> sp->shift) & (sp->bits >= 32 ? 0xffffffffu : ((1u << sp->bits) - 1u));
    default:
      return u % sp->m;
  }
}

typedef struct {
  const uint32_t *keys, *vals;
  uint32_t *keys_out, *vals_out;
  const par_spec *sp;
  size_t lo, hi;
  uint8_t *bkt8;    /* bucket of each key (m <= 256) */
  uint64_t *hist;   /* this chunk's m counts, then its m starts */
} par_task;

static void *par_count(void *arg) {
  par_task *t = (par_task *)arg;
  const uint32_t m = t->sp->m;
  memset(t->hist, 0, m * sizeof(uint64_t));
  for (size_t i = t->lo; i < t->hi; ++i) {
    const uint32_t b = par_bucket(t->keys[i], t->sp);
    t->bkt8[i] = (uint8_t)b;
    t->hist[b] += 1;
  }
  return NULL;
}

static void *par_scatter(void *arg) {
  par_task *t = (par_task *)arg;
  uint64_t *cur = t->hist; /* the starts, advanced in place */
  for (size_t i = t->lo; i < t->hi; ++i) {
    const uint64_t p = cur[t->bkt8[i]]++;
    t->keys_out[p] = t->keys[i];
    if (t->vals) t->vals_out[p] = t->vals[i];
  }
  return NULL;
}

/* Runs fn on every task: tasks 1.. on their own threads, task 0 on the
 * caller's; joins every thread it started.  A task whose thread cannot be
 * started runs on the caller's thread, so the phase is always complete. */
static void run_phase(void *(*fn)(void *), par_task *tasks, pthread_t *tid, int threads) {
  int started[256];
  for (int c = 1; c < threads; ++c) started[c] = pthread_create(&tid[c], NULL, fn, &tasks[c]) == 0;
  fn(&tasks[0]);
  for (int c = 1; c < threads; ++c) {
    if (started[c])
      pthread_join(tid[c], NULL);
    else
      fn(&tasks[c]);
  }
}

/* Stable multisplit on `threads` threads, m <= 256.  vals / vals_out may be
 * NULL.  offsets: m+1 entries.  threads is capped at 256 and at one per 4096
 * keys.  Returns 0, -1 if an allocation fails, -2 for m outside 1..256. */
int par_multisplit(const uint32_t *keys, const uint32_t *vals, size_t n, const par_spec *sp, uint32_t *keys_out,
                   uint32_t *vals_out, uint64_t *offsets, int threads) {
  const uint32_t m = sp->m;
  if (m < 1 || m > 256) return -2;
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  if ((size_t)threads > n / 4096 + 1) threads = (int)(n / 4096 + 1); /* at least 4096 keys a chunk */
  uint8_t *bkt8 = (uint8_t *)malloc(n ? n : 1);
  uint64_t *hist = (uint64_t *)malloc((size_t)threads * m * sizeof(uint64_t));
  par_task *tasks = (par_task *)malloc((size_t)threads * sizeof(par_task));
  pthread_t *tid = (pthread_t *)malloc((size_t)threads * sizeof(pthread_t));
  int rc = 0;
  if (!bkt8 || !hist || !tasks || !tid) rc = -1;
  for (int c = 0; rc == 0 && c < threads; ++c) {
    par_task *t = &tasks[c];
    t->keys = keys;
    t->vals = vals;
    t->keys_out = keys_out;
    t->vals_out = vals_out;
    t->sp = sp;
    t->lo = n * (size_t)c / (size_t)threads;
    t->hi = n * (size_t)(c + 1) / (size_t)threads;
    t->bkt8 = bkt8;
    t->hist = hist + (size_t)c * m;
  }
  /* 1. chunk histograms */
  if (rc == 0) run_phase(par_count, tasks, tid, threads);
  /* 2. bucket-major exclusive scan: starts of (bucket b, chunk c) */
  if (rc == 0) {
    uint64_t run = 0;
    for (uint32_t b = 0; b < m; ++b) {
      offsets[b] = run;
      for (int c = 0; c < threads; ++c) {
        const uint64_t h = hist[(size_t)c * m + b];
        hist[(size_t)c * m + b] = run;
        run += h;
      }
    }
    offsets[m] = run;
  }
  /* 3. stable scatter per chunk */
  if (rc == 0) run_phase(par_scatter, tasks, tid, threads);
  free(bkt8);
  free(hist);
  free(tasks);
  free(tid);
  return rc;
}
