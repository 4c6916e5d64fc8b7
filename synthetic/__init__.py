"""Seeded synthetic inputs for stable multisplit and the multisplit radix sort.

This module only draws inputs.  It computes no bucket identifiers, offsets or
permutations: both the CPU oracle (``oracle/``) and the CUDA path read the same
arrays from here and do their own arithmetic.

The workloads follow the paper's experimental setup (Section 6: uniformly
distributed 32-bit keys, "Key distribution"; Section 6.4: non-uniform
distributions) and the sizes of the benchmark configurations:

* uniform uint32 keys over [0, 2^32);
* range splitters: m-1 sorted, strictly increasing uniform uint32 draws;
* "skewed": a bucket index b ~ Geometric(p=0.5) on {0, 1, ...} clipped to
  m-1, then a key uniform in [s_b, s_{b+1}) with s_0 = 0 and s_m = 2^32, where
  s_1..s_{m-1} are the splitters;
* float32 keys uniform in [0, 1000): u = uint32 draw, x = float32(u >> 8) *
  2^-24 (exact), then x * 1000.0f rounded to float32 (the largest value is
  999.99993896484375 < 1000);
* Section 6.4's non-uniform workloads for delta buckets of width delta over
  [0, m*delta): a bucket slot b drawn from the binomial B(m-1, p) or from the
  "alpha-uniform" mix (a fraction alpha uniform over the m slots, the rest in
  one random slot), then a float32 key in the middle half of the slot,
  x = float32((b + u) * delta) with u uniform in [0.25, 0.75);
* values = original index (makes stability visible) or uniform uint32;
* batched segments: size = floor(2^U), U ~ Uniform(lo, hi);
* serving traces: Poisson arrivals (exponential gaps) with a request mix.

Every generator takes an explicit seed and uses numpy's PCG64 generator.
"""
from __future__ import annotations

import numpy as np

U32_RANGE = 1 << 32


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_u32(n: int, seed: int) -> np.ndarray:
    """n uint32 keys uniform over [0, 2^32)."""
    return rng(seed).integers(0, U32_RANGE, size=int(n), dtype=np.uint64).astype(np.uint32)


def uniform_u32_bits(n: int, nbits: int, seed: int) -> np.ndarray:
    """n uint32 keys whose low ``nbits`` bits are uniform and whose high bits are 0."""
    return rng(seed).integers(0, 1 << nbits, size=int(n), dtype=np.uint64).astype(np.uint32)


def index_values(n: int) -> np.ndarray:
    """value[i] = i: the original index, so stability shows in the output."""
    return np.arange(int(n), dtype=np.uint32)


def range_splitters(m: int, seed: int) -> np.ndarray:
    """m-1 strictly increasing uniform uint32 splitters (redrawn until distinct)."""
    g = rng(seed)
    if m <= 1:
        return np.zeros(0, dtype=np.uint32)
    while True:
        s = np.sort(g.integers(1, U32_RANGE, size=m - 1, dtype=np.uint64))
        if m - 1 < 2 or np.all(np.diff(s) > 0):
            return s.astype(np.uint32)


def skewed_u32(n: int, splitters: np.ndarray, seed: int, p: float = 0.5) -> np.ndarray:
    """Keys whose bucket slot b ~ Geometric(p) on {0,1,...} clipped to m-1.

    The key is then drawn uniformly inside [s_b, s_{b+1}), with s_0 = 0,
    s_m = 2^32 and s_1..s_{m-1} = ``splitters`` (strictly increasing).
    """
    g = rng(seed)
    m = len(splitters) + 1
    b = np.minimum(g.geometric(p, size=int(n)) - 1, m - 1).astype(np.int64)
    lo = np.concatenate([[0], splitters.astype(np.uint64)])
    hi = np.concatenate([splitters.astype(np.uint64), [U32_RANGE]])
    width = (hi - lo)[b]
    off = (g.random(size=int(n)) * width.astype(np.float64)).astype(np.uint64)
    off = np.minimum(off, width - 1)
    return (lo[b] + off).astype(np.uint32)


def uniform_f32_1000(n: int, seed: int) -> np.ndarray:
    """float32 keys uniform in [0, 1000), returned as their uint32 bit patterns."""
    u = uniform_u32(n, seed)
    x = (u >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24)
    x = x * np.float32(1000.0)
    return x.astype(np.float32).view(np.uint32)


def _f32_in_slots(b: np.ndarray, delta: float, g: np.random.Generator) -> np.ndarray:
    u = g.uniform(0.25, 0.75, size=b.shape[0])
    x = ((b.astype(np.float64) + u) * float(np.float32(delta))).astype(np.float32)
    return x.view(np.uint32)


def binomial_f32(n: int, m: int, delta: float, seed: int, p: float = 0.5) -> np.ndarray:
    """float32 keys (as uint32 bit patterns) whose delta-bucket slot is B(m-1, p)."""
    g = rng(seed)
    b = g.binomial(m - 1, p, size=int(n))
    return _f32_in_slots(b, delta, g)


def alpha_uniform_f32(n: int, m: int, delta: float, alpha: float, seed: int) -> np.ndarray:
    """float32 keys: a fraction alpha with a uniform slot in [0, m), the rest
    all in one random slot (Section 6.4's "alpha-uniform" distribution)."""
    g = rng(seed)
    hot = int(g.integers(0, m))
    b = np.where(g.random(size=int(n)) < alpha, g.integers(0, m, size=int(n)), hot)
    return _f32_in_slots(b, delta, g)


def segment_sizes(num: int, lo_log2: float, hi_log2: float, seed: int) -> np.ndarray:
    """Segment sizes floor(2^U), U ~ Uniform(lo_log2, hi_log2)."""
    u = rng(seed).uniform(lo_log2, hi_log2, size=int(num))
    return np.floor(np.exp2(u)).astype(np.int64)


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process over [0, duration_s)."""
    g = rng(seed)
    expected = int(rate_per_s * duration_s * 1.2) + 16
    t = np.cumsum(g.exponential(1.0 / rate_per_s, size=expected))
    while t[-1] < duration_s:
        more = np.cumsum(g.exponential(1.0 / rate_per_s, size=expected)) + t[-1]
        t = np.concatenate([t, more])
    return t[t < duration_s]
