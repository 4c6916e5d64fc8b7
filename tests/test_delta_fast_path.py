"""Host check of the rounding argument behind the delta-bucket fast path.

The kernels compute a float32 delta bucket floor((x - x0) / delta) (IEEE
round-to-nearest subtraction and division, Section 6 delta buckets) without
the division for most keys: q' = (x - x0) * r with r = 1/delta rounded once,
and floor(q') is taken when q' lies more than q' 2^-22 away from every integer
and inside (0, m); every other key takes the division.  The argument: q' is
the exact quotient times (1 + e1)(1 + e2) with |e1|, |e2| <= 2^-24, so it lies
within 3.01 q' 2^-24 of the rounded quotient.  This test replays that decision
rule in numpy float32 arithmetic (IEEE, round-to-nearest) on keys drawn near
bucket edges, where it matters, and checks that whenever the rule takes the
fast path its floor equals the floor of the rounded quotient.  It checks the
arithmetic, not the kernels (the GPU parity tests do that).
"""
import numpy as np

import synthetic


def _fast_path(d, r, m):
    f32 = np.float32
    qa = (d * r).astype(f32)
    k = np.floor(qa).astype(f32)
    fr = (qa - k).astype(f32)
    eps = (qa * f32(2.0 ** -22)).astype(f32)
    take = (qa > 0) & (qa < f32(m)) & (fr > eps) & ((f32(1.0) - fr).astype(f32) > eps)
    return take, k


def _rounded_floor(d, delta):
    return np.floor((d / delta).astype(np.float32))


def test_fast_path_floor_equals_division_floor():
    g = synthetic.rng(2024)
    f32 = np.float32
    taken = 0
    for trial in range(40):
        m = int(g.choice([2, 3, 7, 8, 32, 100, 256, 1000, 65536]))
        delta = f32(g.uniform(1e-3, 1e3)) / f32(m)
        x0 = f32(g.uniform(-100.0, 100.0)) if trial % 2 else f32(0.0)
        r = (f32(1.0) / delta).astype(f32)
        # keys on and next to every reachable bucket edge, and uniform ones
        kk = g.integers(0, m + 1, size=20000).astype(np.float64)
        edge = (x0 + (kk * float(delta))).astype(f32)
        ulps = g.integers(-6, 7, size=edge.size).astype(np.int64)
        bits = edge.view(np.int32).astype(np.int64) + ulps * np.where(edge >= 0, 1, -1)
        near = bits.astype(np.int32).view(f32)
        uni = (x0 + g.uniform(0.0, 1.0, size=20000) * float(delta) * m).astype(f32)
        x = np.concatenate([near, uni]).astype(f32)
        x = x[np.isfinite(x)]
        d = (x - x0).astype(f32)
        take, k = _fast_path(d, r, m)
        exact = _rounded_floor(d[take], delta)
        np.testing.assert_array_equal(k[take], exact, err_msg=f"m={m} delta={delta} x0={x0}")
        taken += int(take.sum())
    assert taken > 100_000  # the fast path is the common case


def test_margin_is_needed():
    """Without the edge margin the product's floor can differ from the
    division's: some key just below an edge rounds up in one and not the other."""
    f32 = np.float32
    found = False
    for m in (3, 7, 100, 1000):
        delta = f32(1000.0) / f32(m)
        r = (f32(1.0) / delta).astype(f32)
        edge = (np.arange(1, m, dtype=np.float64) * float(delta)).astype(f32)
        for s in range(-3, 4):
            x = (edge.view(np.int32) + s).view(f32)
            qa = (x * r).astype(f32)
            if np.any(np.floor(qa) != _rounded_floor(x, delta)):
                found = True
    assert found
