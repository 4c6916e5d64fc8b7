"""Host logic of the serving loop: the ring arena never hands out overlapping
live ranges, never exceeds its size, and returns space as allocations are
freed (checked against an explicit occupancy map); the trace generator."""
import numpy as np

import synthetic
from paper_1701_01189_gb300.serving import RingArena, make_trace


def test_ring_arena_against_occupancy_map():
    g = synthetic.rng(3)
    size = 1000
    ring = RingArena(size)
    owner = np.zeros(size, dtype=np.int64)  # 0 = free
    live = []
    next_id = 1
    for step in range(20000):
        if live and (g.random() < 0.45 or len(live) > 30):
            k = int(g.integers(0, len(live)))  # free in any order
            rec, rid = live.pop(k)
            assert np.all(owner[rec[0]:rec[0] + rec[1]] == rid)
            owner[rec[0]:rec[0] + rec[1]] = 0
            ring.free(rec)
        else:
            w = int(g.integers(1, 300))
            rec = ring.alloc(w)
            if rec is not None:
                assert 0 <= rec[0] and rec[0] + w <= size
                assert np.all(owner[rec[0]:rec[0] + w] == 0), "overlapping live allocations"
                owner[rec[0]:rec[0] + w] = next_id
                live.append((rec, next_id))
                next_id += 1
    for rec, rid in live:
        ring.free(rec)
    assert not ring.live
    assert ring.alloc(size) is not None


def test_ring_arena_fifo_reuse():
    ring = RingArena(100)
    a = ring.alloc(60)
    b = ring.alloc(30)
    assert ring.alloc(20) is None  # 10 left at the end, nothing at the start yet
    ring.free(b)
    assert ring.alloc(20) is None  # b is behind a: space returns in order
    ring.free(a)
    c = ring.alloc(90)
    assert c is not None and c[0] == 0


def test_trace_shape():
    tr = make_trace(20000, 0.5, 1, pool=1 << 25)
    assert 8000 < len(tr) < 12000
    n = np.asarray([r.n for r in tr])
    assert n.min() >= 1 << 10 and n.max() < 1 << 24
    assert {r.kind for r in tr} == {"sort", "multisplit"}
    assert {r.m for r in tr if r.kind == "multisplit"} == {8, 32, 256}
    assert all(0 <= r.in_off and r.in_off + r.n <= 1 << 25 for r in tr)
    arr = np.asarray([r.arrival for r in tr])
    assert np.all(np.diff(arr) >= 0) and arr.max() < 0.5
