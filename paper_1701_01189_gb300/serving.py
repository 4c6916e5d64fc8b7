"""Continuous-batching service for multisplit and radix-sort requests.

Not in the paper; this serves the multisplit of Section 3.1 and the radix
sort of Section 7.1 to a stream of requests of mixed sizes, on one GPU:

* Requests arrive over time (a Poisson trace).  Each is a key-value multisplit
  into m buckets by the service's range splitters for that m, or a key-value
  radix sort over all 32 key bits.  Its input is a window of the service's
  resident input pool (data already on the GPU, as in the paper's setting).
* Admission: a request is admitted when its output (and, for a sort, its
  ping-pong) buffers fit in a fixed device arena (16 GB by default), allocated
  as a ring in arrival order and freed as requests complete.
* Continuous batching: S launch slots, each with its own CUDA stream and its
  own dynamic batch plans.  Whenever a slot is idle, the requests that have
  arrived and fit are batched into it -- one persistent batched launch per
  request class (each m; each of the four sort digits in turn) for the small
  requests, and the plain entry points on the slot's stream for requests of
  at least `plain_min_elements` (they fill the GPU on their own, so batching
  gains them nothing) -- while the batches of other slots are still running
  on the device.  A slot's completion event marks its requests done and frees
  their memory.
* Reported: p50 / p99 latency (arrival to observed completion) and throughput
  in 1e9 elements per second, beside the same trace served one request at a
  time with the plain entry points.

Every result equals the plain entry point's result on that request alone
(bit-exact); ``tests/test_gpu_serving.py`` checks it.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import _binding as B

GIB = 1 << 30


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the trace starts
    kind: str       # "multisplit" or "sort"
    m: int          # buckets (multisplit), 0 for a sort
    n: int
    in_off: int     # first element of the input window in the pool
    # filled while serving
    out_off: int = -1
    tmp_off: int = -1
    admitted: float = -1.0
    done: float = -1.0


def make_trace(rate: float, duration: float, seed: int, pool: int, n_lo: int = 10, n_hi: int = 24,
               ms=(8, 32, 256), sort_fraction: float = 0.5):
    """Poisson arrivals; sizes floor(2^U), U ~ U(n_lo, n_hi); half sorts, half multisplits (m uniform)."""
    import synthetic

    t = synthetic.poisson_arrivals(rate, duration, seed)
    g = synthetic.rng(seed + 1)
    n = np.floor(np.exp2(g.uniform(n_lo, n_hi, size=len(t)))).astype(np.int64)
    is_sort = g.random(len(t)) < sort_fraction
    mm = g.choice(np.asarray(ms), size=len(t))
    offs = (g.random(len(t)) * (pool - n + 1)).astype(np.int64)
    return [Request(i, float(t[i]), "sort" if is_sort[i] else "multisplit", 0 if is_sort[i] else int(mm[i]),
                    int(n[i]), int(offs[i])) for i in range(len(t))]


class RingArena:
    """Device arena (in 4-byte words) handed out as a ring in admission order.

    Allocations are contiguous; a request that does not fit before the end of
    the arena starts again at word 0 (the skipped tail is returned with the
    allocations before it).  Space comes back when the oldest live allocations
    are freed, so out-of-order completions are held until those before them
    finish.
    """

    def __init__(self, words: int):
        self.size = words
        self.head = 0
        self.live = deque()  # [start, words, freed]

    def alloc(self, words: int):
        if words <= 0 or words > self.size:
            return None
        if not self.live:
            self.head = 0
            start = 0
        else:
            tail = self.live[0][0]
            if self.head > tail:
                # live space is [tail, head): free space is [head, size) and [0, tail)
                if self.head + words <= self.size:
                    start = self.head
                elif words <= tail:
                    if self.head < self.size:
                        self.live.append([self.head, self.size - self.head, True])
                    start = 0
                else:
                    return None
            elif self.head < tail:
                # live space wraps around the end: free space is [head, tail)
                if self.head + words <= tail:
                    start = self.head
                else:
                    return None
            else:
                return None  # head == tail: full
        rec = [start, words, False]
        self.live.append(rec)
        self.head = start + words
        return rec

    def free(self, rec):
        rec[2] = True
        while self.live and self.live[0][2]:
            self.live.popleft()


@dataclass
class _Slot:
    stream: object
    plans: dict
    event: object = None
    reqs: list = field(default_factory=list)
    recs: list = field(default_factory=list)


class Service:
    def __init__(self, pool_keys, pool_vals, splitters: dict, arena_bytes: int = 16 * GIB, slots: int = 4,
                 max_batch_segments: int = 256, max_batch_elements: int = 1 << 27,
                 plain_min_elements: int = 1 << 18):
        import torch

        self.torch = torch
        self.dev = pool_keys.device
        self.pk, self.pv = pool_keys, pool_vals
        self.pool = pool_keys.numel()
        self.specs = {m: B.BucketSpec.range_u32(spl) for m, spl in splitters.items()}
        self.radix = [B.BucketSpec.radix(8 * p, 8) for p in range(4)]
        self.arena = torch.empty(arena_bytes // 4, dtype=torch.int32, device=self.dev)
        self.ring = RingArena(self.arena.numel())
        self.max_seg, self.max_el = max_batch_segments, max_batch_elements
        self.plain_min = plain_min_elements
        self.slots = []
        for _ in range(slots):
            plans = {}
            for m, sp in self.specs.items():
                st, h = B.ms_batch_plan_create_dynamic(max_batch_segments, max_batch_elements, True, sp.c())
                B._check(st, "ms_batch_plan_create_dynamic")
                plans[("ms", m)] = h
            for p, sp in enumerate(self.radix):
                st, h = B.ms_batch_plan_create_dynamic(max_batch_segments, max_batch_elements, True, sp.c())
                B._check(st, "ms_batch_plan_create_dynamic")
                plans[("sort", p)] = h
            self.slots.append(_Slot(torch.cuda.Stream(device=self.dev), plans))

    def close(self):
        for s in self.slots:
            for h in s.plans.values():
                B.ms_batch_plan_destroy(h)
        self.slots = []

    # ---------------------------------------------------------------- buffers of one request
    def _plain(self, r: Request) -> bool:
        return r.n >= self.plain_min

    def _words(self, r: Request) -> int:
        # out keys + values (+ the ping-pong of a batched sort; a plain sort keeps its own)
        return 2 * r.n + (2 * r.n if r.kind == "sort" and not self._plain(r) else 0)

    def out_views(self, r: Request):
        a = self.arena
        ko = a[r.out_off:r.out_off + r.n]
        vo = a[r.out_off + r.n:r.out_off + 2 * r.n]
        return ko, vo

    def _ptrs(self, r: Request):
        base = self.arena.data_ptr()
        kin = self.pk.data_ptr() + 4 * r.in_off
        vin = self.pv.data_ptr() + 4 * r.in_off
        ko = base + 4 * r.out_off
        vo = base + 4 * (r.out_off + r.n)
        batched_sort = r.kind == "sort" and not self._plain(r)
        tk = base + 4 * (r.out_off + 2 * r.n) if batched_sort else None
        tv = base + 4 * (r.out_off + 3 * r.n) if batched_sort else None
        return kin, vin, ko, vo, tk, tv

    # ---------------------------------------------------------------- one batch on one slot
    def _launch(self, slot: _Slot, batch):
        torch = self.torch
        sptr = slot.stream.cuda_stream
        groups = {}
        for r in batch:
            if self._plain(r):
                kin, vin, ko, vo, _, _ = self._ptrs(r)
                if r.kind == "multisplit":
                    st = B.ms_multisplit_pairs(kin, vin, r.n, self.specs[r.m].c(), ko, vo, None, sptr)
                else:
                    st = B.ms_radix_sort(kin, vin, r.n, 0, 32, ko, vo, sptr)
                B._check(st, "plain")
                continue
            groups.setdefault((r.kind, r.m), []).append(r)
        for (kind, m), rs in groups.items():
            if kind == "multisplit":
                segs = []
                for r in rs:
                    kin, vin, ko, vo, _, _ = self._ptrs(r)
                    segs.append((kin, vin, ko, vo, None, r.n))
                h = slot.plans[("ms", m)]
                B._check(B.ms_batch_plan_set_segments(h, segs, sptr), "set_segments")
                B._check(B.ms_batch_run(h, sptr), "ms_batch_run")
            else:
                # LSD: digit p moves in -> tmp -> out -> tmp -> out
                for p in range(4):
                    segs = []
                    for r in rs:
                        kin, vin, ko, vo, tk, tv = self._ptrs(r)
                        src = (kin, vin) if p == 0 else ((tk, tv) if p % 2 == 1 else (ko, vo))
                        dst = (tk, tv) if p % 2 == 0 else (ko, vo)
                        segs.append((src[0], src[1], dst[0], dst[1], None, r.n))
                    h = slot.plans[("sort", p)]
                    B._check(B.ms_batch_plan_set_segments(h, segs, sptr), "set_segments")
                    B._check(B.ms_batch_run(h, sptr), "ms_batch_run")
        ev = torch.cuda.Event()
        ev.record(slot.stream)
        slot.event = ev

    def serve(self, trace, real_time: bool = True, on_complete=None):
        """Serves the trace; returns a summary dict.  With real_time, arrivals are
        released at their trace time; otherwise all at once.  on_complete(request)
        is called for every request once its results are in the arena, before its
        memory is released (out_views(request) gives them)."""
        reqs = sorted(trace, key=lambda r: r.arrival)
        queue = deque()
        i = 0
        t0 = time.perf_counter()
        remaining = len(reqs)
        idle = deque(self.slots)
        busy = []
        while remaining:
            now = time.perf_counter() - t0
            while i < len(reqs) and (not real_time or reqs[i].arrival <= now):
                queue.append(reqs[i])
                i += 1
            # completions
            still = []
            for s in busy:
                if s.event.query():
                    tdone = time.perf_counter() - t0
                    for r in s.reqs:
                        r.done = tdone
                        if on_complete is not None:
                            on_complete(r)
                    for rec in s.recs:
                        self.ring.free(rec)
                    remaining -= len(s.reqs)
                    s.reqs, s.recs = [], []
                    idle.append(s)
                else:
                    still.append(s)
            busy = still
            # admission into idle slots
            while idle and queue:
                batch, recs, elems = [], [], 0
                while queue and len(batch) < self.max_seg:
                    r = queue[0]
                    if elems + r.n > self.max_el and batch:
                        break
                    rec = self.ring.alloc(self._words(r))
                    if rec is None:
                        break
                    queue.popleft()
                    r.out_off = rec[0]
                    r.admitted = now
                    batch.append(r)
                    recs.append(rec)
                    elems += r.n
                if not batch:
                    break
                s = idle.popleft()
                s.reqs, s.recs = batch, recs
                self._launch(s, batch)
                busy.append(s)
            if not busy and not queue and i < len(reqs) and real_time:
                time.sleep(max(0.0, min(0.001, reqs[i].arrival - (time.perf_counter() - t0))))
        self.torch.cuda.synchronize()
        return summarize(reqs)


def serve_serial(trace, pool_keys, pool_vals, splitters: dict, real_time: bool = True):
    """The same trace, one request at a time with the plain entry points."""
    import torch

    specs = {m: B.BucketSpec.range_u32(spl) for m, spl in splitters.items()}
    reqs = sorted(trace, key=lambda r: r.arrival)
    nmax = max(r.n for r in reqs)
    ko = torch.empty(nmax, dtype=torch.int32, device=pool_keys.device)
    vo = torch.empty_like(ko)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    t0 = time.perf_counter()
    for r in reqs:
        if real_time:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        kin = pool_keys.data_ptr() + 4 * r.in_off
        vin = pool_vals.data_ptr() + 4 * r.in_off
        r.admitted = time.perf_counter() - t0
        if r.kind == "multisplit":
            st = B.ms_multisplit_pairs(kin, vin, r.n, specs[r.m].c(), ko.data_ptr(), vo.data_ptr(), None, sptr)
        else:
            st = B.ms_radix_sort(kin, vin, r.n, 0, 32, ko.data_ptr(), vo.data_ptr(), sptr)
        B._check(st, "serial")
        stream.synchronize()
        r.done = time.perf_counter() - t0
    return summarize(reqs)


def summarize(reqs):
    lat = np.asarray([r.done - r.arrival for r in reqs]) * 1e3
    elems = sum(r.n for r in reqs)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "elements": int(elems), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "span_s": round(span, 3), "g_elements_s": round(elems / span / 1e9, 3)}


def run_config(seconds: float = 10.0, rate: float = 20000.0, seed: int = 2026, slots: int = 4,
               arena_bytes: int = 16 * GIB, serial: bool = True):
    """The serving configuration: Poisson arrivals at `rate` per second for
    `seconds`, key-value multisplit (m in {8, 32, 256}, range buckets) or
    key-value radix sort, n = floor(2^U), U ~ U(10, 24), a 16 GB arena; then the
    same trace served one request at a time with plain launches."""
    import torch

    import synthetic

    pool = 1 << 25
    dev = torch.device("cuda", torch.cuda.current_device())

    def dev_u32(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)

    pk = dev_u32(synthetic.uniform_u32(pool, seed))
    pv = dev_u32(synthetic.index_values(pool))
    spl = {m: dev_u32(synthetic.range_splitters(m, seed + m)) for m in (8, 32, 256)}
    trace = make_trace(rate, seconds, seed, pool=pool)
    svc = Service(pk, pv, spl, arena_bytes=arena_bytes, slots=slots)
    try:
        batched = svc.serve(trace, real_time=True)
    finally:
        svc.close()
    out = {"trace": {"rate_per_s": rate, "seconds": seconds, "requests": len(trace), "seed": seed},
           "batched": batched}
    if serial:
        trace2 = make_trace(rate, seconds, seed, pool=pool)
        out["serial_plain"] = serve_serial(trace2, pk, pv, spl, real_time=True)
    return out


if __name__ == "__main__":
    import argparse
    import json
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="serve a Poisson trace of multisplit and sort requests")
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--rate", type=float, default=20000.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--no-serial", action="store_true")
    args = ap.parse_args()
    from .build import build

    build()
    print(json.dumps(run_config(args.seconds, args.rate, slots=args.slots, serial=not args.no_serial)))
