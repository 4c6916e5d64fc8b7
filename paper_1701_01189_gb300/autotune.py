"""Autotuner for the multisplit kernel variants.

For a set of workloads (bucket kind, m, keys or pairs, n) it times every
variant the library offers -- post-scan tile shape (8 warps x 16 keys, 16 x 8,
8 x 8), rank mode (warp ballots for m <= 32, per-warp peer tables,
per-thread bucket counters for m <= 32, or ballot peers with per-warp
counters) and reordering (block reorder, or
direct writes for ballot ranks) -- with CUDA
events on the current stream, and installs the fastest for that workload's key
(kind, pairs, ceil(log2 m), size class of n) with ``ms_tune_set``.  Results can
be saved to and loaded from JSON (``tuning.json`` beside this file by default).

The paper fixed its parameters per architecture by hand (Section 6,
"Parameters"); this replaces that with a measurement on the device in use.
"""
from __future__ import annotations

import json
import os

from . import _binding as B

DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def variants(log2m: int):
    out = [(0, 2, 1), (1, 2, 1), (2, 2, 1)] if log2m <= 5 else []
    for shape in (0, 1, 2):
        out.append((shape, 1, 1))
        if log2m >= 4:
            out.append((shape, 3, 1))
        if log2m <= 5:
            out.append((shape, 0, 1))
        if log2m <= 3:
            out.append((shape, 0, 0))
    return out


def _time_call(fn, reps: int) -> float:
    import torch

    for _ in range(2):
        fn()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune_workload(keys, vals, spec: B.BucketSpec, reps: int = 5):
    """Times every variant for this workload, installs the fastest, returns
    (key, best_variant, {variant: ms}).  `keys` may be a list of key arrays of
    one size (e.g. differently distributed inputs): a variant's time is then
    the sum over them."""
    import torch

    key_sets = keys if isinstance(keys, (list, tuple)) else [keys]
    keys = key_sets[0]
    n = keys.numel()
    log2m = (spec.m - 1).bit_length()
    pairs = 1 if vals is not None else 0
    sc = B.ms_tune_size_class(n)
    kind = spec.kind if spec.m > 1 else B.RADIX
    ko = torch.empty_like(keys)
    vo = torch.empty_like(keys) if vals is not None else None
    off = torch.empty(spec.m + 1, dtype=torch.int32, device=keys.device)
    cs = spec.c()
    stream = torch.cuda.current_stream().cuda_stream

    def runner(ks):
        def run():
            if vals is None:
                st = B.ms_multisplit_keys(ks.data_ptr(), n, cs, ko.data_ptr(), off.data_ptr(), stream)
            else:
                st = B.ms_multisplit_pairs(ks.data_ptr(), vals.data_ptr(), n, cs, ko.data_ptr(), vo.data_ptr(),
                                           off.data_ptr(), stream)
            if st != B.MS_OK:
                raise B.MsError(st, "autotune")
        return run

    times = {}
    for v in variants(log2m):
        B._check(B.ms_tune_set(kind, pairs, log2m, sc, *v), "ms_tune_set")
        times[v] = sum(_time_call(runner(ks), reps) for ks in key_sets)
    best = min(times, key=times.get)
    B._check(B.ms_tune_set(kind, pairs, log2m, sc, *best), "ms_tune_set")
    return (kind, pairs, log2m, sc), best, times


def tune_sort(n: int, pairs: bool, reps: int = 3):
    """Times ms_radix_sort (all 32 bits) with one-sweep passes (method 0) and with
    three-stage multisplit passes (method 1, whose variants come from the
    multisplit table, so tune that first); installs and returns the faster:
    ((pairs, size_class), method, {method: ms})."""
    import numpy as np
    import torch

    import synthetic

    dev = torch.device("cuda", torch.cuda.current_device())
    keys = torch.from_numpy(synthetic.uniform_u32(n, 5).view(np.int32)).to(dev)
    vals = torch.arange(n, dtype=torch.int32, device=dev) if pairs else None
    ko = torch.empty_like(keys)
    vo = torch.empty_like(keys) if pairs else None
    stream = torch.cuda.current_stream().cuda_stream
    sc = B.ms_tune_size_class(n)

    def run():
        st = B.ms_radix_sort(keys.data_ptr(), vals.data_ptr() if pairs else None, n, 0, 32, ko.data_ptr(),
                             vo.data_ptr() if pairs else None, stream)
        if st != B.MS_OK:
            raise B.MsError(st, "autotune sort")

    times = {}
    for method in (0, 1):
        B._check(B.ms_tune_set_sort(int(pairs), sc, method), "ms_tune_set_sort")
        times[method] = _time_call(run, reps)
    best = min(times, key=times.get)
    B._check(B.ms_tune_set_sort(int(pairs), sc, best), "ms_tune_set_sort")
    return (int(pairs), sc), best, times


def batch_variants(log2m: int):
    """(shape, rank) candidates of the batched kernel: per-thread counters
    (m <= 32), peer tables and ballot peers in both tile shapes."""
    out = [(0, 2)] if log2m <= 5 else []
    for shape in (0, 1):
        out += [(shape, 1), (shape, 3)]
    return out


def tune_batch(kind_name: str, m: int, pairs: bool, segments: int = 1024, seg_log2=(8.0, 20.0), reps: int = 5):
    """Times every batched-kernel variant on a plan of `segments` segments of
    floor(2^U) keys, U ~ U(seg_log2) (the batched configuration's size law),
    through the CUDA-graph replay; installs the fastest for the key (kind,
    pairs, ceil(log2 m), size class of the mean segment) with
    ms_tune_set_batch and returns (key, best, {variant: ms})."""
    import numpy as np
    import torch

    import synthetic

    dev = torch.device("cuda", torch.cuda.current_device())
    sizes = synthetic.segment_sizes(segments, seg_log2[0], seg_log2[1], 2024)
    total = int(sizes.sum())
    gen = synthetic.uniform_f32_1000 if kind_name == "delta" else synthetic.uniform_u32
    kall = torch.from_numpy(gen(total, 2025).view(np.int32)).to(dev)
    vall = torch.zeros_like(kall) if pairs else None
    ko = torch.empty_like(kall)
    vo = torch.empty_like(kall) if pairs else None
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    segs = []
    for s0, n_ in zip(starts, sizes):
        o = 4 * int(s0)
        segs.append((kall.data_ptr() + o, vall.data_ptr() + o if pairs else None, ko.data_ptr() + o,
                     vo.data_ptr() + o if pairs else None, None, int(n_)))
    spec = _spec(kind_name, m, dev)
    cs = spec.c()
    log2m = (m - 1).bit_length()
    kind = spec.kind if m > 1 else B.RADIX
    sc = B.ms_tune_size_class(total // segments)
    stream = torch.cuda.current_stream().cuda_stream
    times = {}
    for v in batch_variants(log2m):
        B._check(B.ms_tune_set_batch(kind, int(pairs), log2m, sc, *v), "ms_tune_set_batch")
        st, plan = B.ms_batch_plan_create(segs, cs)
        B._check(st, "ms_batch_plan_create")
        try:
            times[v] = _time_call(lambda: B._check(B.ms_batch_run_graph(plan, stream), "ms_batch_run_graph"), reps)
        finally:
            B.ms_batch_plan_destroy(plan)
    best = min(times, key=times.get)
    B._check(B.ms_tune_set_batch(kind, int(pairs), log2m, sc, *best), "ms_tune_set_batch")
    return (kind, int(pairs), log2m, sc), best, times


def _spec(kind_name: str, m: int, dev):
    import numpy as np
    import torch

    import synthetic

    if kind_name == "radix":
        bits = (m - 1).bit_length()
        return B.BucketSpec.radix(32 - bits, bits)
    if kind_name == "range":
        spl = synthetic.range_splitters(m, 3)
        return B.BucketSpec.range_u32(torch.from_numpy(spl.view(np.int32)).to(dev))
    if kind_name == "mod":
        return B.BucketSpec.mod(m)
    return B.BucketSpec.delta_f32(m, float(np.float32(1000.0) / np.float32(m)))


def save(entries, path: str = DEFAULT_PATH, sort_entries=(), batch_entries=()):
    """entries: list of (key, variant) pairs as returned by tune_workload;
    sort_entries: list of (key, method) pairs as returned by tune_sort;
    batch_entries: list of (key, (shape, rank)) pairs as returned by tune_batch."""
    data = [{"kind": k[0], "pairs": k[1], "log2m": k[2], "size_class": k[3], "shape": v[0], "rank": v[1],
             "reorder": v[2]} for k, v in entries]
    sort = [{"pairs": k[0], "size_class": k[1], "method": m} for k, m in sort_entries]
    batch = [{"kind": k[0], "pairs": k[1], "log2m": k[2], "size_class": k[3], "shape": v[0], "rank": v[1]}
             for k, v in batch_entries]
    with open(path, "w") as f:
        json.dump({"format": 1, "entries": data, "sort": sort, "batch": batch}, f, indent=1)


def load(path: str = DEFAULT_PATH) -> int:
    """Installs a saved table; returns the number of entries installed (0 if absent)."""
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        data = json.load(f)
    count = 0
    for e in data.get("entries", []):
        st = B.ms_tune_set(e["kind"], e["pairs"], e["log2m"], e["size_class"], e["shape"], e["rank"], e["reorder"])
        count += st == B.MS_OK
    for e in data.get("sort", []):
        count += B.ms_tune_set_sort(e["pairs"], e["size_class"], e["method"]) == B.MS_OK
    for e in data.get("batch", []):
        count += B.ms_tune_set_batch(e["kind"], e["pairs"], e["log2m"], e["size_class"], e["shape"], e["rank"]) == B.MS_OK
    return count


def tune_suite(n_log2s=(20, 26), ms=(2, 8, 32, 64, 256), kinds=("range", "delta", "mod", "radix"), reps: int = 5):
    """Tunes every (identifier, m, keys or key-value, size) of the list on
    seeded uniform inputs; returns the (key, variant) entries."""
    import numpy as np
    import torch

    import synthetic

    entries = []
    dev = torch.device("cuda", torch.cuda.current_device())
    for n_log2 in n_log2s:
        n = 1 << n_log2
        u = torch.from_numpy(synthetic.uniform_u32(n, 1).view(np.int32)).to(dev)
        f = torch.from_numpy(synthetic.uniform_f32_1000(n, 2).view(np.int32)).to(dev)
        v = torch.arange(n, dtype=torch.int32, device=dev)
        for kind in kinds:
            for m in ms:
                if kind == "radix":
                    bits = (m - 1).bit_length()
                    spec = B.BucketSpec.radix(32 - bits, bits)
                elif kind == "range":
                    spl = synthetic.range_splitters(m, 3)
                    spec = B.BucketSpec.range_u32(torch.from_numpy(spl.view(np.int32)).to(dev))
                elif kind == "mod":
                    spec = B.BucketSpec.mod(m)
                else:
                    spec = B.BucketSpec.delta_f32(m, float(np.float32(1000.0) / np.float32(m)))
                keys = f if kind == "delta" else u
                if kind == "range":  # the benchmark's range inputs: uniform and skewed keys
                    keys = [u, torch.from_numpy(synthetic.skewed_u32(n, spl, 4).view(np.int32)).to(dev)]
                for vals in (None, v):
                    key, best, times = tune_workload(keys, vals, spec, reps=reps)
                    entries.append((key, best))
                    print(f"{kind} m={m} {'pairs' if vals is not None else 'keys'} n=2^{n_log2}: best {best} "
                          f"{times[best]:.4f} ms of {len(times)} variants", flush=True)
    return entries


if __name__ == "__main__":
    import argparse
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="measure the multisplit kernel variants and save the fastest per workload")
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--only-batch", action="store_true",
                    help="tune the batched kernels only, keeping the other entries of the table at --out")
    args = ap.parse_args()
    from .build import build

    build()
    batch_entries = []
    for kind_name in ("mod", "range"):
        for m in (2, 8, 32, 64, 256):
            for pairs in (False, True):
                key, best, times = tune_batch(kind_name, m, pairs, reps=args.reps)
                batch_entries.append((key, best))
                print(f"batched {kind_name} m={m} {'pairs' if pairs else 'keys'}: best {best} "
                      f"({', '.join(f'{k}: {v:.3f} ms' for k, v in times.items())})", flush=True)
    if args.only_batch:
        old = json.load(open(args.out)) if os.path.exists(args.out) else {}
        entries = [((e["kind"], e["pairs"], e["log2m"], e["size_class"]), (e["shape"], e["rank"], e["reorder"]))
                   for e in old.get("entries", [])]
        sort_entries = [((e["pairs"], e["size_class"]), e["method"]) for e in old.get("sort", [])]
        save(entries, args.out, sort_entries, batch_entries)
        print("saved", args.out)
        raise SystemExit(0)
    entries = tune_suite(reps=args.reps)
    sort_entries = []
    for n_log2 in (22, 28):
        for pairs in (False, True):
            key, best, times = tune_sort(1 << n_log2, pairs)
            sort_entries.append((key, best))
            print(f"sort n=2^{n_log2} {'pairs' if pairs else 'keys'}: best method {best} "
                  f"({', '.join(f'{k}: {v:.3f} ms' for k, v in times.items())})", flush=True)
    save(entries, args.out, sort_entries, batch_entries)
    print("saved", args.out)
