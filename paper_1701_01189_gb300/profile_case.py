"""Runs one multisplit or radix-sort case repeatedly, for profiling (e.g. under
Nsight Compute) and quick timing.

    python -m paper_1701_01189_gb300.profile_case --kind range --m 32 --n-log2 26 --reps 3
    python -m paper_1701_01189_gb300.profile_case --kind sort --pairs --n-log2 24
    python -m paper_1701_01189_gb300.profile_case --kind range --m 65536 --n-log2 24
    python -m paper_1701_01189_gb300.profile_case --kind batch --segments 1024 --seg-log2 8 16 --pairs

Prints the mean time per call (CUDA events) and the per-stage times of the
library's stage timer.  Inputs are the seeded uniform keys of ``synthetic``.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--kind", choices=["range", "radix", "mod", "delta", "sort", "batch"], default="range")
    ap.add_argument("--m", type=int, default=32)
    ap.add_argument("--pairs", action="store_true")
    ap.add_argument("--n-log2", type=int, default=26)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--sort-method", type=int, default=None, choices=[0, 1],
                    help="sort: 0 one sweep per digit, 1 a three-stage multisplit per digit (default: tuned)")
    ap.add_argument("--segments", type=int, default=1024, help="batch: number of segments (key mod m)")
    ap.add_argument("--seg-log2", type=float, nargs=2, default=(8.0, 20.0),
                    help="batch: segment sizes floor(2^U), U ~ U(lo, hi)")
    ap.add_argument("--variant", default=None,
                    help="shape,rank,reorder of the kernel variant to run (see ms_tune_set); default: the tuned one")
    args = ap.parse_args(argv)

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import torch

    import paper_1701_01189_gb300 as ms
    import synthetic
    from paper_1701_01189_gb300 import autotune
    from paper_1701_01189_gb300.build import build

    build()
    autotune.load()
    if args.kind == "batch":
        return run_batch(args, ms, torch, np, synthetic)
    n = 1 << args.n_log2
    gen = synthetic.uniform_f32_1000 if args.kind == "delta" else synthetic.uniform_u32
    dk = torch.from_numpy(gen(n, 1).view(np.int32)).cuda()
    dv = torch.arange(n, dtype=torch.int32, device="cuda") if args.pairs else None
    ko = torch.empty_like(dk)
    vo = torch.empty_like(dk) if args.pairs else None
    off = torch.empty(max(args.m, 256) + 1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    if args.kind == "range":
        spec = ms.BucketSpec.range_u32(torch.from_numpy(synthetic.range_splitters(args.m, 3).view(np.int32)).cuda())
    elif args.kind == "radix":
        spec = ms.BucketSpec.radix(0, int(np.log2(args.m)))
    elif args.kind == "mod":
        spec = ms.BucketSpec.mod(args.m)
    else:
        spec = ms.BucketSpec.delta_f32(args.m, float(np.float32(1000.0) / np.float32(args.m)))
    cs = spec.c()
    if args.sort_method is not None:
        st = ms.ms_tune_set_sort(int(args.pairs), ms.ms_tune_size_class(n), args.sort_method)
        if st != ms.MS_OK:
            raise ms.MsError(st, "ms_tune_set_sort")
    if args.variant is not None:
        # for a sort, the variant of radix-digit multisplits with 256 buckets (its ranks)
        shape, rank, reorder = (int(x) for x in args.variant.split(","))
        log2m = 8 if args.kind == "sort" else (args.m - 1).bit_length()
        kind = ms.RADIX if args.kind == "sort" else spec.kind
        for pairs in (0, 1):
            st = ms.ms_tune_set(kind, pairs, log2m, ms.ms_tune_size_class(n), shape, rank, reorder)
            if st != ms.MS_OK:
                raise ms.MsError(st, "ms_tune_set")

    def run():
        if args.kind == "sort":
            st = ms.ms_radix_sort(dk.data_ptr(), dv.data_ptr() if args.pairs else None, n, 0, 32, ko.data_ptr(),
                                  vo.data_ptr() if args.pairs else None, stream)
        elif args.pairs:
            st = ms.ms_multisplit_pairs(dk.data_ptr(), dv.data_ptr(), n, cs, ko.data_ptr(), vo.data_ptr(),
                                        off.data_ptr(), stream)
        else:
            st = ms.ms_multisplit_keys(dk.data_ptr(), n, cs, ko.data_ptr(), off.data_ptr(), stream)
        if st != ms.MS_OK:
            raise ms.MsError(st, "profile_case")

    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    ms.ms_stage_timing(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms.ms_stage_timing(0)
    t = e0.elapsed_time(e1) / args.reps
    pre, scan, post, cnt = ms.ms_stage_times()
    desc = f"{args.kind} m={args.m if args.kind != 'sort' else 256} {'pairs' if args.pairs else 'keys'} n=2^{args.n_log2}"
    if args.variant is not None:
        desc += f" variant {args.variant}"
    line = f"{desc}: {t:.4f} ms per call = {n / t / 1e6:.1f} G elements/s"
    if cnt:
        line += f"; per multisplit: pre-scan {pre / cnt:.4f} ms, scan {scan / cnt:.4f} ms, post-scan {post / cnt:.4f} ms"
    print(line)
    if ms.device_status() != ms.MS_OK:
        raise SystemExit("device status not OK")


def run_batch(args, ms, torch, np, synthetic):
    """A batched plan of key-mod-m segments (values = index when --pairs), run through the graph."""
    sizes = synthetic.segment_sizes(args.segments, args.seg_log2[0], args.seg_log2[1], 2024)
    total = int(sizes.sum())
    kall = torch.from_numpy(synthetic.uniform_u32(total, 2025).view(np.int32)).cuda()
    vall = torch.zeros_like(kall) if args.pairs else None
    ko = torch.empty_like(kall)
    vo = torch.empty_like(kall) if args.pairs else None
    offs = torch.empty((args.segments, args.m + 1), dtype=torch.int32, device="cuda")
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    segs = []
    for i, (s0, n_) in enumerate(zip(starts, sizes)):
        o = 4 * int(s0)
        segs.append((kall.data_ptr() + o, vall.data_ptr() + o if args.pairs else None, ko.data_ptr() + o,
                     vo.data_ptr() + o if args.pairs else None, offs[i].data_ptr(), int(n_)))
    st, plan = ms.ms_batch_plan_create(segs, ms.BucketSpec.mod(args.m).c())
    if st != ms.MS_OK:
        raise ms.MsError(st, "ms_batch_plan_create")
    stream = torch.cuda.current_stream().cuda_stream
    try:
        for _ in range(args.warmup):
            ms.ms_batch_run_graph(plan, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            ms.ms_batch_run_graph(plan, stream)
        e1.record()
        torch.cuda.synchronize()
    finally:
        ms.ms_batch_plan_destroy(plan)
    t = e0.elapsed_time(e1) / args.reps
    print(f"batch {args.segments} segments ({total} {'pairs' if args.pairs else 'keys'}) key mod {args.m}: "
          f"{t:.4f} ms per run = {total / t / 1e6:.1f} G elements/s")
    if ms.device_status() != ms.MS_OK:
        raise SystemExit("device status not OK")


if __name__ == "__main__":
    main()
