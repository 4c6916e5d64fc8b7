"""Benchmark of the stable multisplit on one GB300 (or N replicas).

Workload (one "step"): the multisplit sweep at n = 2^26 -- uniform and skewed
uint32 keys with range buckets from m-1 sorted uniform splitters, m in
{2, 8, 32, 64, 256}, keys only and key-value (value = original index), plus
float32 keys uniform in [0, 1000) with delta buckets (delta = 1000/m), keys
only and key-value: 30 multisplits of 2^26 elements each.  Inputs are seeded,
synthetic, resident in HBM before the timed region, and each 256 MB input is
larger than the 126 MB L2, so no L2 flush is needed between steps.

Printed: one JSON line (rank 0).  ``value`` is the whole-job rate in 1e9
elements per second (keys for key-only cases, pairs for key-value cases);
``sweep`` gives every case's own Gkeys/s or Gpairs/s and its fraction of the
compulsory-bytes HBM roofline (read once + write once: 8 B/key, 16 B/pair).
``roofline`` is the post-scan kernel (the dominant one), timed with CUDA events
recorded by the library around each stage on the launching stream.  ``e2e``
runs the same sweep from pinned host buffers with the host<->device copies in
the timed region (two streams, double-buffered).  ``cpu_baseline`` times the CPU oracle on a bounded sample.  ``extras`` holds
the radix-sort, device-histogram, Section 6.4 distribution (uniform,
0.25-uniform, binomial at m = 256), batched and serving configurations.

``--impl reference`` times the CPU oracle (the reference arm of this
repository) on samples of the same workload.  With N > 1 (torchrun) every
rank runs the same sweep on its own GPU ("replicas only": multisplit needs no
exchange step between GPUs here); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "multisplit Gkeys/s & Gpairs/s and % of HBM roofline vs m; batched vs plain; p99 ms"
MS_LIST = [2, 8, 32, 64, 256]
WORKLOAD = ("multisplit sweep n=2^26: uint32 keys uniform + skewed (geometric p=0.5), range buckets "
            "(m-1 sorted uniform splitters), float32 keys uniform [0,1000) with delta=1000/m, "
            "m in {2,8,32,64,256}, keys-only and key-value (value = index)")


def cases(n_log2: int):
    """(name, key_array_id, kind, m, pairs) for the 30 sweep cases."""
    out = []
    for dist in ("uniform", "skewed"):
        for m in MS_LIST:
            for pairs in (False, True):
                out.append((f"range_{dist}_m{m}_{'pairs' if pairs else 'keys'}", (dist, m), "range", m, pairs))
    for m in MS_LIST:
        for pairs in (False, True):
            out.append((f"delta_f32_m{m}_{'pairs' if pairs else 'keys'}", ("f32", m), "delta", m, pairs))
    return out


def make_inputs(n: int):
    """Host arrays: key arrays by id, splitters per m, values."""
    keys, spl = {}, {}
    uni = synthetic.uniform_u32(n, 2026)
    f32 = synthetic.uniform_f32_1000(n, 2027)
    for m in MS_LIST:
        spl[m] = synthetic.range_splitters(m, 100 + m)
        keys[("uniform", m)] = uni
        keys[("skewed", m)] = synthetic.skewed_u32(n, spl[m], 200 + m)
        keys[("f32", m)] = f32
    vals = synthetic.index_values(n)
    return keys, spl, vals


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_dir: str):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(out_dir, f"clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- roofline inputs
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_sources(names):
    """The files that define the sweep's kernels: the device headers and the
    per-identifier translation units that instantiate them."""
    return sorted(n for n in names if n.endswith(".cuh") or (n.startswith("ms_kind_") and n.endswith(".cu")))


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1701_01189_gb300", "csrc")
    for name in kernel_sources(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per element of the post-scan from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "postscan_traffic.json")
    try:
        with open(p) as f:
            j = json.load(f)
    except Exception:
        return None
    if j.get("source_hash") != kernel_source_hash():
        return None
    return j


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank: int, world: int):
    import torch

    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300 import metrics
    from paper_1701_01189_gb300.build import build

    if rank == 0 or world == 1:
        build()
    if world > 1:
        torch.distributed.barrier()
    ms.lib()
    from paper_1701_01189_gb300 import autotune

    autotune.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 1 << args.n_log2
    hk, hspl, hvals = make_inputs(n)
    case_list = cases(args.n_log2)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)

    dkeys = {}
    for cid, arr in hk.items():
        key = id(arr)
        if key not in dkeys:
            dkeys[key] = to_dev(arr)
    dk = {cid: dkeys[id(arr)] for cid, arr in hk.items()}
    dspl = {m: to_dev(s) for m, s in hspl.items()}
    dvals = to_dev(hvals)
    out_k = torch.empty(n, dtype=torch.int32, device=dev)
    out_v = torch.empty(n, dtype=torch.int32, device=dev)
    offs = torch.empty(257, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    specs = {}
    for name, cid, kind, m, pairs in case_list:
        if kind == "range":
            specs[name] = ms.BucketSpec.range_u32(dspl[m]).c()
        else:
            specs[name] = ms.BucketSpec.delta_f32(m, float(np.float32(1000.0) / np.float32(m))).c()

    def one(name, cid, pairs, kin, vin):
        if pairs:
            st = ms.ms_multisplit_pairs(kin.data_ptr(), vin.data_ptr(), n, specs[name], out_k.data_ptr(),
                                        out_v.data_ptr(), offs.data_ptr(), sptr)
        else:
            st = ms.ms_multisplit_keys(kin.data_ptr(), n, specs[name], out_k.data_ptr(), offs.data_ptr(), sptr)
        if st != ms.MS_OK:
            raise ms.MsError(st, name)

    def step(events=None):
        for ci, (name, cid, kind, m, pairs) in enumerate(case_list):
            if events is not None:
                events[ci][0].record(stream)
            one(name, cid, pairs, dk[cid], dvals)
            if events is not None:
                events[ci][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ms.device_status() != ms.MS_OK:
        raise RuntimeError("device status not OK after warm-up")

    # ---- timed region (device-resident inputs)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in case_list] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", torch.cuda.current_device())), args.clocks_dir)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for s in range(args.steps):
        step(ev[s])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms = t0.elapsed_time(t1)
    if ms.device_status() != ms.MS_OK:
        raise RuntimeError("device status not OK after the timed region")

    # The same steps again with the library's stage timer on (CUDA events on
    # the launching stream around every kernel of every multisplit), for the
    # per-kernel durations of the roofline.  Recording events between the
    # kernels keeps the post-scan from starting early as a programmatic
    # dependent, so this pass is timed separately from the one above.
    torch.cuda.synchronize()
    ms.ms_stage_timing(1)
    for s in range(args.steps):
        step()
    torch.cuda.synchronize()
    ms.ms_stage_timing(0)
    pre_ms, scan_ms, post_ms, n_ms = ms.ms_stage_times()
    if ms.device_status() != ms.MS_OK:
        raise RuntimeError("device status not OK after the stage-timed steps")

    per_case = {}
    for ci, (name, cid, kind, m, pairs) in enumerate(case_list):
        tms = sum(ev[s][ci][0].elapsed_time(ev[s][ci][1]) for s in range(args.steps)) / args.steps
        rate = metrics.rate_g(n, tms * 1e-3)
        peak, _ = measured_peaks()
        comp = metrics.sol_rate_g(peak, metrics.compulsory_bytes_per_element(pairs))
        per_case[name] = {"ms": round(tms, 4), ("gpairs_s" if pairs else "gkeys_s"): round(rate, 2),
                          "frac_compulsory_roofline": round(rate / comp, 4)}

    elems_per_step = n * len(case_list)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = metrics.rate_g(elems_per_step * args.steps * world, total_ms * 1e-3)

    # roofline of the post-scan kernel: algorithmic bytes = read + write of every key (and value)
    peak, peak_kind = measured_peaks()
    n_pairs_cases = sum(1 for c in case_list if c[4])
    n_keys_cases = len(case_list) - n_pairs_cases
    post_bytes = args.steps * n * (n_keys_cases * 8 + n_pairs_cases * 16)
    achieved = post_bytes / (post_ms * 1e-3) / 1e9 if post_ms > 0 else None
    tr = profiled_traffic()
    roofline = {"kernel": "post-scan (k_postscan_tc for m <= 32, k_postscan beyond)", "bound": "hbm", "achieved": round(achieved, 1) if achieved else None,
                "peak": peak, "peak_kind": f"{peak_kind} (copy bandwidth, burst)", "unit": "GB/s",
                "frac": round(achieved / peak, 4) if achieved else None,
                "traffic": (round(tr["bytes_per_launch_full"], 0) if tr else None),
                "algorithmic_bytes_per_launch": post_bytes / max(1, n_ms),
                "stage_ms_per_step": {"prescan": round(pre_ms / args.steps, 4),
                                      "scan": round(scan_ms / args.steps, 4),
                                      "postscan": round(post_ms / args.steps, 4)}}

    result = {"metric": METRIC, "value": round(value, 3), "unit": "G elements/s (keys or pairs)",
              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
              "config": {"workload": WORKLOAD, "n": n, "cases": len(case_list),
                         "l2": "inputs (256 MB each) larger than L2; no flush",
                         "parallelism": "replicas" if world > 1 else "single"},
              # our kernels per multisplit: pre-scan (+ scan in its last CTA) and
              # post-scan for m <= 32; pre-scan, look-back scan, post-scan beyond
              "gpu_launches": sum(2 if c[3] <= 32 else 3 for c in case_list) * args.steps,
              "roofline": roofline, "sweep": per_case, "clocks": clk}

    if not args.no_e2e:
        result["e2e"] = e2e_gpu(args, ms, metrics, torch, dev, hk, hspl, hvals, case_list, specs, n, world)
    del dkeys, dk, dspl, dvals, out_k, out_v
    torch.cuda.empty_cache()
    if not args.no_extras:
        result["extras"] = extras_gpu(args, ms, metrics, torch, dev)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(hk, hspl, hvals, case_list, n, budget_s=args.cpu_budget)
    return result


def e2e_gpu(args, ms, metrics, torch, dev, hk, hspl, hvals, case_list, specs, n, world):
    """The same sweep through the C ABI with host buffers: each case copies its keys (and
    values) from pinned host memory, runs, and copies its outputs and offsets back into
    pinned host memory.  Cases rotate over `--e2e-lanes` streams, each with its own device
    and host buffers, so one case's copies overlap the others' kernels and copies (the
    usual multi-buffered pipeline a caller would write)."""
    pin = {}
    for cid, arr in hk.items():
        if id(arr) not in pin:
            pin[id(arr)] = torch.from_numpy(np.ascontiguousarray(arr).view(np.int32)).pin_memory()
    hkeys = {cid: pin[id(arr)] for cid, arr in hk.items()}
    hv = torch.from_numpy(hvals.view(np.int32)).pin_memory()
    lanes = []
    nl = max(1, args.e2e_lanes)
    for _ in range(nl):
        lanes.append({"stream": torch.cuda.Stream(device=dev),
                      "ho_k": torch.empty(n, dtype=torch.int32).pin_memory(),
                      "ho_v": torch.empty(n, dtype=torch.int32).pin_memory(),
                      "ho_off": torch.empty(257, dtype=torch.int32).pin_memory(),
                      "dk": torch.empty(n, dtype=torch.int32, device=dev),
                      "dv": torch.empty(n, dtype=torch.int32, device=dev),
                      "ok": torch.empty(n, dtype=torch.int32, device=dev),
                      "ov": torch.empty(n, dtype=torch.int32, device=dev),
                      "off": torch.empty(257, dtype=torch.int32, device=dev)})
    h2d = d2h = 0

    def step():
        nonlocal h2d, d2h
        for ci, (name, cid, kind, m, pairs) in enumerate(case_list):
            L = lanes[ci % nl]
            with torch.cuda.stream(L["stream"]):
                sptr = L["stream"].cuda_stream
                L["dk"].copy_(hkeys[cid], non_blocking=True)
                h2d += 4 * n
                if pairs:
                    L["dv"].copy_(hv, non_blocking=True)
                    h2d += 4 * n
                    st = ms.ms_multisplit_pairs(L["dk"].data_ptr(), L["dv"].data_ptr(), n, specs[name],
                                                L["ok"].data_ptr(), L["ov"].data_ptr(), L["off"].data_ptr(), sptr)
                else:
                    st = ms.ms_multisplit_keys(L["dk"].data_ptr(), n, specs[name], L["ok"].data_ptr(),
                                               L["off"].data_ptr(), sptr)
                if st != ms.MS_OK:
                    raise ms.MsError(st, name)
                L["ho_k"].copy_(L["ok"], non_blocking=True)
                d2h += 4 * n
                if pairs:
                    L["ho_v"].copy_(L["ov"], non_blocking=True)
                    d2h += 4 * n
                L["ho_off"][: m + 1].copy_(L["off"][: m + 1], non_blocking=True)
                d2h += 4 * (m + 1)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    h2d = d2h = 0
    steps = max(1, args.steps)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    main = torch.cuda.current_stream()
    t0.record(main)
    for L in lanes:
        L["stream"].wait_event(t0)
    for _ in range(steps):
        step()
    for L in lanes:
        ev = torch.cuda.Event()
        ev.record(L["stream"])
        main.wait_event(ev)
    t1.record(main)
    torch.cuda.synchronize()
    ms_total = t0.elapsed_time(t1)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    value = metrics.rate_g(n * len(case_list) * steps * world, ms_total * 1e-3)
    return {"value": round(value, 3), "unit": "G elements/s (keys or pairs)",
            "h2d_bytes_per_step": h2d // steps, "d2h_bytes_per_step": d2h // steps,
            "pipeline": f"{nl} streams, each with its own buffers (copies of one case overlap the others' kernels "
                        "and copies)"}


# ----------------------------------------------------------------------------- other configurations
def _time(torch, fn, reps: int, warmup: int = 2) -> float:
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def extras_gpu(args, ms, metrics, torch, dev):
    """The radix-sort and batched configurations, timed after the main step (not in `value`)."""
    peak, _ = measured_peaks()
    out = {}

    def dev_u32(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)

    # LSD radix sort: n = 2^28 keys (and pairs), 4 passes; n = 2^24 keys of 16 random bits, 2 passes
    for name, n, bits, pairs in (("sort_2p28_keys", 1 << 28, 32, False), ("sort_2p28_pairs", 1 << 28, 32, True),
                                 ("sort_2p24_16bit_keys", 1 << 24, 16, False),
                                 ("sort_2p24_16bit_pairs", 1 << 24, 16, True)):
        keys = dev_u32(synthetic.uniform_u32_bits(n, bits, 7) if bits < 32 else synthetic.uniform_u32(n, 7))
        vals = dev_u32(synthetic.uniform_u32(n, 8)) if pairs else None
        ko = torch.empty_like(keys)
        vo = torch.empty_like(keys) if pairs else None
        sptr = torch.cuda.current_stream().cuda_stream

        def run():
            st = ms.ms_radix_sort(keys.data_ptr(), vals.data_ptr() if pairs else None, n, 0, bits, ko.data_ptr(),
                                  vo.data_ptr() if pairs else None, sptr)
            if st != ms.MS_OK:
                raise ms.MsError(st, name)

        t = _time(torch, run, reps=5)
        passes = (bits + 7) // 8
        rate = metrics.rate_g(n, t * 1e-3)
        comp = metrics.sol_rate_g(peak, metrics.sort_compulsory_bytes_per_element(pairs, passes))
        out[name] = {"ms": round(t, 4), ("gpairs_s" if pairs else "gkeys_s"): round(rate, 2),
                     "frac_compulsory_roofline": round(rate / comp, 4), "passes": passes}
        del keys, vals, ko, vo
    torch.cuda.empty_cache()

    # radix width r = 4..8 (Section 6.3's sort table): n = 2^25, all 32 bits, ceil(32 / r) passes
    n = 1 << 25
    keys = dev_u32(synthetic.uniform_u32(n, 9))
    vals = dev_u32(synthetic.uniform_u32(n, 10))
    ko, vo = torch.empty_like(keys), torch.empty_like(keys)
    sptr = torch.cuda.current_stream().cuda_stream
    for pairs in (False, True):
        for r in (4, 5, 6, 7, 8):
            def run_r():
                st = ms.ms_radix_sort_r(keys.data_ptr(), vals.data_ptr() if pairs else None, n, 0, 32, r,
                                        ko.data_ptr(), vo.data_ptr() if pairs else None, sptr)
                if st != ms.MS_OK:
                    raise ms.MsError(st, f"sort r={r}")

            t = _time(torch, run_r, reps=5)
            rate = metrics.rate_g(n, t * 1e-3)
            out[f"sort_r{r}_2p25_{'pairs' if pairs else 'keys'}"] = {
                "ms": round(t, 4), ("gpairs_s" if pairs else "gkeys_s"): round(rate, 2), "passes": (32 + r - 1) // r}
    del keys, vals, ko, vo

    # more than 256 buckets (Section 6.3): two digit passes, n = 2^26 uniform keys
    n = 1 << 26
    keys_u = dev_u32(synthetic.uniform_u32(n, 51))
    keys_f = dev_u32(synthetic.uniform_f32_1000(n, 52))
    vals = dev_u32(synthetic.index_values(n))
    ko, vo = torch.empty_like(vals), torch.empty_like(vals)
    offs = torch.empty(65537, dtype=torch.int32, device=dev)
    sptr = torch.cuda.current_stream().cuda_stream
    for name, keys, spec in (("range_m1024", keys_u, ms.BucketSpec.range_u32(dev_u32(synthetic.range_splitters(1024, 53)))),
                             ("range_m65536", keys_u, ms.BucketSpec.range_u32(dev_u32(synthetic.range_splitters(65536, 54)))),
                             ("delta_f32_m65536", keys_f, ms.BucketSpec.delta_f32(65536, float(np.float32(1000.0) / np.float32(65536)))),
                             ("mod_m65535", keys_u, ms.BucketSpec.mod(65535))):
        cs = spec.c()
        for pairs in (False, True):
            def run_w():
                if pairs:
                    st = ms.ms_multisplit_pairs(keys.data_ptr(), vals.data_ptr(), n, cs, ko.data_ptr(),
                                                vo.data_ptr(), offs.data_ptr(), sptr)
                else:
                    st = ms.ms_multisplit_keys(keys.data_ptr(), n, cs, ko.data_ptr(), offs.data_ptr(), sptr)
                if st != ms.MS_OK:
                    raise ms.MsError(st, name)

            t = _time(torch, run_w, reps=5)
            rate = metrics.rate_g(n, t * 1e-3)
            comp = metrics.sol_rate_g(peak, metrics.compulsory_bytes_per_element(pairs))
            out[f"wide_{name}_{'pairs' if pairs else 'keys'}"] = {
                "ms": round(t, 4), ("gpairs_s" if pairs else "gkeys_s"): round(rate, 2),
                "frac_compulsory_roofline": round(rate / comp, 4), "passes": 2}
    del keys_u, keys_f, vals, ko, vo, offs
    torch.cuda.empty_cache()

    # device histogram (Section 7.3): n = 2^26, Range (range splitters) and Even (float32 delta) buckets
    n = 1 << 26
    hk = dev_u32(synthetic.uniform_u32(n, 31))
    hf = dev_u32(synthetic.uniform_f32_1000(n, 32))
    counts = torch.empty(256, dtype=torch.int32, device=dev)
    for m in (32, 256):
        for name, keys, spec in ((f"histogram_range_m{m}", hk, ms.BucketSpec.range_u32(dev_u32(synthetic.range_splitters(m, 33)))),
                                 (f"histogram_even_f32_m{m}", hf,
                                  ms.BucketSpec.delta_f32(m, float(np.float32(1000.0) / np.float32(m))))):
            cs = spec.c()
            sptr = torch.cuda.current_stream().cuda_stream

            def run_h():
                st = ms.ms_histogram(keys.data_ptr(), n, cs, counts.data_ptr(), sptr)
                if st != ms.MS_OK:
                    raise ms.MsError(st, name)

            t = _time(torch, run_h, reps=20)
            rate = metrics.rate_g(n, t * 1e-3)
            out[name] = {"ms": round(t, 4), "gkeys_s": round(rate, 2),
                         "frac_read_roofline": round(rate / metrics.sol_rate_g(peak, 4), 4)}
    del hk, hf, counts
    torch.cuda.empty_cache()

    # Section 6.4 / Table 6: delta buckets, m = 256, n = 2^25, uniform vs 0.25-uniform vs binomial B(255, 0.5)
    n = 1 << 25
    m = 256
    delta = float(np.float32(1000.0) / np.float32(m))
    spec = ms.BucketSpec.delta_f32(m, delta).c()
    vals = dev_u32(synthetic.index_values(n))
    ko, vo = torch.empty_like(vals), torch.empty_like(vals)
    offs = torch.empty(m + 1, dtype=torch.int32, device=dev)
    sptr = torch.cuda.current_stream().cuda_stream
    dist_rates = {}
    for dname, gen in (("uniform", lambda: synthetic.uniform_f32_1000(n, 41)),
                       ("0.25-uniform", lambda: synthetic.alpha_uniform_f32(n, m, delta, 0.25, 42)),
                       ("binomial", lambda: synthetic.binomial_f32(n, m, delta, 43))):
        keys = dev_u32(gen())
        for pairs in (False, True):
            def run_d():
                if pairs:
                    st = ms.ms_multisplit_pairs(keys.data_ptr(), vals.data_ptr(), n, spec, ko.data_ptr(),
                                                vo.data_ptr(), offs.data_ptr(), sptr)
                else:
                    st = ms.ms_multisplit_keys(keys.data_ptr(), n, spec, ko.data_ptr(), offs.data_ptr(), sptr)
                if st != ms.MS_OK:
                    raise ms.MsError(st, dname)

            t = _time(torch, run_d, reps=10)
            dist_rates[(dname, pairs)] = metrics.rate_g(n, t * 1e-3)
        del keys
    for (dname, pairs), rate in dist_rates.items():
        out[f"dist_delta_m256_{dname}_{'pairs' if pairs else 'keys'}"] = {
            ("gpairs_s" if pairs else "gkeys_s"): round(rate, 2),
            "speedup_vs_uniform": round(rate / dist_rates[("uniform", pairs)], 3)}
    del vals, ko, vo, offs
    torch.cuda.empty_cache()

    # batched: 4096 segments, sizes floor(2^U), U ~ U(8, 20), key mod 32, pairs (value = index)
    sizes = synthetic.segment_sizes(4096, 8, 20, 2024)
    total = int(sizes.sum())
    kall = dev_u32(synthetic.uniform_u32(total, 2025))
    vall = torch.empty_like(kall)
    ko_all, vo_all = torch.empty_like(kall), torch.empty_like(kall)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    for st_, n_ in zip(starts, sizes):  # value = index within the segment
        vall[int(st_):int(st_ + n_)] = torch.arange(int(n_), dtype=torch.int32, device=dev)
    offs = torch.empty((4096, 33), dtype=torch.int32, device=dev)
    spec = ms.BucketSpec.mod(32)
    segs = []
    for i, (st_, n_) in enumerate(zip(starts, sizes)):
        o = int(st_) * 4
        segs.append((kall.data_ptr() + o, vall.data_ptr() + o, ko_all.data_ptr() + o, vo_all.data_ptr() + o,
                     offs[i].data_ptr(), int(n_)))
    cs = spec.c()
    stc, plan = ms.ms_batch_plan_create(segs, cs)
    if stc != ms.MS_OK:
        raise ms.MsError(stc, "ms_batch_plan_create")
    sptr = torch.cuda.current_stream().cuda_stream
    try:
        t_graph = _time(torch, lambda: ms.ms_batch_run_graph(plan, sptr), reps=5)
        t_launch = _time(torch, lambda: ms.ms_batch_run(plan, sptr), reps=5)
        # outside the timed regions: the batched outputs must equal one plain launch per segment
        b_k, b_v, b_o = ko_all.clone(), vo_all.clone(), offs.clone()

        def plain():
            for (kin, vin, kout, vout, off, n_) in segs:
                st = ms.ms_multisplit_pairs(kin, vin, n_, cs, kout, vout, off, sptr)
                if st != ms.MS_OK:
                    raise ms.MsError(st, "plain")

        t_plain = _time(torch, plain, reps=2, warmup=1)
        torch.cuda.synchronize()
        if not (torch.equal(b_k, ko_all) and torch.equal(b_v, vo_all) and torch.equal(b_o, offs)):
            raise RuntimeError("batched outputs differ from the per-segment plain launches")
        del b_k, b_v, b_o
    finally:
        ms.ms_batch_plan_destroy(plan)
    comp = metrics.sol_rate_g(peak, metrics.compulsory_bytes_per_element(True))
    out["batched_4096_segments_mod32_pairs"] = {
        "total_pairs": total, "graph_ms": round(t_graph, 3), "launch_ms": round(t_launch, 3),
        "plain_per_segment_ms": round(t_plain, 3),
        "gpairs_s_graph": round(metrics.rate_g(total, t_graph * 1e-3), 2),
        "gpairs_s_plain": round(metrics.rate_g(total, t_plain * 1e-3), 2),
        "speedup_vs_plain": round(t_plain / t_graph, 2), "equal_to_plain": True,
        "frac_compulsory_roofline_graph": round(metrics.rate_g(total, t_graph * 1e-3) / comp, 4)}
    del kall, vall, ko_all, vo_all, offs
    torch.cuda.empty_cache()

    # serving: Poisson arrivals of multisplit and sort requests, continuous batching
    if args.serve_seconds > 0:
        from paper_1701_01189_gb300 import serving

        out["serving"] = serving.run_config(seconds=args.serve_seconds)
    if ms.device_status() != ms.MS_OK:
        raise RuntimeError("device status not OK after the extras")
    return out


# ----------------------------------------------------------------------------- CPU oracle
def _oracle_spec(kind, m, hspl):
    import oracle

    if kind == "range":
        return oracle.Spec(oracle.RANGE_U32, m, splitters=hspl[m])
    return oracle.Spec(oracle.DELTA_F32, m, x0=0.0, delta=float(np.float32(1000.0) / np.float32(m)))


def oracle_sample(hk, hspl, hvals, case_list, sample_n: int, parallel: bool = False):
    """Runs the oracle (or, with parallel, the all-core CPU baseline) on the
    first sample_n elements of every case; returns (elements, seconds)."""
    import oracle

    fn = oracle.multisplit_parallel if parallel else oracle.multisplit
    elems, secs = 0, 0.0
    for name, cid, kind, m, pairs in case_list:
        keys = hk[cid][:sample_n]
        vals = hvals[:sample_n] if pairs else None
        spec = _oracle_spec(kind, m, hspl)
        t = time.perf_counter()
        fn(keys, vals, spec)
        secs += time.perf_counter() - t
        elems += len(keys)
    return elems, secs


def host_cpu():
    """(cores this process may use, CPU model string) of the host."""
    import oracle

    model = ""
    try:
        fields = {}
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                fields.setdefault(k.strip(), v.strip())
        model = fields.get("Model name") or fields.get("Vendor ID", "")
    except Exception:  # noqa: BLE001 -- lscpu missing: fall back to /proc/cpuinfo
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return oracle.host_threads(), model or platform.machine()


def cpu_baseline(hk, hspl, hvals, case_list, n, budget_s: float = 15.0):
    """The single-threaded oracle and the all-core CPU baseline, each on a
    sample calibrated to about budget_s seconds (half the budget each)."""
    import oracle

    cores, model = host_cpu()

    def calibrated(parallel, budget):
        e, s = oracle_sample(hk, hspl, hvals, case_list, 1 << 16, parallel)
        per_elem = s / max(1, e)
        sample_n = int(min(n, max(1 << 16, budget / max(per_elem, 1e-12) / len(case_list))))
        sample_n = 1 << max(16, int(np.floor(np.log2(sample_n))))
        e, s = oracle_sample(hk, hspl, hvals, case_list, sample_n, parallel)
        return e, s, sample_n

    e, s, sample_n = calibrated(False, budget_s / 2)
    pe, ps, psample = calibrated(True, budget_s / 2)
    return {"value": round(e / s / 1e9, 5), "unit": "G elements/s (keys or pairs)", "cores": 1,
            "kind": "oracle", "seconds": round(s, 2),
            "sample": f"each of the {len(case_list)} sweep cases on its first {sample_n} elements "
                      f"(single-threaded C oracle, Eq. 1 by counting)",
            "host": {"nproc": os.cpu_count(), "usable_cores": cores, "cpu_model": model},
            "all_core": {"value": round(pe / ps / 1e9, 5), "unit": "G elements/s (keys or pairs)",
                         "cores": min(cores, 256), "kind": "all-core C baseline (POSIX threads: chunk "
                         "histograms, bucket-major scan, stable scatter per chunk), bit-exact vs the oracle",
                         "seconds": round(ps, 2),
                         "sample": f"each of the {len(case_list)} sweep cases on its first {psample} elements"}}


def run_reference(args):
    """The reference arm: the CPU oracle on bounded samples of the same workload."""
    n = 1 << args.n_log2
    sample_n = min(n, 1 << args.ref_sample_log2)
    hk, hspl, hvals = make_inputs(sample_n)
    case_list = cases(args.n_log2)
    for _ in range(args.warmup):
        oracle_sample(hk, hspl, hvals, case_list, sample_n)
    e_tot, s_tot = 0, 0.0
    for _ in range(args.steps):
        e, s = oracle_sample(hk, hspl, hvals, case_list, sample_n)
        e_tot += e
        s_tot += s
    value = e_tot / s_tot / 1e9
    desc = (f"each step: the {len(case_list)} sweep cases on {sample_n} elements each "
            f"(single-threaded C oracle)")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5),
            "unit": "G elements/s (keys or pairs)", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * s_tot / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "cases": len(case_list), "sample_n": sample_n},
            "cpu_baseline": {"value": round(value, 5), "unit": "G elements/s (keys or pairs)", "cores": 1,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 5), "unit": "G elements/s (keys or pairs)", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ms", choices=["ms", "reference"])
    ap.add_argument("--n-log2", type=int, default=26)
    ap.add_argument("--ref-sample-log2", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-lanes", type=int, default=3, help="streams (each with its own buffers) of the e2e pipeline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                    help="where the nvidia-smi clock samples of the timed region are written")
    ap.add_argument("--no-extras", action="store_true", help="skip the radix-sort, batched and serving configurations")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="length of the serving trace (0: skip)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    import torch

    if world > 1:
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    if args.warmup < 3:
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    res = run_gpu(args, rank, world)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
