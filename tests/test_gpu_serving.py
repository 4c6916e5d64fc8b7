"""Serving: requests that arrive while others are on the GPU are batched into
the persistent kernel on several streams, and every result equals the CPU
oracle's result on that request alone and the plain entry point's (bit
exact)."""
import numpy as np
import pytest

import oracle
import synthetic
from parity import to_dev, to_host

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    import torch

    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300 import serving

    pool = 1 << 20
    hk, hv = synthetic.uniform_u32(pool, 1), synthetic.uniform_u32(pool, 2)
    pk, pv = to_dev(hk), to_dev(hv)
    hspl = {m: synthetic.range_splitters(m, m) for m in (8, 32, 256)}
    spl = {m: to_dev(t) for m, t in hspl.items()}
    trace = serving.make_trace(3000, 0.15, 5, pool=pool, n_lo=6, n_hi=18)
    svc = serving.Service(pk, pv, spl, arena_bytes=64 << 20, slots=3, max_batch_segments=64,
                          max_batch_elements=1 << 21, plain_min_elements=1 << 15)
    got = {}

    def keep(r):  # called when r's results are ready, before its memory is reused
        ko, vo = svc.out_views(r)
        got[r.rid] = (to_host(ko), to_host(vo))

    summary = svc.serve(trace, real_time=True, on_complete=keep)
    assert summary["requests"] == len(trace) == len(got)
    assert ms.device_status() == ms.MS_OK
    specs = {m: ms.BucketSpec.range_u32(t) for m, t in spl.items()}
    checked = batched_sorts = 0
    for r in trace:
        got_k, got_v = got[r.rid]
        what = f"request {r.rid} {r.kind} m={r.m} n={r.n}"
        # the CPU oracle on the request's input alone
        hkin, hvin = hk[r.in_off:r.in_off + r.n], hv[r.in_off:r.in_off + r.n]
        if r.kind == "multisplit":
            ok, ov, _ = oracle.multisplit(hkin, hvin, oracle.Spec(oracle.RANGE_U32, r.m, splitters=hspl[r.m]))
        else:
            ok, ov = oracle.radix_sort(hkin, hvin, 0, 32)
            batched_sorts += r.n < (1 << 15)  # the four batched digit passes
        np.testing.assert_array_equal(got_k, ok, err_msg=what + " vs oracle")
        np.testing.assert_array_equal(got_v, ov, err_msg=what + " values vs oracle")
        # and the plain entry point on the same request alone
        kin = pk[r.in_off:r.in_off + r.n]
        vin = pv[r.in_off:r.in_off + r.n]
        if r.kind == "multisplit":
            ek, ev, _ = ms.multisplit_pairs(kin, vin, specs[r.m])
        else:
            ek, ev = ms.radix_sort(kin, vin, 0, 32)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got_k, to_host(ek), err_msg=what)
        np.testing.assert_array_equal(got_v, to_host(ev))
        checked += 1
    assert checked == len(trace)
    assert batched_sorts > 0
    assert any(r.n >= 1 << 15 for r in trace) and any(r.n < 1 << 15 for r in trace)  # both paths ran
    svc.close()


def test_serial_baseline_runs():
    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300 import serving

    pool = 1 << 18
    pk = to_dev(synthetic.uniform_u32(pool, 3))
    pv = to_dev(synthetic.uniform_u32(pool, 4))
    spl = {m: to_dev(synthetic.range_splitters(m, m)) for m in (8, 32, 256)}
    trace = serving.make_trace(2000, 0.05, 6, pool=pool, n_lo=6, n_hi=16)
    summary = serving.serve_serial(trace, pk, pv, spl, real_time=True)
    assert summary["requests"] == len(trace) and summary["p99_ms"] >= summary["p50_ms"]
    assert ms.device_status() == ms.MS_OK
