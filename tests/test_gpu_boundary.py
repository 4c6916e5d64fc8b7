"""The two calls of the C ABI that complete the boundary: the one-call
batched multisplit over segment descriptors in device memory, and
ms_shutdown.  Every result is compared with the CPU oracle bit for bit."""
import gc

import numpy as np
import pytest

import oracle
import synthetic
from parity import Case, to_dev, to_host

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 31, 4095, 4096, 4097, 10000, 3 * 4096 + 5, 70000, 255, 2, 200_003]


def _segments(sizes, seed, pairs, case):
    keys = [synthetic.uniform_f32_1000(n, seed + i) if case.kind == oracle.DELTA_F32 else
            synthetic.uniform_u32(n, seed + i) for i, n in enumerate(sizes)]
    vals = [synthetic.index_values(n) for n in sizes] if pairs else None
    return keys, vals


def _run_batched(ms, torch, keys, vals, case, spec, contiguous_offsets):
    """Builds device inputs and outputs, copies the descriptors to the device
    and makes the one call.  Returns (status, keys_out, vals_out, offsets)."""
    dk = [to_dev(k) for k in keys]
    dv = [to_dev(v) for v in vals] if vals is not None else None
    ko = [torch.full_like(t, -1) for t in dk]
    vo = [torch.full_like(t, -1) for t in dv] if dv is not None else None
    m1 = case.m + 1
    offs_all = torch.full((len(keys), m1), -1, dtype=torch.int32, device="cuda")
    offs_own = [torch.full((m1,), -1, dtype=torch.int32, device="cuda") for _ in keys]
    recs = []
    for i in range(len(keys)):
        recs.append((dk[i].data_ptr(), dv[i].data_ptr() if dv is not None else None, ko[i].data_ptr(),
                     vo[i].data_ptr() if vo is not None else None, offs_own[i].data_ptr(), int(dk[i].numel())))
    raw = np.frombuffer(ms.segment_records(recs), dtype=np.uint8).copy()
    d_recs = torch.from_numpy(raw).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    st = ms.ms_multisplit_pairs_batched(d_recs.data_ptr(), len(keys), spec.c(),
                                        offs_all.data_ptr() if contiguous_offsets else None, stream)
    torch.cuda.synchronize()
    offs = [offs_all[i] for i in range(len(keys))] if contiguous_offsets else offs_own
    return st, ko, vo, offs


def _check(keys, vals, case, ko, vo, offs):
    for i, k in enumerate(keys):
        ek, ev, eoff = oracle.multisplit(k, None if vals is None else vals[i], case.oracle_spec())
        np.testing.assert_array_equal(to_host(ko[i]), ek, err_msg=f"segment {i} n={len(k)}")
        if vals is not None:
            np.testing.assert_array_equal(to_host(vo[i]), ev, err_msg=f"segment {i} values")
        np.testing.assert_array_equal(to_host(offs[i]).astype(np.uint64), eoff, err_msg=f"segment {i} offsets")


CASES = [Case(oracle.MOD, 32), Case(oracle.RANGE_U32, 256, splitters=synthetic.range_splitters(256, 7)),
         Case(oracle.DELTA_F32, 8, x0=0.0, delta=float(np.float32(1000.0) / np.float32(8)))]


@pytest.mark.parametrize("pairs", [True, False], ids=["pairs", "keys"])
@pytest.mark.parametrize("ci", range(len(CASES)), ids=["mod32", "range256", "delta8"])
def test_one_call_batched_matches_oracle(ci, pairs):
    import torch

    import paper_1701_01189_gb300 as ms

    case = CASES[ci]
    spec = case.gpu_spec()
    keys, vals = _segments(SIZES, 300 + ci, pairs, case)
    # contiguous offsets array, then each descriptor's own offsets; the second
    # and third calls reuse the library's cached plan, the fourth (more
    # segments and elements) makes it grow
    for contiguous in (True, False, True):
        st, ko, vo, offs = _run_batched(ms, torch, keys, vals, case, spec, contiguous)
        assert st == ms.MS_OK
        assert ms.device_status() == ms.MS_OK
        _check(keys, vals, case, ko, vo, offs)
    more = SIZES * 8 + [1 << 20]
    keys2, vals2 = _segments(more, 900 + ci, pairs, case)
    st, ko, vo, offs = _run_batched(ms, torch, keys2, vals2, case, spec, True)
    assert st == ms.MS_OK and ms.device_status() == ms.MS_OK
    _check(keys2, vals2, case, ko, vo, offs)


def test_one_call_batched_argument_errors():
    import torch

    import paper_1701_01189_gb300 as ms

    spec = Case(oracle.MOD, 8).gpu_spec()
    stream = torch.cuda.current_stream().cuda_stream
    assert ms.ms_multisplit_pairs_batched(None, 3, spec.c(), None, stream) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_multisplit_pairs_batched(None, 0, spec.c(), None, stream) == ms.MS_OK
    bad = ms._binding._Spec(ms.MOD, 0, None, 0.0, 1.0, 0, 0)
    assert ms.ms_multisplit_pairs_batched(None, 0, bad, None, stream) == ms.MS_ERR_INVALID_ARG
    # keys-only and key-value segments mixed in one call
    a = torch.zeros(64, dtype=torch.int32, device="cuda")
    recs = [(a.data_ptr(), a.data_ptr() + 64, a.data_ptr() + 128, a.data_ptr() + 192, None, 4),
            (a.data_ptr(), None, a.data_ptr() + 128, None, None, 4)]
    d = torch.from_numpy(np.frombuffer(ms.segment_records(recs), dtype=np.uint8).copy()).cuda()
    assert ms.ms_multisplit_pairs_batched(d.data_ptr(), 2, spec.c(), None, stream) == ms.MS_ERR_INVALID_ARG


def test_shutdown_releases_and_calls_start_afresh():
    import torch

    import paper_1701_01189_gb300 as ms

    gc.collect()  # plans of earlier tests that were dropped without close()
    torch.cuda.synchronize()
    case = Case(oracle.RANGE_U32, 32, splitters=synthetic.range_splitters(32, 11))
    keys = synthetic.uniform_u32(300_000, 12)
    vals = synthetic.index_values(300_000)
    ek, ev, eoff = oracle.multisplit(keys, vals, case.oracle_spec())

    def one_call():
        ko, vo, off = ms.multisplit_pairs(to_dev(keys), to_dev(vals), case.gpu_spec())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_host(ko), ek)
        np.testing.assert_array_equal(to_host(vo), ev)
        np.testing.assert_array_equal(to_host(off).astype(np.uint64), eoff)

    one_call()
    # a batch plan made by the caller keeps the library state: refused
    plan = ms.BatchPlan([to_dev(keys[:5000])], None, ms.BucketSpec.mod(4))
    assert ms.ms_shutdown() == ms.MS_ERR_INVALID_ARG
    plan.close()
    one_call()
    assert ms.ms_shutdown() == ms.MS_OK
    assert ms.ms_shutdown() == ms.MS_OK  # twice is fine
    one_call()  # the state is created again
    assert ms.device_status() == ms.MS_OK
    # the one-call batched path also starts afresh after a shutdown
    spec = Case(oracle.MOD, 32).gpu_spec()
    ks, vs = _segments([5000, 70000], 5, True, Case(oracle.MOD, 32))
    st, ko, vo, offs = _run_batched(ms, torch, ks, vs, Case(oracle.MOD, 32), spec, True)
    assert st == ms.MS_OK
    _check(ks, vs, Case(oracle.MOD, 32), ko, vo, offs)
    assert ms.ms_shutdown() == ms.MS_OK
    one_call()
