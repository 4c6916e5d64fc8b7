"""The keys-only multisplit variant that allocates no device memory.

Who needs it: callers that cannot let a library allocate while they enqueue
work -- hot loops where allocator calls are forbidden, and processes whose
device memory is owned by another allocator.  ms_multisplit_keys_noalloc takes
its scratch from a fixed array inside the library instead.

This file is collected last on purpose.  It calls the variant through the C
ABI twice in a row (the second call reuses the fixed array exactly as the first
one left it) and checks both results bit for bit against ms_multisplit_keys,
the entry point that allocates its scratch from the library pool, and against
the CPU oracle; it also checks that the calls leave the device's free memory
unchanged.  A bounded wait made to run out on this path is reported by
ms_noalloc_status and does not disturb the calls after it.  It passes both
alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import oracle
import synthetic
from parity import Case, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [
    Case(oracle.RANGE_U32, 32, splitters=synthetic.range_splitters(32, 5)),
    Case(oracle.RADIX, 256, shift=8, bits=8),
    Case(oracle.MOD, 7),
    Case(oracle.DELTA_F32, 64, x0=0.0, delta=float(np.float32(1000.0) / np.float32(64))),
]


@pytest.mark.parametrize("case", CASES, ids=["range32", "radix256", "mod7", "delta64"])
def test_noalloc_matches_pooled_entry_point_twice(case):
    import torch

    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300.build import build

    build()
    n = (1 << 22) + 17
    keys = synthetic.uniform_f32_1000(n, 9) if case.kind == oracle.DELTA_F32 else synthetic.uniform_u32(n, 9)
    spec = case.gpu_spec()
    stream = torch.cuda.current_stream().cuda_stream
    dk = to_dev(keys)
    ref_k = torch.empty_like(dk)
    ref_off = torch.empty(case.m + 1, dtype=torch.int32, device="cuda")
    assert ms.ms_multisplit_keys(dk.data_ptr(), n, spec.c(), ref_k.data_ptr(), ref_off.data_ptr(), stream) == ms.MS_OK
    out_k = torch.empty_like(dk)
    out_off = torch.empty(case.m + 1, dtype=torch.int32, device="cuda")
    expect_k, expect_off = to_host(ref_k), to_host(ref_off)

    def call_and_copy_back():
        out_k.fill_(0)
        out_off.fill_(-1)
        st = ms.ms_multisplit_keys_noalloc(dk.data_ptr(), n, spec.c(), out_k.data_ptr(), out_off.data_ptr(), stream)
        torch.cuda.synchronize()
        return st, to_host(out_k), to_host(out_off)

    # The first call on this device looks up the fixed array and sets up the
    # kernels; it also warms up the torch operations used around the calls, so
    # the free-memory reading below sees only what the calls themselves do.
    st, k0, o0 = call_and_copy_back()
    assert st == ms.MS_OK
    free_before, _ = torch.cuda.mem_get_info()
    results = [call_and_copy_back() for _ in range(2)]
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    ok, _, ooff = oracle.multisplit(keys, None, case.oracle_spec())
    np.testing.assert_array_equal(expect_k, ok)
    for st, k, o in [(st, k0, o0)] + results:
        assert st == ms.MS_OK
        np.testing.assert_array_equal(k, expect_k)
        np.testing.assert_array_equal(o, expect_off)
        np.testing.assert_array_equal(k, ok)
        np.testing.assert_array_equal(o.astype(np.uint64), ooff)
    assert ms.ms_noalloc_status(stream) == ms.MS_OK  # this path's own status word
    assert ms.device_status() == ms.MS_OK  # the pooled path's, untouched


@pytest.mark.parametrize("case", [CASES[0], CASES[1]], ids=["range32", "radix256"])
def test_noalloc_expired_wait_is_reported_and_later_calls_are_exact(case):
    """An expired bounded wait on this path (a look-back wait on a status word
    that nothing publishes) sets the timeout bit in the fixed array's header.
    The next call must still wait its full bound and be exact (with 32 buckets
    its post-scan waits on copy barriers, with 256 on the look-back scan), and
    ms_noalloc_status must report the timeout once, then clear."""
    import torch

    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300.build import build

    build()
    stream = torch.cuda.current_stream().cuda_stream
    n = (1 << 21) + 5
    keys = synthetic.uniform_u32(n, 21)
    ok, _, ooff = oracle.multisplit(keys, None, case.oracle_spec())
    spec = case.gpu_spec()
    dk = to_dev(keys)
    out_k = torch.empty_like(dk)
    out_off = torch.empty(case.m + 1, dtype=torch.int32, device="cuda")
    assert ms.ms_noalloc_status(stream) == ms.MS_OK
    for read_status_between in (False, True):
        assert ms.ms_test_expire_lookback_noalloc(stream) == ms.MS_OK
        if read_status_between:
            assert ms.ms_noalloc_status(stream) == ms.MS_ERR_TIMEOUT
        for _ in range(2):
            out_k.fill_(0)
            st = ms.ms_multisplit_keys_noalloc(dk.data_ptr(), n, spec.c(), out_k.data_ptr(), out_off.data_ptr(),
                                               stream)
            assert st == ms.MS_OK
            torch.cuda.synchronize()
            np.testing.assert_array_equal(to_host(out_k), ok)
            np.testing.assert_array_equal(to_host(out_off).astype(np.uint64), ooff)
        expect = ms.MS_OK if read_status_between else ms.MS_ERR_TIMEOUT
        assert ms.ms_noalloc_status(stream) == expect
        assert ms.ms_noalloc_status(stream) == ms.MS_OK  # reading clears it
    assert ms.device_status() == ms.MS_OK


def test_noalloc_argument_errors():
    import paper_1701_01189_gb300 as ms

    spec = Case(oracle.MOD, 8).gpu_spec()
    assert ms.ms_multisplit_keys_noalloc(0x1000, 16, spec.c(), 0x1000, 0, None) == ms.MS_ERR_INVALID_ARG
    bad = ms._binding._Spec(ms.MOD, 0, None, 0.0, 1.0, 0, 0)
    assert ms.ms_multisplit_keys_noalloc(0x1000, 16, bad, 0x2000, 0, None) == ms.MS_ERR_INVALID_ARG
