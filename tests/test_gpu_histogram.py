"""GPU parity of the device histogram (Section 7.3: Even histogram = float32
delta buckets, Range histogram = range splitters; radix and mod buckets too)
against the CPU oracle's histogram, bit exact, through the C ABI."""
import numpy as np
import pytest

import oracle
import synthetic
from parity import Case, to_dev, to_host

pytestmark = pytest.mark.gpu


def gpu_hist(keys, case):
    import torch

    import paper_1701_01189_gb300 as ms

    counts = ms.histogram(to_dev(keys), case.gpu_spec())
    torch.cuda.synchronize()
    assert ms.device_status() == ms.MS_OK
    return to_host(counts).astype(np.int64)


def cases(m, seed):
    out = [Case(oracle.RANGE_U32, m, splitters=synthetic.range_splitters(m, seed)), Case(oracle.MOD, m),
           Case(oracle.DELTA_F32, m, x0=0.0, delta=float(np.float32(1000.0) / np.float32(m)))]
    if m & (m - 1) == 0:
        bits = m.bit_length() - 1
        out.append(Case(oracle.RADIX, m, shift=32 - max(bits, 1) if bits else 0, bits=bits))
    return out


@pytest.mark.parametrize("m", [1, 2, 3, 8, 31, 32, 33, 64, 255, 256])
@pytest.mark.parametrize("n", [0, 1, 33, 4095, 4097, 3 * 4096 + 5, 1 << 20])
def test_histogram_matches_oracle(m, n):
    for case in cases(m, 5 + m):
        keys = synthetic.uniform_f32_1000(n, 9) if case.kind == oracle.DELTA_F32 else synthetic.uniform_u32(n, 9)
        want = oracle.histogram(keys, case.oracle_spec()).astype(np.int64)
        got = gpu_hist(keys, case)
        np.testing.assert_array_equal(got, want, err_msg=f"kind {case.kind} m {m} n {n}")
        assert got.sum() == n


@pytest.mark.parametrize("m", [2, 32, 256])
def test_histogram_full_size_skewed(m):
    """n = 2^26 keys, skewed (geometric bucket ids): every count bit exact."""
    spl = synthetic.range_splitters(m, 1000 + m)
    keys = synthetic.skewed_u32(1 << 26, spl, 3000 + m)
    case = Case(oracle.RANGE_U32, m, splitters=spl)
    np.testing.assert_array_equal(gpu_hist(keys, case), oracle.histogram(keys, case.oracle_spec()).astype(np.int64))
