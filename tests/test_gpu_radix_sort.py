"""GPU parity of the multisplit radix sort (Section 7.1) against the oracle's
stable sort by key bits, bit exact; full-size cases are checked through
properties that pin the unique stable result (sorted keys, keys_out =
keys_in[vals_out] with vals = original index, vals increasing inside runs of
equal keys)."""
import numpy as np
import pytest

import oracle
import synthetic
from parity import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300.build import build

    build()
    ms.lib()


def gpu_sort(keys, vals, b, e):
    import paper_1701_01189_gb300 as ms
    import torch

    dk = to_dev(keys)
    dv = to_dev(vals) if vals is not None else None
    ko, vo = ms.radix_sort(dk, dv, b, e)
    torch.cuda.synchronize()
    assert ms.device_status() == ms.MS_OK
    return to_host(ko), (None if vo is None else to_host(vo))


@pytest.mark.parametrize("bits", [(0, 32), (0, 16), (0, 8), (0, 0), (4, 28), (3, 30), (8, 9), (0, 31),
                                  (1, 32), (16, 32)])
@pytest.mark.parametrize("n", [0, 1, 33, 4097, 100_000, 1 << 20])
def test_sort_matches_oracle(bits, n):
    b, e = bits
    keys = synthetic.uniform_u32(n, n + b * 64 + e)
    vals = synthetic.uniform_u32(n, n + 7)
    gk, gv = gpu_sort(keys, vals, b, e)
    ok, ov = oracle.radix_sort(keys, vals, b, e)
    np.testing.assert_array_equal(gk, ok)
    np.testing.assert_array_equal(gv, ov)
    gk2, gv2 = gpu_sort(keys, None, b, e)
    assert gv2 is None
    np.testing.assert_array_equal(gk2, ok)


def test_sort_duplicates():
    n = 300_000
    keys = synthetic.uniform_u32_bits(n, 6, 3) * np.uint32(0x01010101)
    vals = synthetic.index_values(n)
    gk, gv = gpu_sort(keys, vals, 0, 32)
    ok, ov = oracle.radix_sort(keys, vals, 0, 32)
    np.testing.assert_array_equal(gk, ok)
    np.testing.assert_array_equal(gv, ov)


def test_config_16bit_2p24():
    """n = 2^24 keys with 16 random low bits, bits [0, 16): 2 passes."""
    n = 1 << 24
    keys = synthetic.uniform_u32_bits(n, 16, 11)
    vals = synthetic.uniform_u32(n, 12)
    gk, gv = gpu_sort(keys, vals, 0, 16)
    ok, ov = oracle.radix_sort(keys, vals, 0, 16)
    np.testing.assert_array_equal(gk, ok)
    np.testing.assert_array_equal(gv, ov)


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
def test_config_2p28(pairs):
    """n = 2^28 uniform keys, 4 passes of 8-bit digits."""
    n = 1 << 28
    keys = synthetic.uniform_u32(n, 21)
    vals = synthetic.index_values(n) if pairs else None
    gk, gv = gpu_sort(keys, vals, 0, 32)
    assert np.all(gk[1:] >= gk[:-1])
    if pairs:
        seen = np.zeros(n, dtype=bool)
        seen[gv] = True
        assert seen.all()  # n indices, all distinct: a permutation
        np.testing.assert_array_equal(gk, keys[gv])  # each key travels with its value
        same = gk[1:] == gk[:-1]
        assert np.all(gv[1:][same] > gv[:-1][same])  # stable among equal keys
    else:
        np.testing.assert_array_equal(gk, np.sort(keys))


@pytest.mark.parametrize("rank", [1, 3], ids=["peer-tables", "ballot-peers"])
@pytest.mark.parametrize("n", [4097, (1 << 20) + 5, (1 << 22) + 3])
def test_sort_rank_modes(rank, n):
    """Both ways the one-sweep passes can rank 8-bit digits (selected by the
    tuning entry of radix-digit multisplits with 256 buckets), keys and pairs."""
    import paper_1701_01189_gb300 as ms

    keys = synthetic.uniform_u32(n, 71)
    vals = synthetic.index_values(n)
    try:
        for pairs in (0, 1):
            assert ms.ms_tune_set(ms.RADIX, pairs, 8, ms.ms_tune_size_class(n), 0, rank, 1) == ms.MS_OK
        ek, ev = oracle.radix_sort(keys, vals, 0, 32)
        gk, gv = gpu_sort(keys, vals, 0, 32)
        np.testing.assert_array_equal(gk, ek)
        np.testing.assert_array_equal(gv, ev)
        gk2, _ = gpu_sort(keys, None, 0, 32)
        np.testing.assert_array_equal(gk2, ek)
    finally:
        ms.ms_tune_reset()


@pytest.mark.parametrize("bits", [(0, 32), (0, 16), (3, 30)])
@pytest.mark.parametrize("n", [1, 4097, (1 << 20) + 5, (1 << 22) + 3])
def test_sort_by_multisplit_passes(bits, n):
    """The sort made of three-stage multisplit passes (tuning method 1), keys
    and pairs, against the oracle."""
    import paper_1701_01189_gb300 as ms

    keys = synthetic.uniform_u32(n, 91)
    vals = synthetic.index_values(n)
    try:
        for pairs in (0, 1):
            assert ms.ms_tune_set_sort(pairs, ms.ms_tune_size_class(n), 1) == ms.MS_OK
        ek, ev = oracle.radix_sort(keys, vals, *bits)
        gk, gv = gpu_sort(keys, vals, *bits)
        np.testing.assert_array_equal(gk, ek)
        np.testing.assert_array_equal(gv, ev)
        gk2, _ = gpu_sort(keys, None, *bits)
        np.testing.assert_array_equal(gk2, ek)
    finally:
        ms.ms_tune_reset()


@pytest.mark.parametrize("r", [1, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("bits", [(0, 32), (3, 30), (0, 16)])
@pytest.mark.parametrize("n", [1, 4097, (1 << 20) + 5])
def test_sort_with_r_bit_digits(r, bits, n):
    """The sort in r-bit digits (ceil(width / r) passes, the last one taking the
    bits left over), keys and pairs, against the oracle."""
    import paper_1701_01189_gb300 as ms
    import torch

    keys = synthetic.uniform_u32(n, 17 * r + n)
    vals = synthetic.index_values(n)
    ek, ev = oracle.radix_sort(keys, vals, *bits)
    ko, vo = ms.radix_sort(to_dev(keys), to_dev(vals), *bits, r=r)
    ko2, _ = ms.radix_sort(to_dev(keys), None, *bits, r=r)
    torch.cuda.synchronize()
    assert ms.device_status() == ms.MS_OK
    np.testing.assert_array_equal(to_host(ko), ek)
    np.testing.assert_array_equal(to_host(vo), ev)
    np.testing.assert_array_equal(to_host(ko2), ek)
