"""GPU parity of multisplit with more than 256 buckets (Section 6.3, larger
multisplits): two passes over the 8-bit digits of the bucket id, then the
bucket offsets by bisection.  Every case is compared bit for bit with the
oracle, which evaluates Eq. 1 directly for any m.  Sizes span several tiles
and ragged tails; cases cover m just above 256, super-bucket boundaries
(m = 8192, 8193), the largest m (65536), skewed keys, duplicated splitters,
keys on splitters, float32 special values and key mod m near its multiples."""
import numpy as np
import pytest

import oracle
import synthetic
from parity import Case, check_multisplit, clustered_splitters, range_case, run_gpu

pytestmark = pytest.mark.gpu

SIZES = [1, 33, 4097, 3 * 4096 + 17, (1 << 20) + 77]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300.build import build

    build()
    ms.lib()


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("m", [257, 300, 1000, 4096, 8192, 8193, 65536])
def test_wide_range_sizes(m, pairs):
    case = range_case(m, 11 + m)
    for i, n in enumerate(SIZES):
        keys = synthetic.uniform_u32(n, 500 + i)
        vals = synthetic.index_values(n) if pairs else None
        check_multisplit(keys, vals, case)


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("m", [300, 1000, 20000])
def test_wide_range_skewed(m, pairs):
    spl = synthetic.range_splitters(m, 21)
    n = 300_007
    keys = synthetic.skewed_u32(n, spl, 22)
    vals = synthetic.index_values(n) if pairs else None
    check_multisplit(keys, vals, Case(oracle.RANGE_U32, m, splitters=spl))


@pytest.mark.parametrize("m", [257, 513, 5000, 65536])
def test_wide_range_duplicate_splitters_and_boundaries(m):
    spl = synthetic.range_splitters(m, 31)
    spl[200:700] = spl[200]  # a run of equal splitters across super-bucket edges: empty buckets
    spl[m // 2:m // 2 + 3] = spl[m // 2]
    spl = np.sort(spl)
    keys = np.concatenate([spl, spl - np.uint32(1), spl + np.uint32(1), np.array([0, 0xFFFFFFFF], np.uint32),
                           synthetic.uniform_u32(20000, 32)])
    keys = keys[synthetic.rng(33).permutation(len(keys))]
    check_multisplit(keys, synthetic.index_values(len(keys)), Case(oracle.RANGE_U32, m, splitters=spl))


@pytest.mark.parametrize("m", [300, 5000, 65536])
def test_wide_range_clustered_splitters(m):
    # clusters of 1 to 7 splitters within 4096: lookup-table cells with 0, 1, a few or many
    spl = clustered_splitters(m, 34 + m)
    g = synthetic.rng(35)
    near = spl.astype(np.int64)[g.integers(0, m - 1, size=50000)] + g.integers(-4096, 4096, size=50000)
    keys = np.concatenate([spl, spl - np.uint32(1), spl + np.uint32(1), np.clip(near, 0, 0xFFFFFFFF).astype(np.uint32),
                           synthetic.uniform_u32(50000, 36)])
    keys = keys[g.permutation(len(keys))]
    check_multisplit(keys, synthetic.index_values(len(keys)), Case(oracle.RANGE_U32, m, splitters=spl))


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("m", [257, 1000, 4096, 65536])
def test_wide_delta(m, pairs):
    delta = float(np.float32(1000.0) / np.float32(m))
    special = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0xBF800000, 0x00000001,
                        0x447A0000, 0x4479FFFF], np.uint32)  # 0, -0, +inf, -inf, NaN, -1, subnormal, 1000, <1000
    for i, n in enumerate(SIZES):
        keys = np.concatenate([special, synthetic.uniform_f32_1000(n, 40 + i)])
        vals = synthetic.index_values(len(keys)) if pairs else None
        check_multisplit(keys, vals, Case(oracle.DELTA_F32, m, delta=delta))


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("m", [257, 1000, 4097, 65535, 65536])
def test_wide_mod(m, pairs):
    edge = np.array([0, 1, m - 1, m, m + 1, 2 * m - 1, 0xFFFFFFFF, 0xFFFFFFFE, 0x80000000], np.uint32)
    for i, n in enumerate(SIZES):
        keys = np.concatenate([edge, synthetic.uniform_u32(n, 60 + i)])
        vals = synthetic.index_values(len(keys)) if pairs else None
        check_multisplit(keys, vals, Case(oracle.MOD, m))


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("shift_bits", [(0, 9), (7, 12), (16, 16), (0, 16)])
def test_wide_radix(shift_bits, pairs):
    shift, bits = shift_bits
    for i, n in enumerate(SIZES):
        keys = synthetic.uniform_u32(n, 80 + i)
        vals = synthetic.index_values(n) if pairs else None
        check_multisplit(keys, vals, Case(oracle.RADIX, 1 << bits, shift=shift, bits=bits))


def test_wide_empty_input_gives_zero_offsets():
    case = range_case(1000, 3)
    gk, gv, goff = run_gpu(np.zeros(0, np.uint32), np.zeros(0, np.uint32), case)
    assert len(gk) == 0 and len(gv) == 0
    np.testing.assert_array_equal(goff, np.zeros(1001, np.uint32))


def test_wide_full_size_65536_buckets():
    # n = 2^24 + 3 uniform keys into 65536 range buckets, pairs: every element
    n = (1 << 24) + 3
    keys = synthetic.uniform_u32(n, 90)
    check_multisplit(keys, synthetic.index_values(n), range_case(65536, 91))
