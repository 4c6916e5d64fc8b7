"""GPU parity: the CUDA multisplit (through the C ABI) against the CPU oracle,
element by element, bit exact.  Sizes span several tiles and ragged tails;
edge cases cover empty input, single elements, all keys in one bucket, sorted
and reverse-sorted keys, every m from 1 to 256 for key mod m, duplicated
splitters, float32 special values, and the full-size configurations."""
import numpy as np
import pytest

import oracle
import synthetic
from parity import Case, check_multisplit, range_case, run_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu

TILE = 4096  # tile of the default configuration (16 warps x 32 lanes x 8 keys)
SIZES = [0, 1, 31, 32, 33, 255, 1000, TILE - 1, TILE, TILE + 1, 3 * TILE + 17, 65537, 1 << 20]
MS = [1, 2, 3, 8, 31, 32, 33, 64, 255, 256]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300.build import build

    build()
    ms.lib()


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("m", MS)
def test_range_sizes(m, pairs):
    for i, n in enumerate(SIZES):
        keys = synthetic.uniform_u32(n, 1000 + i)
        vals = synthetic.index_values(n) if pairs else None
        check_multisplit(keys, vals, range_case(m, 7 + m))


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("m", [2, 8, 32, 64, 256])
def test_range_skewed(m, pairs):
    spl = synthetic.range_splitters(m, 3)
    n = 200_003
    keys = synthetic.skewed_u32(n, spl, 4)
    vals = synthetic.index_values(n) if pairs else None
    check_multisplit(keys, vals, Case(oracle.RANGE_U32, m, splitters=spl))


def test_range_duplicate_splitters_and_boundaries():
    for m in (3, 9, 40, 256):
        spl = synthetic.range_splitters(m, 5)
        spl[1:m // 2] = spl[1]  # many empty buckets
        keys = np.concatenate([spl, spl - np.uint32(1), spl + np.uint32(1), np.array([0, 0xFFFFFFFF], np.uint32),
                               synthetic.uniform_u32(10000, 6)])
        check_multisplit(keys, synthetic.index_values(len(keys)), Case(oracle.RANGE_U32, m, splitters=spl))


@pytest.mark.parametrize("m", list(range(1, 257)))
def test_mod_every_m(m):
    n = 5000 + m
    keys = np.concatenate([np.array([0, 1, m - 1, m, 0xFFFFFFFF, 0xFFFFFFFE, 0x80000000], np.uint32),
                           synthetic.uniform_u32(n, m)])
    check_multisplit(keys, synthetic.index_values(len(keys)), Case(oracle.MOD, m))


@pytest.mark.parametrize("shift,bits", [(0, 0), (0, 1), (31, 1), (0, 4), (29, 3), (24, 8), (13, 8), (0, 8),
                                        (27, 5), (26, 6)])
def test_radix_digit(shift, bits):
    for n in (TILE * 5 + 3, 100_000):
        keys = synthetic.uniform_u32(n, shift * 10 + bits)
        check_multisplit(keys, synthetic.index_values(n), Case(oracle.RADIX, 1 << bits, shift=shift, bits=bits))


@pytest.mark.parametrize("m", [1, 2, 8, 32, 64, 256, 7, 100])
def test_delta_f32(m):
    delta = np.float32(1000.0) / np.float32(m)
    grid = (np.arange(m + 1, dtype=np.float32) * delta).astype(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -5.0, 1e30, -1e30, 1e-45, 999.9999],
                       np.float32)
    near = np.concatenate([grid, np.nextafter(grid, np.float32(-np.inf)), np.nextafter(grid, np.float32(np.inf)),
                           special]).astype(np.float32)
    keys = np.concatenate([near.view(np.uint32), synthetic.uniform_f32_1000(70_000, m)])
    check_multisplit(keys, synthetic.index_values(len(keys)), Case(oracle.DELTA_F32, m, x0=0.0, delta=float(delta)))
    check_multisplit(keys, None, Case(oracle.DELTA_F32, m, x0=-3.5, delta=float(delta) * 0.75))


@pytest.mark.parametrize("m", [3, 7, 100, 256, 1000, 65536])
def test_delta_f32_every_bucket_edge(m):
    """Keys on every bucket edge k * delta and up to four ulps either side
    (the division's rounding decides their bucket), for deltas that are not
    exact in binary32 and for an offset x0; m above 256 takes the digit passes."""
    for x0, scale in ((0.0, 1.0), (-3.5, 0.75)):
        delta = np.float32(np.float32(1000.0) / np.float32(m) * np.float32(scale))
        edge = (np.float32(x0) + np.arange(m + 1, dtype=np.float32) * delta).astype(np.float32)
        near = [edge]
        lo = hi = edge
        for _ in range(4):
            lo = np.nextafter(lo, np.float32(-np.inf)).astype(np.float32)
            hi = np.nextafter(hi, np.float32(np.inf)).astype(np.float32)
            near += [lo, hi]
        keys = np.concatenate([np.concatenate(near).view(np.uint32), synthetic.uniform_f32_1000(50_000, m)])
        keys = keys[synthetic.rng(m).permutation(len(keys))]
        check_multisplit(keys, synthetic.index_values(len(keys)),
                         Case(oracle.DELTA_F32, m, x0=x0, delta=float(delta)))


@pytest.mark.parametrize("pattern", ["same", "sorted", "reversed", "one_bucket", "alternating"])
@pytest.mark.parametrize("m", [2, 32, 256])
def test_patterns(pattern, m):
    n = 3 * TILE + 5
    base = synthetic.uniform_u32(n, 99)
    if pattern == "same":
        keys = np.full(n, 0x12345678, np.uint32)
    elif pattern == "sorted":
        keys = np.sort(base)
    elif pattern == "reversed":
        keys = np.sort(base)[::-1].copy()
    elif pattern == "one_bucket":
        keys = (base % np.uint32(97)) * np.uint32(m)  # mod m == 0 for all
    else:
        keys = np.arange(n, dtype=np.uint32)
    check_multisplit(keys, synthetic.index_values(n), Case(oracle.MOD, m))
    check_multisplit(keys, None, range_case(m, 1))


def test_offsets_null_and_empty():
    import paper_1701_01189_gb300 as ms
    import torch

    keys = synthetic.uniform_u32(TILE + 3, 1)
    dk = to_dev(keys)
    out = torch.empty_like(dk)
    spec = Case(oracle.MOD, 8).gpu_spec()
    st = ms.ms_multisplit_keys(dk.data_ptr(), dk.numel(), spec.c(), out.data_ptr(), None,
                               torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK
    ok, _, _ = oracle.multisplit(keys, None, oracle.Spec(oracle.MOD, 8))
    np.testing.assert_array_equal(to_host(out), ok)
    # n = 0: offsets all zero, nothing else touched
    off = torch.full((9,), 7, dtype=torch.int32, device="cuda")
    st = ms.ms_multisplit_keys(0, 0, spec.c(), 0, off.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK
    assert to_host(off).tolist() == [0] * 9


def test_repeated_calls_and_streams():
    """Same result on a side stream, twice in a row (scratch reused from the pool)."""
    import paper_1701_01189_gb300 as ms
    import torch

    keys = synthetic.uniform_u32(300_000, 17)
    vals = synthetic.index_values(300_000)
    case = range_case(64, 2)
    ok, ov, ooff = oracle.multisplit(keys, vals, case.oracle_spec())
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dk, dv = to_dev(keys), to_dev(vals)
        for _ in range(2):
            ko, vo, off = ms.multisplit_pairs(dk, dv, case.gpu_spec(), stream=s)
            s.synchronize()
            np.testing.assert_array_equal(to_host(ko), ok)
            np.testing.assert_array_equal(to_host(vo), ov)


# ----------------------------------------------------------------- full-size configurations
def test_config_plain_2p20_key_shift29():
    """n = 2^20 uniform keys, m = 8, bucket = key >> 29, keys only, 9 offsets."""
    keys = synthetic.uniform_u32(1 << 20, 1)
    gk, _, goff = run_gpu(keys, None, Case(oracle.RADIX, 8, shift=29, bits=3))
    ok, _, ooff = oracle.multisplit(keys, None, oracle.Spec(oracle.RADIX, 8, shift=29, bits=3))
    assert len(goff) == 9
    np.testing.assert_array_equal(goff.astype(np.uint64), ooff)
    np.testing.assert_array_equal(gk, ok)


@pytest.mark.parametrize("dist", ["uniform", "skewed"])
@pytest.mark.parametrize("m", [2, 8, 32, 64, 256])
def test_config_sweep_2p26(m, dist):
    """n = 2^26 range buckets, keys only and key-value (value = index)."""
    n = 1 << 26
    spl = synthetic.range_splitters(m, 1000 + m)
    keys = synthetic.uniform_u32(n, 2000 + m) if dist == "uniform" else synthetic.skewed_u32(n, spl, 3000 + m)
    case = Case(oracle.RANGE_U32, m, splitters=spl)
    check_multisplit(keys, None, case)
    check_multisplit(keys, synthetic.index_values(n), case)


@pytest.mark.parametrize("m", [2, 8, 32, 64, 256])
def test_config_sweep_2p26_f32(m):
    n = 1 << 26
    keys = synthetic.uniform_f32_1000(n, 4000 + m)
    case = Case(oracle.DELTA_F32, m, x0=0.0, delta=float(np.float32(1000.0) / np.float32(m)))
    check_multisplit(keys, None, case)
    check_multisplit(keys, synthetic.index_values(n), case)


@pytest.mark.parametrize("dist", ["binomial", "alpha0.25"])
@pytest.mark.parametrize("m", [32, 256])
def test_section64_distributions(m, dist):
    """Section 6.4's non-uniform inputs (binomial B(m-1, 0.5), 0.25-uniform) with
    delta buckets, keys and key-value, bit exact."""
    n = (1 << 22) + 3
    delta = float(np.float32(1000.0) / np.float32(m))
    keys = (synthetic.binomial_f32(n, m, delta, 21) if dist == "binomial"
            else synthetic.alpha_uniform_f32(n, m, delta, 0.25, 22))
    case = Case(oracle.DELTA_F32, m, x0=0.0, delta=delta)
    check_multisplit(keys, None, case)
    check_multisplit(keys, synthetic.index_values(n), case)


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("m", [2, 8, 32, 64, 256, 1000])
def test_unaligned_buffers(m, pairs):
    """Inputs and outputs 4 bytes past a 16-byte boundary: the kernels fall
    back from bulk and tensor copies to plain loads; the result is the same."""
    import torch

    import paper_1701_01189_gb300 as ms

    n = 7 * 4096 + 123
    keys = synthetic.uniform_u32(n, 300 + m)
    vals = synthetic.index_values(n)
    case = range_case(m, 301 + m)
    dk = to_dev(np.concatenate([np.zeros(1, np.uint32), keys]))[1:]
    dv = to_dev(np.concatenate([np.zeros(1, np.uint32), vals]))[1:]
    ko = torch.empty(n + 1, dtype=torch.int32, device="cuda")[1:]
    vo = torch.empty(n + 1, dtype=torch.int32, device="cuda")[1:]
    assert dk.data_ptr() % 16 == 4 and ko.data_ptr() % 16 == 4
    spec = case.gpu_spec()
    if pairs:
        _, _, off = ms.multisplit_pairs(dk, dv, spec, keys_out=ko, vals_out=vo)
    else:
        _, off = ms.multisplit_keys(dk, spec, keys_out=ko)
    torch.cuda.synchronize()
    assert ms.device_status() == ms.MS_OK
    ok, ov, ooff = oracle.multisplit(keys, vals if pairs else None, case.oracle_spec())
    np.testing.assert_array_equal(to_host(ko), ok)
    if pairs:
        np.testing.assert_array_equal(to_host(vo), ov)
    np.testing.assert_array_equal(to_host(off).astype(np.uint64), ooff)
    if m <= ms.MAX_M:
        counts = ms.histogram(dk, spec)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_host(counts).astype(np.uint64), np.diff(ooff))
    sk, sv = ms.radix_sort(dk, dv if pairs else None, 0, 32, keys_out=ko, vals_out=vo if pairs else None)
    torch.cuda.synchronize()
    ek, ev = oracle.radix_sort(keys, vals if pairs else None, 0, 32)
    np.testing.assert_array_equal(to_host(sk), ek)
    if pairs:
        np.testing.assert_array_equal(to_host(sv), ev)
