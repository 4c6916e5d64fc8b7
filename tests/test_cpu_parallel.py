"""The all-core CPU baseline (oracle/ms_cpu_parallel.c) against the oracle:
bit-exact for every bucket kind, several thread counts (one chunk per thread,
so chunk boundaries fall inside bucket runs), ragged sizes and the empty
input."""
import numpy as np
import pytest

import oracle
import synthetic


def specs():
    return [oracle.Spec(oracle.RANGE_U32, 32, splitters=synthetic.range_splitters(32, 1)),
            oracle.Spec(oracle.RANGE_U32, 256, splitters=synthetic.range_splitters(256, 2)),
            oracle.Spec(oracle.DELTA_F32, 64, x0=0.0, delta=float(np.float32(1000.0) / np.float32(64))),
            oracle.Spec(oracle.RADIX, 256, shift=8, bits=8), oracle.Spec(oracle.MOD, 7), oracle.Spec(oracle.MOD, 1)]


@pytest.mark.parametrize("si", range(6))
@pytest.mark.parametrize("threads", [1, 3, 16])
@pytest.mark.parametrize("n", [0, 1, 4095, 100_003])
def test_parallel_baseline_equals_oracle(si, threads, n):
    spec = specs()[si]
    keys = synthetic.uniform_f32_1000(n, 5) if spec.kind == oracle.DELTA_F32 else synthetic.uniform_u32(n, 5)
    vals = synthetic.index_values(n)
    ek, ev, eoff = oracle.multisplit(keys, vals, spec)
    gk, gv, goff = oracle.multisplit_parallel(keys, vals, spec, threads=threads)
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(gv, ev)
    np.testing.assert_array_equal(goff, eoff)
    kk, kv, koff = oracle.multisplit_parallel(keys, None, spec, threads=threads)
    assert kv is None
    np.testing.assert_array_equal(kk, ek)
    np.testing.assert_array_equal(koff, eoff)


def test_parallel_baseline_skewed_keys():
    spec = oracle.Spec(oracle.RANGE_U32, 32, splitters=synthetic.range_splitters(32, 3))
    keys = synthetic.skewed_u32(1 << 18, spec.splitters, 4)
    ek, _, eoff = oracle.multisplit(keys, None, spec)
    gk, _, goff = oracle.multisplit_parallel(keys, None, spec, threads=8)
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(goff, eoff)
