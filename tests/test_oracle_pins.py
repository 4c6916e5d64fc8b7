"""Pins for the CPU oracle: checks against what the paper and plain mathematics fix.

None of these re-types the oracle's own arithmetic.  They use a different
algorithm (a stable sort by (bucket, index) instead of counting; numpy
broadcasting instead of bisection; numpy float32 division instead of C), the
paper's worked examples (tests/golden/), the two- and three-level forms of the
permutation (Eq. 2, Eq. 3) and the output invariants of Section 3.1.  The last
test plants each of the oracle's test mutants and checks that some pin fails.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- independent bucket ids
def np_bucket_ids(keys, spec):
    """Bucket ids by numpy, each from its definition, not from the oracle's code path."""
    keys = np.asarray(keys, np.uint32)
    if spec.kind == oracle.RANGE_U32:
        s = np.asarray(spec.splitters, np.uint64)
        return (s[None, :] <= keys.astype(np.uint64)[:, None]).sum(axis=1).astype(np.int64)
    if spec.kind == oracle.MOD:
        return (keys.astype(np.int64) % spec.m)
    if spec.kind == oracle.RADIX:
        return ((keys.astype(np.int64) >> spec.shift) & ((1 << spec.bits) - 1))
    if spec.kind == oracle.DELTA_F32:
        x = keys.view(np.float32)
        with np.errstate(all="ignore"):
            q = (x - np.float32(spec.x0)) / np.float32(spec.delta)
            f = np.floor(q)
        out = np.zeros(len(keys), np.int64)
        ok = (f > 0) & ~np.isnan(f)
        out[ok] = np.minimum(f[ok], spec.m - 1).astype(np.int64)
        out[np.isnan(q)] = spec.m - 1
        return out
    raise ValueError(spec.kind)


def brute_force(keys, vals, ids):
    """Stable multisplit by a stable sort on (bucket id, input index)."""
    order = sorted(range(len(keys)), key=lambda i: (int(ids[i]), i))
    ko = np.asarray([keys[i] for i in order], np.uint32)
    vo = None if vals is None else np.asarray([vals[i] for i in order], np.uint32)
    m = int(max(ids) + 1) if len(ids) else 0
    return ko, vo, order


def check_invariants(keys, vals_index, spec, ko, vo, off):
    """Section 3.1: a permutation; buckets contiguous, ascending; order kept inside each."""
    n = len(keys)
    assert off[0] == 0 and int(off[-1]) == n
    assert np.all(np.diff(off.astype(np.int64)) >= 0)
    ids_in = np_bucket_ids(keys, spec)
    np.testing.assert_array_equal(np.diff(off.astype(np.int64)), np.bincount(ids_in, minlength=spec.m))
    # vo is the original index: the output is the input permuted
    assert sorted(vo.tolist()) == list(range(n))
    np.testing.assert_array_equal(ko, np.asarray(keys)[vo])
    ids_out = np_bucket_ids(ko, spec)
    for j in range(spec.m):
        seg = slice(int(off[j]), int(off[j + 1]))
        assert np.all(ids_out[seg] == j)
        assert np.all(np.diff(vo[seg].astype(np.int64)) > 0)


# ---------------------------------------------------------------- pins (mutant-parameterised)
def pin_range_ids(mutant=0):
    g = synthetic.rng(11)
    for m in (2, 3, 8, 33, 256):
        spl = np.sort(g.integers(0, 1 << 32, size=m - 1, dtype=np.uint64)).astype(np.uint32)
        if m > 3:
            spl[m // 3] = spl[m // 3 - 1]  # a duplicated splitter: an empty bucket
        keys = np.concatenate([g.integers(0, 1 << 32, 3000, dtype=np.uint64).astype(np.uint32),
                               spl, spl - np.uint32(1), spl + np.uint32(1),
                               np.array([0, 0xFFFFFFFF], np.uint32)])
        spec = oracle.Spec(oracle.RANGE_U32, m, splitters=spl)
        np.testing.assert_array_equal(oracle.bucket_ids(keys, spec, mutant), np_bucket_ids(keys, spec))


def pin_mod_radix_ids(mutant=0):
    keys = np.concatenate([synthetic.uniform_u32(5000, 3), np.array([0, 1, 0xFFFFFFFF], np.uint32)])
    for m in (1, 2, 3, 7, 31, 32, 33, 255, 256):
        spec = oracle.Spec(oracle.MOD, m)
        np.testing.assert_array_equal(oracle.bucket_ids(keys, spec, mutant), np_bucket_ids(keys, spec))
    for shift, bits in ((0, 8), (8, 8), (24, 8), (29, 3), (28, 4), (0, 1), (31, 1)):
        spec = oracle.Spec(oracle.RADIX, 1 << bits, shift=shift, bits=bits)
        np.testing.assert_array_equal(oracle.bucket_ids(keys, spec, mutant), np_bucket_ids(keys, spec))


def pin_delta_golden(mutant=0):
    for c in _golden("delta_f32_spot.json")["cases"]:
        spec = oracle.Spec(oracle.DELTA_F32, c["m"], x0=c["x0"], delta=c["delta"])
        key = np.array([int(c["x_bits"], 16)], np.uint32)
        got = int(oracle.bucket_ids(key, spec, mutant)[0])
        assert got == c["bucket"], (c, got)


def pin_delta_numpy(mutant=0):
    for m in (2, 8, 32, 64, 256):
        delta = np.float32(1000.0) / np.float32(m)
        grid = (np.arange(m + 1, dtype=np.float32) * delta).astype(np.float32)
        near = np.concatenate([grid, np.nextafter(grid, np.float32(-np.inf)),
                               np.nextafter(grid, np.float32(np.inf))]).astype(np.float32)
        keys = np.concatenate([synthetic.uniform_f32_1000(4000, m), near.view(np.uint32)])
        spec = oracle.Spec(oracle.DELTA_F32, m, x0=0.0, delta=float(delta))
        np.testing.assert_array_equal(oracle.bucket_ids(keys, spec, mutant), np_bucket_ids(keys, spec))


def _small_specs(m):
    specs = [oracle.Spec(oracle.MOD, m)]
    if m > 1:
        specs.append(oracle.Spec(oracle.RANGE_U32, m,
                                 splitters=np.arange(1, m, dtype=np.uint32)))
    return specs


def pin_bruteforce_exhaustive(mutant=0):
    """Every key sequence over a small alphabet, n <= 6, m in {1, 2, 3, 8}."""
    for m in (1, 2, 3, 8):
        alphabet = list(range(min(m + 1, 4))) if m < 8 else [0, 3, 5, 7]
        for spec in _small_specs(m):
            for n in range(0, 7 if m < 8 else 5):
                for seq in itertools.product(alphabet, repeat=n):
                    keys = np.asarray(seq, np.uint32)
                    vals = np.arange(n, dtype=np.uint32) + np.uint32(100)
                    ko, vo, off = oracle.multisplit(keys, vals, spec, mutant)
                    ids = np_bucket_ids(keys, spec)
                    bk, bv, _ = brute_force(keys, vals, ids)
                    np.testing.assert_array_equal(ko, bk)
                    np.testing.assert_array_equal(vo, bv)
                    np.testing.assert_array_equal(
                        off, np.concatenate([[0], np.cumsum(np.bincount(ids, minlength=m))]))


def pin_random_vs_argsort(mutant=0):
    g = synthetic.rng(5)
    for trial in range(36):
        n = int(g.integers(0, 4097))
        # m beyond 256 too: Eq. 1 defines the result for any bucket count (Section 6.3)
        m = int(g.choice([1, 2, 3, 8, 31, 32, 33, 64, 255, 256, 257, 1000, 65536]))
        keys = synthetic.uniform_u32(n, 100 + trial)
        kind = trial % 3
        if kind == 0:
            spec = oracle.Spec(oracle.RANGE_U32, m, splitters=synthetic.range_splitters(m, trial))
        elif kind == 1:
            spec = oracle.Spec(oracle.MOD, m)
        else:
            bits = max(0, int(np.log2(m)))
            spec = oracle.Spec(oracle.RADIX, 1 << bits, shift=int(g.integers(0, 33 - max(bits, 1))),
                               bits=bits)
        vals = synthetic.index_values(n)
        ko, vo, off = oracle.multisplit(keys, vals, spec, mutant)
        ids = np_bucket_ids(keys, spec)
        order = np.argsort(ids, kind="stable")
        np.testing.assert_array_equal(ko, keys[order])
        np.testing.assert_array_equal(vo, vals[order])
        check_invariants(keys, vals, spec, ko, vo, off)


def pin_fig3(mutant=0):
    """Fig. 3: local offsets 0..5 and count 6 for B_j at positions 1, 4, 5, 8, 11, 14."""
    gd = _golden("fig3_local_offsets.json")
    w = gd["window"]
    in_j = set(gd["positions_in_bucket"])
    # bucket 1 is B_j; other positions alternate between buckets 0 and 2
    keys = np.array([1 if i in in_j else (0 if i % 2 else 2) for i in range(w)], np.uint32)
    spec = oracle.Spec(oracle.MOD, 3)
    ko, vo, off = oracle.multisplit(keys, np.arange(w, dtype=np.uint32), spec, mutant)
    assert int(off[2]) - int(off[1]) == gd["bucket_count"]
    pos = np.empty(w, np.int64)
    pos[vo] = np.arange(w)  # p(i) for every input element
    local = [int(pos[i]) - int(off[1]) for i in gd["positions_in_bucket"]]
    assert local == gd["local_offsets"]


def pin_eq2_two_level(mutant=0):
    """Eq. 2: p(i) from L per-subproblem histograms (global + per-subproblem + local terms)."""
    g = synthetic.rng(21)
    for trial in range(8):
        n = int(g.integers(1, 3000))
        m = int(g.choice([2, 5, 32, 64]))
        spec = oracle.Spec(oracle.RANGE_U32, m, splitters=synthetic.range_splitters(m, 50 + trial))
        keys = synthetic.uniform_u32(n, 60 + trial)
        ids = np_bucket_ids(keys, spec)
        L = int(g.integers(1, 9))
        cuts = np.sort(g.integers(0, n + 1, size=L - 1))
        bounds = np.concatenate([[0], cuts, [n]])
        H = np.zeros((m, L), np.int64)
        for l in range(L):
            H[:, l] = np.bincount(ids[bounds[l]:bounds[l + 1]], minlength=m)
        p = np.empty(n, np.int64)
        for l in range(L):
            for i in range(bounds[l], bounds[l + 1]):
                j = ids[i]
                term1 = H[:j, :].sum()
                term2 = H[j, :l].sum()
                term3 = int(np.sum(ids[bounds[l]:i] == j))
                p[i] = term1 + term2 + term3
        ko, vo, off = oracle.multisplit(keys, np.arange(n, dtype=np.uint32), spec, mutant)
        got = np.empty(n, np.int64)
        got[vo] = np.arange(n)
        np.testing.assert_array_equal(got, p)


def pin_eq3_three_level(mutant=0):
    """Eq. 3 with the Fig. 2 hierarchy (L0, L1, L2) = (2, 3, 5) of equal-size subproblems."""
    gd = _golden("fig2_localization.json")
    L0, L1, L2 = gd["levels"]
    t0, t1, t2 = gd["tuple"]
    assert (t0 * L1 + t1) * L2 + t2 == gd["flat_index"] and L0 * L1 * L2 == gd["total"]
    sub = 7  # elements per last-level subproblem
    n = L0 * L1 * L2 * sub
    m = 6
    keys = synthetic.uniform_u32(n, 77)
    spec = oracle.Spec(oracle.MOD, m)
    ids = np_bucket_ids(keys, spec)
    h = np.zeros((m, L0, L1, L2), np.int64)
    for a, b, c in itertools.product(range(L0), range(L1), range(L2)):
        s = ((a * L1 + b) * L2 + c) * sub
        h[:, a, b, c] = np.bincount(ids[s:s + sub], minlength=m)
    p = np.empty(n, np.int64)
    for i in range(n):
        leaf, r = divmod(i, sub)
        a, rest = divmod(leaf, L1 * L2)
        b, c = divmod(rest, L2)
        j = ids[i]
        p[i] = (h[:j].sum() + h[j, :a].sum() + h[j, a, :b].sum() + h[j, a, b, :c].sum()
                + int(np.sum(ids[leaf * sub:i] == j)))
    ko, vo, off = oracle.multisplit(keys, np.arange(n, dtype=np.uint32), spec, mutant)
    got = np.empty(n, np.int64)
    got[vo] = np.arange(n)
    np.testing.assert_array_equal(got, p)


def pin_histogram_bincount(mutant=0):
    keys = synthetic.uniform_u32(20000, 9)
    for spec in (oracle.Spec(oracle.MOD, 37), oracle.Spec(oracle.RADIX, 256, shift=8, bits=8),
                 oracle.Spec(oracle.RANGE_U32, 64, splitters=synthetic.range_splitters(64, 3))):
        np.testing.assert_array_equal(oracle.histogram(keys, spec, mutant),
                                      np.bincount(np_bucket_ids(keys, spec), minlength=spec.m))


def pin_identity_bucket_sort(mutant=0):
    """Section 7.1: identity buckets == a sort on the low ceil(log m) bits; radix-digit
    buckets f(u) = (u >> s) & (2^r - 1) give a stable sort on bits [s, s + r)."""
    keys = synthetic.uniform_u32_bits(5000, 8, 4)
    ko, _, _ = oracle.multisplit(keys, None, oracle.Spec(oracle.RADIX, 256, shift=0, bits=8), mutant)
    np.testing.assert_array_equal(ko, np.sort(keys))
    keys = synthetic.uniform_u32(5000, 5)
    vals = synthetic.index_values(5000)
    for s, r in ((0, 8), (8, 8), (13, 5), (24, 8)):
        ko, vo, _ = oracle.multisplit(keys, vals, oracle.Spec(oracle.RADIX, 1 << r, shift=s, bits=r),
                                      mutant)
        digit = (keys.astype(np.int64) >> s) & ((1 << r) - 1)
        order = sorted(range(len(keys)), key=lambda i: (digit[i], i))
        np.testing.assert_array_equal(vo, np.asarray(order, np.uint32))


def pin_lsd_composition(mutant=0):
    """Section 7.1: ceil(32 / r) multisplit passes with f_k = (u >> kr) & (2^r - 1)
    sort the keys; with values = index, the result is the stable sort."""
    keys = synthetic.uniform_u32(3000, 6) & np.uint32(0xFFFF00FF)  # ties in the middle digits
    vals = synthetic.index_values(3000)
    k, v = keys, vals
    for p in range(4):
        k, v, _ = oracle.multisplit(k, v, oracle.Spec(oracle.RADIX, 256, shift=8 * p, bits=8), mutant)
    order = sorted(range(len(keys)), key=lambda i: (int(keys[i]), i))
    np.testing.assert_array_equal(v, np.asarray(order, np.uint32))
    np.testing.assert_array_equal(k, keys[order])


PINS = [pin_range_ids, pin_mod_radix_ids, pin_delta_golden, pin_delta_numpy,
        pin_bruteforce_exhaustive, pin_random_vs_argsort, pin_fig3, pin_eq2_two_level,
        pin_eq3_three_level, pin_histogram_bincount, pin_identity_bucket_sort, pin_lsd_composition]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin(0)


# ---------------------------------------------------------------- radix-sort oracle pins
def test_radix_sort_oracle_small_bruteforce():
    g = synthetic.rng(8)
    for trial in range(40):
        n = int(g.integers(0, 60))
        keys = g.integers(0, 16, size=n, dtype=np.uint64).astype(np.uint32) * np.uint32(0x01010101)
        vals = np.arange(n, dtype=np.uint32)
        b, e = sorted(g.integers(0, 33, size=2).tolist())
        ko, vo = oracle.radix_sort(keys, vals, b, e)
        width = e - b
        dig = [((int(k) >> b) & ((1 << width) - 1)) if width > 0 else 0 for k in keys]
        order = sorted(range(n), key=lambda i: (dig[i], i))
        assert vo.tolist() == order
        assert ko.tolist() == [int(keys[i]) for i in order]


def test_radix_sort_oracle_full_key_unique():
    keys = synthetic.uniform_u32(100000, 12)
    ko, _ = oracle.radix_sort(keys, None, 0, 32)
    np.testing.assert_array_equal(ko, np.sort(keys))


def test_radix_sort_16bit():
    keys = synthetic.uniform_u32_bits(50000, 16, 13)
    vals = synthetic.index_values(50000)
    ko, vo = oracle.radix_sort(keys, vals, 0, 16)
    np.testing.assert_array_equal(ko, np.sort(keys))
    assert np.all(np.diff(vo[np.concatenate([[False], np.diff(ko) == 0])].astype(np.int64)) != 0)


def test_position_single_element():
    keys = synthetic.uniform_u32(500, 14)
    spec = oracle.Spec(oracle.MOD, 7)
    ko, vo, off = oracle.multisplit(keys, np.arange(500, dtype=np.uint32), spec)
    pos = np.empty(500, np.int64)
    pos[vo] = np.arange(500)
    h = oracle.histogram(keys, spec)
    for i in (0, 1, 17, 250, 499):
        assert oracle.position(keys, spec, i, h) == pos[i]


def test_multisplit_empty_and_m1():
    ko, vo, off = oracle.multisplit(np.zeros(0, np.uint32), np.zeros(0, np.uint32), oracle.Spec(oracle.MOD, 5))
    assert len(ko) == 0 and off.tolist() == [0] * 6
    keys = synthetic.uniform_u32(100, 1)
    ko, vo, off = oracle.multisplit(keys, None, oracle.Spec(oracle.MOD, 1))
    np.testing.assert_array_equal(ko, keys)
    assert off.tolist() == [0, 100]


# ---------------------------------------------------------------- the pins catch planted mistakes
MUTANTS = {
    1: "global offset drops h_0",
    2: "local offset counts r <= i",
    3: "unstable: reversed inside a bucket",
    4: "values not carried",
    5: "buckets in descending order",
    6: "range bucket is a lower bound",
    7: "delta uses round instead of floor",
    8: "radix shift off by one",
    9: "mod uses a power-of-two mask",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=[MUTANTS[k] for k in sorted(MUTANTS)])
def test_pins_catch_mutant(mutant):
    caught = []
    for pin in PINS:
        try:
            pin(mutant)
        except (AssertionError, IndexError, ValueError):
            caught.append(pin.__name__)
    assert caught, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"
