"""Parameter invariance: every kernel variant the tuner can choose (tile shape,
rank mode, reordering) gives the oracle's result bit for bit."""
import itertools

import numpy as np
import pytest

import oracle
import synthetic
from parity import Case, check_multisplit, clustered_splitters

pytestmark = pytest.mark.gpu


def variants(log2m):
    from paper_1701_01189_gb300.autotune import variants as tuner_variants

    return tuner_variants(log2m)


CASES = []
for m, kind in itertools.product([1, 2, 3, 8, 17, 32, 33, 256], ["range", "mod", "radix", "delta"]):
    if kind == "radix" and m & (m - 1):
        continue
    CASES.append((kind, m))


def make_case(kind, m):
    if kind == "range":
        return Case(oracle.RANGE_U32, m, splitters=synthetic.range_splitters(m, m))
    if kind == "mod":
        return Case(oracle.MOD, m)
    if kind == "radix":
        bits = m.bit_length() - 1
        return Case(oracle.RADIX, m, shift=32 - max(bits, 1) if bits else 0, bits=bits)
    return Case(oracle.DELTA_F32, m, x0=0.0, delta=float(np.float32(1000.0) / np.float32(m)))


@pytest.mark.parametrize("kind,m", CASES, ids=[f"{k}-m{m}" for k, m in CASES])
def test_every_variant_matches_oracle(kind, m):
    import paper_1701_01189_gb300 as ms

    case = make_case(kind, m)
    log2m = (m - 1).bit_length()
    n = 3 * 4096 + 129
    keys = synthetic.uniform_f32_1000(n, 3) if kind == "delta" else synthetic.uniform_u32(n, 3)
    try:
        for shape, rank, reorder in variants(log2m):
            for pairs in (0, 1):
                assert ms.ms_tune_set(case.kind, pairs, log2m, ms.ms_tune_size_class(n), shape, rank,
                                      reorder) == ms.MS_OK
            check_multisplit(keys, None, case)
            check_multisplit(keys, synthetic.index_values(n), case)
    finally:
        ms.ms_tune_reset()


@pytest.mark.parametrize("m", [3, 8, 17, 32, 33, 64, 200, 256])
def test_every_variant_clustered_splitters(m):
    """Range buckets whose splitters come in tight clusters: every kernel
    variant, keys on, just below and just above each splitter, near the
    clusters and uniform."""
    import paper_1701_01189_gb300 as ms

    spl = clustered_splitters(m, 70 + m)
    g = synthetic.rng(71 + m)
    near = (spl.astype(np.int64)[g.integers(0, m - 1, size=6000)] + g.integers(-4096, 4096, size=6000))
    keys = np.concatenate([spl, spl - np.uint32(1), spl + np.uint32(1),
                           np.clip(near, 0, 0xFFFFFFFF).astype(np.uint32), synthetic.uniform_u32(6000, 72)])
    keys = keys[g.permutation(len(keys))]
    n = len(keys)
    case = Case(oracle.RANGE_U32, m, splitters=spl)
    log2m = (m - 1).bit_length()
    try:
        for shape, rank, reorder in variants(log2m):
            for pairs in (0, 1):
                assert ms.ms_tune_set(case.kind, pairs, log2m, ms.ms_tune_size_class(n), shape, rank,
                                      reorder) == ms.MS_OK
            check_multisplit(keys, None, case)
            check_multisplit(keys, synthetic.index_values(n), case)
    finally:
        ms.ms_tune_reset()


@pytest.mark.parametrize("shape", [0, 1, 2], ids=["16-per-thread", "16-per-thread-3-slots", "8-per-thread"])
@pytest.mark.parametrize("m", [2, 8, 32])
def test_counter_variants_many_tiles_per_chunk(m, shape):
    """Per-thread-counter kernels at a size where every CTA walks many tiles
    (and the last one is ragged), for both tile shapes."""
    import paper_1701_01189_gb300 as ms

    n = (1 << 22) + 77
    case = make_case("range", m)
    log2m = (m - 1).bit_length()
    keys = synthetic.uniform_u32(n, 11)
    try:
        for pairs in (0, 1):
            assert ms.ms_tune_set(case.kind, pairs, log2m, ms.ms_tune_size_class(n), shape, 2, 1) == ms.MS_OK
        check_multisplit(keys, None, case)
        check_multisplit(keys, synthetic.index_values(n), case)
    finally:
        ms.ms_tune_reset()


def shipped_variants():
    """(kind, log2m, shape, rank, reorder) of every entry of the shipped tuning table."""
    import json
    import os

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1701_01189_gb300",
                        "tuning.json")
    if not os.path.exists(path):
        return []
    out = set()
    for e in json.load(open(path))["entries"]:
        out.add((e["kind"], e["log2m"], e["shape"], e["rank"], e["reorder"]))
    return sorted(out)


@pytest.mark.parametrize("entry", shipped_variants(), ids=lambda e: "k{}-lg{}-v{}{}{}".format(*e))
def test_shipped_tuning_variants_many_tiles(entry):
    """Every variant the shipped tuning table selects, at a size where every CTA
    walks many tiles, bit exact against the oracle (keys and key-value)."""
    import paper_1701_01189_gb300 as ms

    kind, log2m, shape, rank, reorder = entry
    m = 1 << log2m
    name = {oracle.RANGE_U32: "range", oracle.MOD: "mod", oracle.RADIX: "radix", oracle.DELTA_F32: "delta"}[kind]
    case = make_case(name, m)
    n = (1 << 22) + 77
    keys = synthetic.uniform_f32_1000(n, 13) if name == "delta" else synthetic.uniform_u32(n, 13)
    try:
        for pairs in (0, 1):
            assert ms.ms_tune_set(case.kind, pairs, log2m, ms.ms_tune_size_class(n), shape, rank, reorder) == ms.MS_OK
        check_multisplit(keys, None, case)
        check_multisplit(keys, synthetic.index_values(n), case)
    finally:
        ms.ms_tune_reset()
