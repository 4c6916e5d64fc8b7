"""Host-side checks that need no GPU: the C ABI loads and exports what
include/ms.h declares, argument validation returns MS_ERR_INVALID_ARG before
touching the device, and the rate / byte models match the paper's figures."""
import ctypes
import json
import os
import re

import pytest

import paper_1701_01189_gb300 as ms
from paper_1701_01189_gb300 import metrics
from paper_1701_01189_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def lib():
    build()
    return ms.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ms_[a-z0-9_]+)\s*\(", text,
                                flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for f in ("ms_multisplit_keys", "ms_multisplit_pairs", "ms_radix_sort", "ms_device_status",
              "ms_status_string", "ms_version"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    assert "sm_103a" in ms.ms_version()
    assert ms.ms_status_string(ms.MS_ERR_TIMEOUT) == "MS_ERR_TIMEOUT"
    assert ms.ms_status_string(99) == "MS_ERR_UNKNOWN"


def _spec(kind, m, **kw):
    return ms._binding._Spec(kind, m, kw.get("splitters"), kw.get("x0", 0.0), kw.get("delta", 1.0),
                             kw.get("shift", 0), kw.get("bits", 0))


BAD_SPECS = [
    _spec(ms.MOD, 0),
    _spec(ms.MOD, 65537),
    _spec(ms.RANGE_U32, 70000, splitters=0x5000),
    _spec(ms.RANGE_U32, 300, splitters=None),
    _spec(ms.DELTA_F32, 1000, delta=0.0),
    _spec(ms.RADIX, 1 << 17, shift=0, bits=17),
    _spec(ms.RADIX, 1 << 16, shift=20, bits=16),
    _spec(ms.RADIX, 1000, shift=0, bits=10),
    _spec(9, 1000),
    _spec(ms.RANGE_U32, 4, splitters=None),
    _spec(ms.DELTA_F32, 8, delta=0.0),
    _spec(ms.DELTA_F32, 8, delta=-1.0),
    _spec(ms.DELTA_F32, 8, delta=float("inf")),
    _spec(ms.DELTA_F32, 8, delta=1.0, x0=float("nan")),
    _spec(ms.RADIX, 256, shift=28, bits=8),
    _spec(ms.RADIX, 128, shift=0, bits=8),
    _spec(ms.RADIX, 512, shift=0, bits=8),
    _spec(7, 8),
]

# valid for ms_multisplit_keys / _pairs (two digit passes) but not for the
# histogram, batched plans and the no-allocation entry point (m <= 256)
WIDE_SPECS = [
    _spec(ms.MOD, 257),
    _spec(ms.DELTA_F32, 65536, delta=1.0),
    _spec(ms.RANGE_U32, 1000, splitters=0x5000),
    _spec(ms.RADIX, 512, shift=0, bits=9),
]


@pytest.mark.parametrize("i", range(len(BAD_SPECS)))
def test_bad_spec_rejected_before_device(lib, i):
    assert ms.ms_multisplit_keys(0x1000, 16, BAD_SPECS[i], 0x2000, 0, None) == ms.MS_ERR_INVALID_ARG


@pytest.mark.parametrize("i", range(len(WIDE_SPECS)))
def test_wide_specs_only_for_the_plain_calls(lib, i):
    spec = WIDE_SPECS[i]
    assert ms.ms_histogram(0x1000, 16, spec, 0x2000, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_multisplit_keys_noalloc(0x1000, 16, spec, 0x2000, 0, None) == ms.MS_ERR_INVALID_ARG
    st, _h = ms.ms_batch_plan_create([(0x1000, None, 0x2000, None, 0x3000, 16)], spec)
    assert st == ms.MS_ERR_INVALID_ARG
    # the plain call checks the pointers first (no device work here)
    assert ms.ms_multisplit_keys(None, 16, spec, 0x2000, 0, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_multisplit_keys(0x1000, 16, spec, 0x1020, 0, None) == ms.MS_ERR_INVALID_ARG


def test_bad_radix_width_rejected(lib):
    for r in (0, 9, -1):
        assert ms.ms_radix_sort_r(0x1000, None, 16, 0, 32, r, 0x2000, None, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_radix_sort_r(0x1000, None, 16, 8, 4, 4, 0x2000, None, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_radix_sort_r(0x1000, None, 16, 0, 32, 4, 0x1000, None, None) == ms.MS_ERR_INVALID_ARG


def test_bad_pointers_rejected(lib):
    good = _spec(ms.MOD, 8)
    assert ms.ms_multisplit_keys(None, 16, good, 0x2000, 0, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_multisplit_keys(0x1000, 16, good, 0x1000, 0, None) == ms.MS_ERR_INVALID_ARG  # aliasing
    assert ms.ms_multisplit_keys(0x1000, 16, good, 0x1020, 0, None) == ms.MS_ERR_INVALID_ARG  # overlap
    assert ms.ms_multisplit_keys(0x1000, 1 << 32, good, 0x80001000, 0, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_multisplit_pairs(0x1000, None, 16, good, 0x2000, 0x3000, 0, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_multisplit_pairs(0x1000, 0x4000, 16, good, 0x2000, 0x4000, 0, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_radix_sort(0x1000, None, 16, 8, 4, 0x2000, None, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_radix_sort(0x1000, None, 16, 0, 33, 0x2000, None, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_radix_sort(0x1000, 0x3000, 16, 0, 32, 0x2000, None, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_histogram(0x1000, 16, good, None, None) == ms.MS_ERR_INVALID_ARG  # no counts
    assert ms.ms_histogram(None, 16, good, 0x2000, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_histogram(0x1000, 1 << 32, good, 0x2000, None) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_histogram(0x1000, 16, BAD_SPECS[0], 0x2000, None) == ms.MS_ERR_INVALID_ARG


def test_speed_of_light_model_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_rates.json")))
    for row in g["sol"]:
        k = metrics.sol_rate_g(row["gbs"], metrics.method_bytes_per_element(False))
        p = metrics.sol_rate_g(row["gbs"], metrics.method_bytes_per_element(True))
        assert abs(k - row["keys_gkeys"]) < 0.1 and abs(p - row["pairs_gpairs"]) < 0.1


def test_rate_definition_matches_tables_4_and_5():
    r = json.load(open(os.path.join(GOLDEN, "paper_rates.json")))["rate"]
    got = metrics.rate_g(r["n"], r["ms"] * 1e-3)
    assert abs(got - r["gkeys"]) / r["gkeys"] < r["rel_tol"]


def test_compulsory_bytes():
    assert metrics.compulsory_bytes_per_element(False) == 8
    assert metrics.compulsory_bytes_per_element(True) == 16
    assert metrics.sort_compulsory_bytes_per_element(True, 4) == 64


def test_tuning_table_validation_and_defaults(lib):
    ms.ms_tune_reset()
    assert ms.ms_tune_size_class(0) == 0 and ms.ms_tune_size_class(1 << 16) == 1
    assert ms.ms_tune_size_class((1 << 24) - 1) == 2 and ms.ms_tune_size_class(1 << 28) == 3
    assert ms.ms_tune_get(ms.RANGE_U32, 0, 1, 3) == (0, 2, 1)  # m = 2: per-thread counters
    assert ms.ms_tune_get(ms.RANGE_U32, 1, 8, 3) == (1, 1, 1)  # m = 256 pairs: peer tables, 16 x 8
    assert ms.ms_tune_get(ms.MOD, 0, 5, 3) == (0, 2, 1)  # m = 32: per-thread counters
    assert ms.ms_tune_get(ms.MOD, 1, 6, 3) == (2, 1, 1)  # m = 64 pairs: peer tables, 8 x 8
    assert ms.ms_tune_set(ms.MOD, 0, 6, 3, 1, 0, 1) == ms.MS_ERR_INVALID_ARG  # ballots need log2 m <= 5
    assert ms.ms_tune_set(ms.MOD, 0, 4, 3, 1, 0, 0) == ms.MS_ERR_INVALID_ARG  # direct writes need log2 m <= 3
    assert ms.ms_tune_set(ms.MOD, 0, 5, 3, 1, 1, 0) == ms.MS_ERR_INVALID_ARG  # tables always reorder
    assert ms.ms_tune_set(ms.MOD, 0, 5, 3, 3, 1, 1) == ms.MS_ERR_INVALID_ARG  # no shape 3
    assert ms.ms_tune_set(4, 0, 5, 3, 0, 1, 1) == ms.MS_ERR_INVALID_ARG
    assert ms.ms_tune_set(ms.MOD, 0, 6, 3, 0, 2, 1) == ms.MS_ERR_INVALID_ARG  # counters need log2 m <= 5
    assert ms.ms_tune_set(ms.MOD, 0, 5, 3, 0, 2, 0) == ms.MS_ERR_INVALID_ARG  # counters always reorder
    assert ms.ms_tune_set(ms.MOD, 0, 5, 3, 2, 1, 1) == ms.MS_OK
    assert ms.ms_tune_get(ms.MOD, 0, 5, 3) == (2, 1, 1)
    ms.ms_tune_reset()
    assert ms.ms_tune_get(ms.MOD, 0, 5, 3) == (0, 2, 1)
    assert ms.ms_tune_get_sort(1, 3) == 0  # one-sweep passes by default
    assert ms.ms_tune_set_sort(1, 3, 1) == ms.MS_OK and ms.ms_tune_get_sort(1, 3) == 1
    assert ms.ms_tune_set_sort(1, 3, 2) == ms.MS_ERR_INVALID_ARG and ms.ms_tune_set_sort(2, 3, 1) == ms.MS_ERR_INVALID_ARG
    ms.ms_tune_reset()
    assert ms.ms_tune_get_sort(1, 3) == 0
    # batched kernels: counters for m <= 32, peer tables beyond, by default
    assert ms.ms_tune_get_batch(ms.MOD, 1, 5, 2) == (ms.MS_OK, 0, 2)
    assert ms.ms_tune_get_batch(ms.MOD, 1, 8, 2) == (ms.MS_OK, 0, 1)
    assert ms.ms_tune_set_batch(ms.MOD, 1, 8, 2, 0, 2) == ms.MS_ERR_INVALID_ARG  # counters need log2 m <= 5
    assert ms.ms_tune_set_batch(ms.MOD, 1, 5, 2, 1, 2) == ms.MS_ERR_INVALID_ARG  # counters: 8 x 16 only
    assert ms.ms_tune_set_batch(ms.MOD, 1, 5, 2, 2, 1) == ms.MS_ERR_INVALID_ARG  # shapes 0, 1
    assert ms.ms_tune_set_batch(ms.MOD, 1, 5, 2, 0, 0) == ms.MS_ERR_INVALID_ARG  # no plain ballots
    assert ms.ms_tune_set_batch(ms.MOD, 1, 5, 2, 1, 3) == ms.MS_OK
    assert ms.ms_tune_get_batch(ms.MOD, 1, 5, 2) == (ms.MS_OK, 1, 3)
    ms.ms_tune_reset()
    assert ms.ms_tune_get_batch(ms.MOD, 1, 5, 2) == (ms.MS_OK, 0, 2)


def test_shipped_tuning_table_is_valid(lib):
    """Every entry of the shipped tuning table is a variant the library accepts."""
    import json

    from paper_1701_01189_gb300 import autotune

    ms.ms_tune_reset()
    try:
        if os.path.exists(autotune.DEFAULT_PATH):
            d = json.load(open(autotune.DEFAULT_PATH))
            n = len(d["entries"]) + len(d.get("sort", [])) + len(d.get("batch", []))
            assert autotune.load() == n > 0
    finally:
        ms.ms_tune_reset()
