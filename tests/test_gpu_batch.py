"""The batched multisplit: every segment of a plan equals the oracle's
multisplit of that segment alone (bit exact), for keys and pairs, every
bucket kind, segment sizes from 0 to several tiles, through the direct launch
and the CUDA-graph replay, twice in a row."""
import numpy as np
import pytest

import oracle
import synthetic
from parity import Case, clustered_splitters, to_dev, to_host

pytestmark = pytest.mark.gpu

# 0 to several tiles of 4096 keys; 8 and 9 tiles and 70000 (18 tiles) cross
# the 8-tile work items of the per-thread-counter batched kernel
SIZES = [0, 1, 31, 4095, 4096, 4097, 10000, 3 * 4096 + 5, 8 * 4096, 8 * 4096 + 1, 70000, 255, 2]


def cases():
    return [Case(oracle.MOD, 32), Case(oracle.RANGE_U32, 8, splitters=synthetic.range_splitters(8, 1)),
            Case(oracle.RADIX, 256, shift=24, bits=8),
            Case(oracle.DELTA_F32, 64, x0=0.0, delta=float(np.float32(1000.0) / np.float32(64))),
            Case(oracle.MOD, 1),
            Case(oracle.RANGE_U32, 256, splitters=synthetic.range_splitters(256, 2)),
            Case(oracle.RANGE_U32, 64, splitters=clustered_splitters(64, 3)),
            Case(oracle.RANGE_U32, 32, splitters=clustered_splitters(32, 4))]


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("ci", range(8))
def test_batch_matches_oracle(ci, pairs):
    import torch

    import paper_1701_01189_gb300 as ms

    case = cases()[ci]
    keys = [synthetic.uniform_f32_1000(n, 10 + i) if case.kind == oracle.DELTA_F32 else synthetic.uniform_u32(n, 10 + i)
            for i, n in enumerate(SIZES)]
    vals = [synthetic.index_values(n) for n in SIZES] if pairs else None
    dk = [to_dev(k) for k in keys]
    dv = [to_dev(v) for v in vals] if pairs else None
    plan = ms.BatchPlan(dk, dv, case.gpu_spec())
    try:
        for graph in (False, True, True):
            for t in plan.keys_out:
                t.fill_(-1)
            plan.run(graph=graph)
            torch.cuda.synchronize()
            assert ms.device_status() == ms.MS_OK
            for i, n in enumerate(SIZES):
                ok, ov, ooff = oracle.multisplit(keys[i], None if vals is None else vals[i], case.oracle_spec())
                np.testing.assert_array_equal(to_host(plan.keys_out[i]), ok, err_msg=f"segment {i} n={n}")
                if pairs:
                    np.testing.assert_array_equal(to_host(plan.vals_out[i]), ov, err_msg=f"segment {i} values")
                np.testing.assert_array_equal(to_host(plan.offsets[i]).astype(np.uint64), ooff)
    finally:
        plan.close()


def test_batch_config_4096_segments_small():
    """The batched configuration's shape at a tenth of its total size: 4096
    segments with log-uniform sizes in [2^8, 2^16], key mod 32, pairs."""
    import torch

    import paper_1701_01189_gb300 as ms

    sizes = synthetic.segment_sizes(4096, 8, 16, 42)
    keys = [synthetic.uniform_u32(int(n), 1000 + i) for i, n in enumerate(sizes)]
    vals = [synthetic.index_values(int(n)) for n in sizes]
    plan = ms.BatchPlan([to_dev(k) for k in keys], [to_dev(v) for v in vals], ms.BucketSpec.mod(32))
    try:
        plan.run(graph=True)
        torch.cuda.synchronize()
        assert ms.device_status() == ms.MS_OK
        for i in range(0, 4096, 97):
            ok, ov, ooff = oracle.multisplit(keys[i], vals[i], oracle.Spec(oracle.MOD, 32))
            np.testing.assert_array_equal(to_host(plan.keys_out[i]), ok)
            np.testing.assert_array_equal(to_host(plan.vals_out[i]), ov)
            np.testing.assert_array_equal(to_host(plan.offsets[i]).astype(np.uint64), ooff)
    finally:
        plan.close()


@pytest.mark.slow
def test_batch_config_4096_segments_full_size():
    """The batched configuration as the benchmark times it: 4096 segments of
    floor(2^U) pairs, U ~ U(8, 20) (about 516 M pairs), key mod 32, value =
    index within the segment, graph replay.  Checked against the oracle on the
    20 largest and 20 smallest segments and every 61st, and, on the device, the
    whole output against one plain launch per segment."""
    import torch

    import paper_1701_01189_gb300 as ms

    sizes = synthetic.segment_sizes(4096, 8, 20, 2024)  # the benchmark's seed
    total = int(sizes.sum())
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    hk = synthetic.uniform_u32(total, 2025)
    kall = to_dev(hk)
    vall = torch.empty_like(kall)
    for st_, n_ in zip(starts, sizes):
        vall[int(st_):int(st_ + n_)] = torch.arange(int(n_), dtype=torch.int32, device="cuda")
    ko, vo = torch.full_like(kall, -1), torch.full_like(kall, -1)
    offs = torch.full((4096, 33), -1, dtype=torch.int32, device="cuda")
    segs = [(kall.data_ptr() + 4 * int(s0), vall.data_ptr() + 4 * int(s0), ko.data_ptr() + 4 * int(s0),
             vo.data_ptr() + 4 * int(s0), offs[i].data_ptr(), int(n_)) for i, (s0, n_) in enumerate(zip(starts, sizes))]
    spec = ms.BucketSpec.mod(32).c()
    st, plan = ms.ms_batch_plan_create(segs, spec)
    assert st == ms.MS_OK
    sptr = torch.cuda.current_stream().cuda_stream
    try:
        for _ in range(2):  # a replay over outputs already written
            assert ms.ms_batch_run_graph(plan, sptr) == ms.MS_OK
        torch.cuda.synchronize()
        assert ms.device_status() == ms.MS_OK
    finally:
        ms.ms_batch_plan_destroy(plan)
    order = np.argsort(sizes, kind="stable")
    pick = sorted(set(order[:20].tolist()) | set(order[-20:].tolist()) | set(range(0, 4096, 61)))
    for i in pick:
        s0, n_ = int(starts[i]), int(sizes[i])
        ok, ov, ooff = oracle.multisplit(hk[s0:s0 + n_], synthetic.index_values(n_), oracle.Spec(oracle.MOD, 32))
        np.testing.assert_array_equal(to_host(ko[s0:s0 + n_]), ok, err_msg=f"segment {i} n={n_}")
        np.testing.assert_array_equal(to_host(vo[s0:s0 + n_]), ov, err_msg=f"segment {i} values")
        np.testing.assert_array_equal(to_host(offs[i]).astype(np.uint64), ooff, err_msg=f"segment {i} offsets")
    # every segment against one plain launch per segment, compared on the device
    pk, pvo = torch.full_like(kall, -2), torch.full_like(kall, -2)
    poffs = torch.full((4096, 33), -2, dtype=torch.int32, device="cuda")
    for i, (s0, n_) in enumerate(zip(starts, sizes)):
        o = 4 * int(s0)
        assert ms.ms_multisplit_pairs(kall.data_ptr() + o, vall.data_ptr() + o, int(n_), spec, pk.data_ptr() + o,
                                      pvo.data_ptr() + o, poffs[i].data_ptr(), sptr) == ms.MS_OK
    torch.cuda.synchronize()
    assert torch.equal(pk, ko) and torch.equal(pvo, vo) and torch.equal(poffs, offs)


BATCH_VARIANT_CASES = [Case(oracle.MOD, 32), Case(oracle.RANGE_U32, 256, splitters=synthetic.range_splitters(256, 5)),
                       Case(oracle.DELTA_F32, 8, x0=0.0, delta=float(np.float32(1000.0) / np.float32(8)))]


@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
@pytest.mark.parametrize("ci", range(3), ids=["mod32", "range256", "delta8"])
def test_every_batched_kernel_variant(ci, pairs):
    """Each kernel the batched variant table can select (per-thread counters,
    peer tables or ballot peers; 8 x 16 or 16 x 8 tiles), forced for this
    identifier, against the oracle; the table is restored afterwards."""
    import torch

    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300 import autotune

    case = BATCH_VARIANT_CASES[ci]
    sizes = SIZES + [200_000, 65_536]
    keys = [synthetic.uniform_f32_1000(n, 40 + i) if case.kind == oracle.DELTA_F32 else synthetic.uniform_u32(n, 40 + i)
            for i, n in enumerate(sizes)]
    vals = [synthetic.index_values(n) for n in sizes] if pairs else None
    dk = [to_dev(k) for k in keys]
    dv = [to_dev(v) for v in vals] if pairs else None
    log2m = (case.m - 1).bit_length()
    expect = [oracle.multisplit(keys[i], None if vals is None else vals[i], case.oracle_spec()) for i in range(len(sizes))]
    try:
        for shape, rank in autotune.batch_variants(log2m):
            for sc in range(4):
                assert ms.ms_tune_set_batch(case.kind, int(pairs), log2m, sc, shape, rank) == ms.MS_OK
            plan = ms.BatchPlan(dk, dv, case.gpu_spec())
            try:
                plan.run(graph=True)
                torch.cuda.synchronize()
                assert ms.device_status() == ms.MS_OK
                for i, n in enumerate(sizes):
                    ok, ov, ooff = expect[i]
                    what = f"variant ({shape}, {rank}) segment {i} n={n}"
                    np.testing.assert_array_equal(to_host(plan.keys_out[i]), ok, err_msg=what)
                    if pairs:
                        np.testing.assert_array_equal(to_host(plan.vals_out[i]), ov, err_msg=what)
                    np.testing.assert_array_equal(to_host(plan.offsets[i]).astype(np.uint64), ooff, err_msg=what)
            finally:
                plan.close()
    finally:
        ms.ms_tune_reset()
        autotune.load()


def test_batch_rejects_mixed_segments():
    import paper_1701_01189_gb300 as ms

    spec = ms.BucketSpec.mod(4).c()
    st, _ = ms.ms_batch_plan_create([(0x1000, 0x2000, 0x3000, 0x4000, None, 4), (0x5000, None, 0x6000, None, None, 4)],
                                    spec)
    assert st == ms.MS_ERR_INVALID_ARG
