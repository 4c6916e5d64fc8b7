"""GB300-native stable multisplit and multisplit radix sort (Ashkiani et al., "GPU Multisplit").

The compute path is the CUDA library ``libms.so`` (C ABI in ``include/ms.h``),
built for sm_103a by ``paper_1701_01189_gb300.build``.  This package is its
thin Python binding (``_binding``) plus host-side helpers (``metrics``).
"""
from ._binding import (  # noqa: F401
    DELTA_F32, MAX_M, MAX_M_WIDE, MOD, MS_ERR_CUDA, MS_ERR_INVALID_ARG, MS_ERR_OUT_OF_MEMORY, MS_ERR_TIMEOUT,
    MS_ERR_UNSUPPORTED, MS_OK, RADIX, RANGE_U32, BatchPlan, BucketSpec, MsError, ms_batch_plan_create,
    ms_batch_plan_create_dynamic, ms_batch_plan_destroy, ms_batch_plan_set_segments, ms_batch_run, ms_batch_run_graph, device_status, lib,
    ms_device_status, ms_histogram, histogram, ms_multisplit_keys, ms_multisplit_keys_noalloc, ms_multisplit_pairs, ms_radix_sort, ms_radix_sort_r, ms_stage_times, ms_stage_timing,
    ms_status_string, ms_test_expire_lookback, ms_test_expire_lookback_noalloc, ms_noalloc_status, ms_shutdown,
    ms_multisplit_pairs_batched, segment_records, ms_tune_get, ms_tune_get_sort, ms_tune_reset, ms_tune_set, ms_tune_set_sort, ms_tune_size_class,
    ms_tune_set_batch, ms_tune_get_batch,
    ms_version,
    multisplit_keys, multisplit_pairs, radix_sort,
)
