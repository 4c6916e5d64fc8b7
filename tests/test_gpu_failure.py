"""Failure detection without a GPU fault: a bounded device-side wait on a flag
that nothing sets runs out, the kernel records MS_ERR_TIMEOUT and returns, the
host reads it, and the context stays usable for a correct multisplit after."""
import numpy as np
import pytest

import oracle
import synthetic
from parity import Case, check_multisplit

pytestmark = pytest.mark.gpu


def test_lookback_wait_expires_and_context_survives():
    import torch

    import paper_1701_01189_gb300 as ms
    from paper_1701_01189_gb300.build import build

    build()
    s = torch.cuda.current_stream().cuda_stream
    assert ms.ms_device_status(s) == ms.MS_OK
    assert ms.ms_test_expire_lookback(s) == ms.MS_OK
    assert ms.ms_device_status(s) == ms.MS_ERR_TIMEOUT
    assert ms.ms_device_status(s) == ms.MS_OK  # reading clears it
    keys = synthetic.uniform_u32(50_000, 3)
    check_multisplit(keys, synthetic.index_values(50_000), Case(oracle.MOD, 13))
