"""Failure detection on the GPU without a fault: a bounded device wait on a word nothing sets gives
up after its budget, reports FFTU_ERR_TIMEOUT through the status word, and the context keeps
working (a transform right after matches the oracle)."""
import numpy as np
import pytest

import oracle
from fftu_inputs import complex_uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fftu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as f
    return f


@pytest.mark.parametrize("limit", [0.01, 0.2])
def test_expired_wait_reports_timeout_and_context_survives(fftu, limit):
    import torch
    waited = fftu.fftu_selftest_bounded_wait(limit)
    assert limit <= waited < limit + 0.5
    x = complex_uniform(91, (32, 32, 32), dtype=np.complex64)
    with fftu.Plan(x.shape, (2, 2, 2)) as plan:
        y = plan.exec(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        plan.check_device_status()  # the plan's own status word is clean
    assert oracle.rel_l2(y.cpu().numpy(), oracle.fftn(x.astype(np.complex128))) < 1e-4
