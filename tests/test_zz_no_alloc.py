"""fftu_exec_noalloc: the allocation-free entry point against fftu_exec.

Some callers cannot allocate device memory where they run the FFT (code under
CUDA graph capture, plugins whose host owns every allocation, real-time loops
that must not enter the allocator).  fftu_exec_noalloc serves them with scratch
held in static device arrays.  This test calls it through the C ABI twice in a
row (the second call reuses the first call's scratch and counters) and checks
both outputs against fftu_exec's, at the tolerance the parity tests use for
complex64 (relative L2 <= 1e-5 * log2 N).  It lives in a file of its own that
pytest collects last, and passes alone in a fresh process as well.
"""
import math

import numpy as np
import pytest

from fftu_inputs import complex_uniform

pytestmark = pytest.mark.gpu

SHAPE, P = (512, 512, 512), (8, 8, 8)


@pytest.fixture(scope="module")
def fftu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as f
    return f


def _rel(a, b):
    import torch
    return float((torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item())


@pytest.mark.parametrize("inverse", [False, True])
def test_noalloc_matches_exec_twice(fftu, inverse):
    import torch
    x = torch.from_numpy(complex_uniform(4242, SHAPE, dtype=np.complex64)).cuda()
    direction = fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD
    with fftu.Plan(SHAPE, P, inverse=inverse) as plan:
        ref = plan.exec(x)
    tol = 1e-5 * math.log2(x.numel())
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full_like(x, float("nan"))
        fftu.fftu_exec_noalloc(3, SHAPE, P, fftu.FFTU_C64, direction, x.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert _rel(out, ref) <= tol


def test_noalloc_rejects_what_it_cannot_run(fftu):
    import torch
    x = torch.zeros(SHAPE, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    cases = [
        ((512, 512, 512), (4, 4, 4), fftu.FFTU_C64, x, y, 3),   # residue unit of 64 MiB > 16 MiB slot
        ((512, 512, 512), (8, 8, 8), fftu.FFTU_C64, x, x, 1),   # in == out
        ((512, 512, 512), (8, 8, 8), fftu.FFTU_C128, x, y, 3),  # complex64 only
        ((512, 512, 512), (32, 8, 8), fftu.FFTU_C64, x, y, 2),  # 32^2 does not divide 512
        ((512, 512, 512), (16, 8, 8), fftu.FFTU_C64, x, y, 3),  # p_0 = p_1 = p_2 only
    ]
    for shape, p, dt, a, b, code in cases:
        with pytest.raises(fftu.FFTUError) as ei:
            fftu.fftu_exec_noalloc(3, shape, p, dt, fftu.FFTU_FORWARD, a.data_ptr(), b.data_ptr(), 0)
        assert ei.value.status == code
        assert fftu.fftu_last_error()
