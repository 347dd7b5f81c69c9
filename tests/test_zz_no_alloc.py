"""fftu_exec_noalloc: the allocation-free entry point, against the FP64 oracle and fftu_exec.

Some callers cannot allocate device memory where they run the FFT (code under
CUDA graph capture, plugins whose host owns every allocation, real-time loops
that must not enter the allocator).  fftu_exec_noalloc serves them with scratch
held in static device arrays.  These tests call it through the C ABI:

* twice in a row (the second call reuses the first call's scratch and
  counters), each output against the FP64 oracle on the same input and against
  fftu_exec's output, at the complex64 tolerance of the parity tests
  (relative L2 <= 1e-5 * log2 N);
* captured into a CUDA graph after one eager call, the graph replayed on two
  fresh inputs, each result against the oracle;
* the failure-detection path: a bounded device wait that expires into the
  shared status word is reported once by fftu_noalloc_check_status, the word is
  then clear, and the next transform is still right.

The file is collected last and passes alone in a fresh process as well.
"""
import math

import numpy as np
import pytest

import oracle
from fftu_inputs import complex_uniform

pytestmark = pytest.mark.gpu

SHAPE, P = (512, 512, 512), (8, 8, 8)
TOL = 1e-5 * math.log2(512 ** 3)


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


def _oracle(x, inverse):
    return oracle.fftn(x.astype(np.complex128), inverse=inverse)


@pytest.mark.parametrize("inverse", [False, True])
def test_noalloc_matches_oracle_twice(fftu, inverse):
    import torch
    x = complex_uniform(4242 + int(inverse), SHAPE, dtype=np.complex64)
    xt = torch.from_numpy(x).cuda()
    direction = fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD
    with fftu.Plan(SHAPE, P, inverse=inverse) as plan:
        ref_exec = plan.exec(xt)
    ref = _oracle(x, inverse)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full_like(xt, float("nan"))
        fftu.fftu_exec_noalloc(3, SHAPE, P, fftu.FFTU_C64, direction, xt.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        fftu.fftu_noalloc_check_status(stream)
        err = oracle.rel_l2(out.cpu().numpy(), ref)
        assert err <= TOL, err
        assert _rel(out, ref_exec) <= TOL


def test_noalloc_graph_capture_replays(fftu):
    """One eager call, then the call captured into a CUDA graph and replayed on fresh inputs."""
    import torch
    xin = torch.empty(SHAPE, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(xin)
    xin.copy_(torch.from_numpy(complex_uniform(31, SHAPE, dtype=np.complex64)))
    stream = torch.cuda.current_stream().cuda_stream
    fftu.fftu_exec_noalloc(3, SHAPE, P, fftu.FFTU_C64, fftu.FFTU_FORWARD, xin.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cs = torch.cuda.current_stream().cuda_stream
        fftu.fftu_exec_noalloc(3, SHAPE, P, fftu.FFTU_C64, fftu.FFTU_FORWARD, xin.data_ptr(), out.data_ptr(), cs)
    for seed in (32, 33):
        x = complex_uniform(seed, SHAPE, dtype=np.complex64)
        xin.copy_(torch.from_numpy(x))
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        fftu.fftu_noalloc_check_status(stream)
        err = oracle.rel_l2(out.cpu().numpy(), _oracle(x, False))
        assert err <= TOL, (seed, err)
    del g


def test_noalloc_timeout_is_reported_once(fftu):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    fftu.fftu_noalloc_check_status(stream)  # start from a clear word
    fftu.fftu_noalloc_selftest_timeout(0.05, stream)
    with pytest.raises(fftu.FFTUError) as ei:
        fftu.fftu_noalloc_check_status(stream)
    assert ei.value.status == 6  # FFTU_ERR_TIMEOUT
    fftu.fftu_noalloc_check_status(stream)  # read-and-clear: now clear
    x = complex_uniform(77, SHAPE, dtype=np.complex64)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    fftu.fftu_exec_noalloc(3, SHAPE, P, fftu.FFTU_C64, fftu.FFTU_FORWARD, xt.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    fftu.fftu_noalloc_check_status(stream)
    assert oracle.rel_l2(out.cpu().numpy(), _oracle(x, False)) <= TOL


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
    with pytest.raises(fftu.FFTUError) as ei:
        fftu.fftu_noalloc_selftest_timeout(5.0, 0)  # budget out of range
    assert ei.value.status == 1
