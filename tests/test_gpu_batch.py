"""Many uneven transforms in one persistent launch (fftu_batch_*), against the FP64 oracle."""
import math

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


def uneven_shapes(count, seed):
    """Each n_l drawn independently from {32, 64, 128} (cubes included)."""
    rng = np.random.default_rng(seed)
    return [tuple(int(v) for v in rng.choice([32, 64, 128], size=3)) for _ in range(count)]


def _run_batch(fftu, shapes, inverse, dtype=np.complex64, in_place=False, graph=False):
    import torch
    xs = [torch.from_numpy(complex_uniform(100 + i, s, dtype=dtype)).cuda() for i, s in enumerate(shapes)]
    outs = [x if in_place else torch.empty_like(x) for x in xs]
    keep = [x.clone() for x in xs] if in_place else xs
    plans = [fftu.Plan(s, None, dtype=xs[0].dtype, inverse=inverse) for s in shapes]
    b = fftu.fftu_batch_create([p.handle for p in plans])
    try:
        stream = torch.cuda.current_stream()
        if graph:
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                with torch.cuda.graph(g, stream=side):
                    fftu.fftu_batch_exec(b, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs],
                                         side.cuda_stream)
            stream.wait_stream(side)
            for _ in range(2):  # replays give the same result (inputs are not in place here)
                g.replay()
        else:
            fftu.fftu_batch_exec(b, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs], stream.cuda_stream)
        torch.cuda.synchronize()
        fftu.fftu_batch_check_status(b)
    finally:
        fftu.fftu_batch_destroy(b)
        for p in plans:
            p.close()
    return [k.cpu().numpy() for k in keep], [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("inverse", [False, True])
def test_batch_matches_oracle(fftu, inverse):
    shapes = uneven_shapes(12, seed=3)
    xs, ys = _run_batch(fftu, shapes, inverse)
    for x, y in zip(xs, ys):
        ref = oracle.fftn(x.astype(np.complex128), inverse=inverse)
        assert oracle.rel_l2(y, ref) <= 1e-5 * math.log2(x.size)


def test_batch_in_place_and_complex128(fftu):
    shapes = [(32, 64, 32), (64, 32, 128), (16, 16, 16, 16)]
    xs, ys = _run_batch(fftu, shapes, False, dtype=np.complex128, in_place=True)
    for x, y in zip(xs, ys):
        assert oracle.rel_l2(y, oracle.fftn(x)) <= 1e-12


def test_batch_captured_in_cuda_graph(fftu):
    shapes = uneven_shapes(6, seed=9)
    xs, ys = _run_batch(fftu, shapes, False, graph=True)
    for x, y in zip(xs, ys):
        assert oracle.rel_l2(y, oracle.fftn(x.astype(np.complex128))) <= 1e-5 * math.log2(x.size)


def test_batch_rejects_mixed_plans(fftu):
    import torch
    with fftu.Plan((32, 32, 32), None) as a, fftu.Plan((32, 32, 32), None, inverse=True) as b, \
            fftu.Plan((32, 32, 32), None, dtype=torch.complex128) as c:
        for pair in ((a, b), (a, c)):
            with pytest.raises(fftu.FFTUError) as ei:
                fftu.fftu_batch_create([pair[0].handle, pair[1].handle])
            assert ei.value.status == 1
    with fftu.Plan((32768,), (128,)) as longline:   # phase A alternates with a workspace
        with pytest.raises(fftu.FFTUError) as ei:
            fftu.fftu_batch_create([longline.handle])
        assert ei.value.status == 3


def test_batch_after_smaller_batch_is_created(fftu):
    """The kernel's shared-memory limit is shared by all batches: creating a batch with smaller
    tiles must not break a batch with larger ones (found with the serving loop)."""
    import torch
    big_shapes = [(128, 128, 128), (64, 128, 32)]
    xs = [torch.from_numpy(complex_uniform(300 + i, s, dtype=np.complex64)).cuda() for i, s in enumerate(big_shapes)]
    outs = [torch.empty_like(x) for x in xs]
    plans = [fftu.Plan(s, None) for s in big_shapes]
    small = fftu.Plan((8, 8), None)
    big = fftu.fftu_batch_create([p.handle for p in plans])
    little = fftu.fftu_batch_create([small.handle])
    try:
        stream = torch.cuda.current_stream()
        fftu.fftu_batch_exec(big, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs], stream.cuda_stream)
        torch.cuda.synchronize()
        fftu.fftu_batch_check_status(big)
    finally:
        fftu.fftu_batch_destroy(little)
        fftu.fftu_batch_destroy(big)
        for p in plans + [small]:
            p.close()
    for x, y in zip(xs, outs):
        ref = oracle.fftn(x.cpu().numpy().astype(np.complex128))
        assert oracle.rel_l2(y.cpu().numpy(), ref) <= 1e-5 * math.log2(x.numel())
