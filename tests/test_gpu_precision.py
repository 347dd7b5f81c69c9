"""Split-precision tensor-core radix-16 stages (fftu_options.precision) against the FP64 oracle.

Assertion: every result meets the complex64 bound the native path is held to, relative L2
<= 1e-5 log2 N against the FP64 oracle, so the split forms are reported at the same stated
accuracy as the FP32 CUDA-core path.

Error model (printed beside each result as a diagnostic, not asserted): an operand v is carried
as v_hi + v_lo in a 16-bit type with unit roundoff u (bfloat16 2^-8, float16 2^-11), so its
representation error is at most u^2 |v|; with the dropped lo x lo product, each real 16-point
product has absolute error at most 3 u^2 |F| |x| entrywise, i.e. a relative L2 error of at most
12 u^2 per radix-16 stage (|F| has 16 ones per row against ||F||_2 = 4).  Stages compose
additively to first order, so the model's bound is S * 12 u^2 plus the FP32 budget, S =
radix-16 stages per element.  Inputs: uniform[-1, 1) and log-uniform magnitudes over [1e-3, 1e3)."""
import math

import numpy as np
import pytest

import oracle
from fftu_inputs import complex_loguniform, complex_uniform

pytestmark = pytest.mark.gpu

U = {1: 2.0 ** -8, 2: 2.0 ** -11}


@pytest.fixture(scope="module")
def fftu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as f
    return f


def tc_stages(shape, p):
    return sum(int(math.log2(n // q)) // 4 for n, q in zip(shape, p))


def tolerance(shape):
    """The complex64 bound every result is asserted against."""
    return 1e-5 * math.log2(math.prod(shape))


def model_bound(shape, p, precision):
    """First-order error model of the split stages (diagnostic only)."""
    return tc_stages(shape, p) * 12 * U[precision] ** 2 + tolerance(shape)


def make(kind, seed, shape):
    f = complex_uniform if kind == "uniform" else complex_loguniform
    return f(seed, shape, dtype=np.complex64)


def run(fftu, x, p, precision, inverse=False):
    import torch
    t = torch.from_numpy(x).cuda()
    with fftu.Plan(x.shape, p, dtype=t.dtype, inverse=inverse, precision=precision) as plan:
        y = plan.exec(t)
        torch.cuda.synchronize()
        plan.check_device_status()
        info = plan.info
    return y.cpu().numpy(), info


CASES = [((64, 64, 64), (4, 4, 4)),        # L = 16: one tensor-core stage per axis
         ((128, 128, 128), (2, 2, 2)),     # L = 64: radix 16 (tensor cores) then radix 4
         ((32, 512), (2, 2)),              # L = 16 and 256 (two tensor-core stages)
         ((8192,), (4,)),                  # L = 2048 = 16 * 16 * 8
         ((16, 16, 16, 16), (2, 2, 2, 2))]  # L = 8: no radix-16 stage, CUDA cores only


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
@pytest.mark.parametrize("precision", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("kind", ["uniform", "loguniform"])
@pytest.mark.parametrize("inverse", [False, True], ids=["fwd", "inv"])
def test_split_precision_matches_oracle(fftu, case, precision, kind, inverse):
    shape, p = case
    x = make(kind, 31, shape)
    y, info = run(fftu, x, p, precision, inverse)
    assert info["precision"] == precision and info["schedule"] == fftu.FFTU_SCHED_GENERIC_A
    err = oracle.rel_l2(y, oracle.fftn(x.astype(np.complex128), inverse=inverse))
    print(f"split {'bf16' if precision == 1 else 'fp16'} {kind} {shape} {'inv' if inverse else 'fwd'}: "
          f"rel L2 {err:.3e} (bound {tolerance(shape):.1e}, error model {model_bound(shape, p, precision):.1e})")
    assert err <= tolerance(shape)


def test_full_size_512_errors(fftu):
    """The 512^3 workload (p = 8^3, L = 64 = 16 x 4) with both split precisions and both input
    distributions, against the full FP64 oracle; the native FP32 path on the same schedule is
    measured alongside."""
    shape, p = (512, 512, 512), (8, 8, 8)
    for kind in ("uniform", "loguniform"):
        x = make(kind, 2027, shape)
        ref = oracle.fftn(x.astype(np.complex128))
        for precision in (0, 1, 2):
            y, _ = run(fftu, x, p, precision)
            err = oracle.rel_l2(y, ref)
            print(f"512^3 {kind} precision {precision}: rel L2 {err:.3e} (bound {tolerance(shape):.1e})")
            assert err <= tolerance(shape)
            del y


def test_precision_validation(fftu):
    import torch
    with pytest.raises(fftu.FFTUError) as ei:   # complex128 has no split-precision stages
        fftu.Plan((64, 64), None, dtype=torch.complex128, precision=1)
    assert ei.value.status == 3
    with pytest.raises(fftu.FFTUError) as ei:   # the fused schedule has no strided radix-16 stages
        fftu.Plan((64, 64), None, schedule=fftu.FFTU_SCHED_FUSED, precision=2)
    assert ei.value.status == 1
    with fftu.Plan((64, 64, 64), None, precision=1) as a:
        with pytest.raises(fftu.FFTUError) as ei:
            fftu.fftu_batch_create([a.handle])
        assert ei.value.status == 3
