"""Full-array parity at the configured full sizes: every output element against the FP64 oracle.

Workloads (seeded uniform[-1, 1) inputs, as in the parity tests):
* 1024^3 complex64 (8 GiB) at every cyclic grid the library runs it on: the default p = 8^3
  (two-kernel phase A), p = 4^3 (strided passes), p = 16^3 and the tuned p = 16 x 16 x 8
  (persistent ring with 32 MiB residue units); forward for all four, inverse for the default
  and tuned grids.  The oracle's result (16 GiB) is computed once per direction and shared.
* 4D 64^4 complex128 at p = 8^4 and 5D 32^5 complex64 at p = 4^5, both directions.
* 2D 16384^2 complex64 with the plan the tuner picks (p = 16^2, per-axis phase A, strided tile of
  4096 elements), both directions.
* the batch of 64 uneven 3D complex64 transforms (each n_l drawn from {32, 64, 128}) in one
  persistent launch per direction, each transform against the oracle.

Tolerance (relative L2 over the whole array): 1e-12 for complex128, 1e-5 log2 N for complex64;
for complex64 the max-abs error over max|ref| is held to the same bound.  The comparisons run in
chunks of 2^26 elements so that host memory stays near three copies of the array.
"""
import gc
import math

import numpy as np
import pytest

import oracle
from fftu_inputs import complex_uniform

pytestmark = pytest.mark.gpu

CHUNK = 1 << 26


def tolerance(dtype, N):
    return 1e-12 if np.dtype(dtype) == np.complex128 else 1e-5 * max(1.0, math.log2(N))


@pytest.fixture(scope="module")
def fftu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as f
    return f


def errors(y, ref):
    """(relative L2, max-abs / max|ref|) in FP64, accumulated over chunks."""
    y, ref = y.reshape(-1), ref.reshape(-1)
    num = den = 0.0
    emax = rmax = 0.0
    for i in range(0, y.size, CHUNK):
        r = ref[i:i + CHUNK].astype(np.complex128, copy=False)
        dlt = y[i:i + CHUNK].astype(np.complex128) - r
        num += float(np.vdot(dlt, dlt).real)
        den += float(np.vdot(r, r).real)
        emax = max(emax, float(np.abs(dlt).max()))
        rmax = max(rmax, float(np.abs(r).max()))
    return math.sqrt(num / den), emax / rmax


def gpu_transform(fftu, x, p, inverse=False, **opts):
    """One transform through fftu_exec on a device copy of x; the result back on the host."""
    import torch
    xt = torch.from_numpy(x).cuda()
    with fftu.Plan(x.shape, p, dtype=xt.dtype, inverse=inverse, **opts) as plan:
        y = plan.exec(xt)
        torch.cuda.synchronize()
        plan.check_device_status()
        info = plan.info
    del xt
    out = y.cpu().numpy()
    del y
    torch.cuda.empty_cache()
    return out, info


def check(y, ref, dtype, N, label):
    err, emax = errors(y, ref)
    print(f"{label}: relative L2 {err:.3e}, max-abs / max|ref| {emax:.3e}")
    assert err <= tolerance(dtype, N), label
    if np.dtype(dtype) == np.complex64:
        assert emax <= tolerance(dtype, N), label


# ---- 1024^3 complex64 -----------------------------------------------------------------------

SHAPE_1024 = (1024, 1024, 1024)
_cache = {}


def _input_1024():
    if "x" not in _cache:
        _cache["x"] = complex_uniform(2026, SHAPE_1024, dtype=np.complex64)
    return _cache["x"]


def _oracle_1024(inverse):
    key = ("ref", inverse)
    if key not in _cache:
        for k in [k for k in _cache if k[0] == "ref"]:  # hold one 16 GiB reference at a time
            del _cache[k]
        gc.collect()
        _cache[key] = oracle.fftn(_input_1024(), inverse=inverse)
    return _cache[key]


CASES_1024 = [((8, 8, 8), False), ((16, 16, 8), False), ((16, 16, 16), False), ((4, 4, 4), False),
              ((8, 8, 8), True), ((16, 16, 8), True)]


@pytest.mark.parametrize("p,inverse", CASES_1024,
                         ids=[("inv_" if inv else "fwd_") + "p" + "x".join(map(str, p)) for p, inv in CASES_1024])
def test_full_1024(fftu, p, inverse):
    x = _input_1024()
    y, info = gpu_transform(fftu, x, p, inverse=inverse)
    check(y, _oracle_1024(inverse), np.complex64, x.size,
          f"1024^3 p={p} {'inverse' if inverse else 'forward'} (phase-A launches {info['launches_phase_a']})")
    del y
    if (p, inverse) == CASES_1024[-1]:
        _cache.clear()
        gc.collect()


# ---- other dimensionalities --------------------------------------------------------------------

OTHER = [((64, 64, 64, 64), (8, 8, 8, 8), np.complex128, {}),
         ((32, 32, 32, 32, 32), (4, 4, 4, 4, 4), np.complex64, {}),
         # the plan the tuner picks for 16384^2: per-axis phase A (schedule 3), strided tile 4096
         ((16384, 16384), (16, 16), np.complex64, {"schedule": 3, "tile": 4096})]


@pytest.mark.parametrize("case", OTHER, ids=["64x4_c128_p8", "32x5_c64_p4", "16384x2_c64_p16_tuned"])
@pytest.mark.parametrize("inverse", [False, True], ids=["fwd", "inv"])
def test_full_other_dimensionalities(fftu, case, inverse):
    shape, p, dt, opts = case
    x = complex_uniform(2030 + len(shape), shape, dtype=dt)
    y, info = gpu_transform(fftu, x, p, inverse=inverse, **opts)
    if opts.get("tile"):
        assert info["tile"] == opts["tile"] and info["schedule"] == opts["schedule"]
    ref = oracle.fftn(x, inverse=inverse)
    check(y, ref, dt, x.size, f"{shape} p={p} {np.dtype(dt).name} {'inverse' if inverse else 'forward'}")


# ---- the batch of 64 uneven transforms ---------------------------------------------------------

def uneven_shapes(count, seed):
    """Each n_l drawn independently from {32, 64, 128} (cubes included), as the benchmark draws them."""
    rng = np.random.default_rng(seed)
    return [tuple(int(v) for v in rng.choice([32, 64, 128], size=3)) for _ in range(count)]


@pytest.mark.parametrize("inverse", [False, True], ids=["fwd", "inv"])
def test_full_batch_64_uneven(fftu, inverse):
    import torch
    shapes = uneven_shapes(64, seed=2024)
    xs_h = [complex_uniform(5000 + i, s, dtype=np.complex64) for i, s in enumerate(shapes)]
    xs = [torch.from_numpy(x).cuda() for x in xs_h]
    outs = [torch.empty_like(x) for x in xs]
    plans = [fftu.Plan(s, None, inverse=inverse) for s in shapes]
    b = fftu.fftu_batch_create([q.handle for q in plans])
    try:
        fftu.fftu_batch_exec(b, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs],
                             torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        fftu.fftu_batch_check_status(b)
    finally:
        fftu.fftu_batch_destroy(b)
        for q in plans:
            q.close()
    worst = 0.0
    for i, (x, o) in enumerate(zip(xs_h, outs)):
        err, emax = errors(o.cpu().numpy(), oracle.fftn(x, inverse=inverse))
        worst = max(worst, err)
        assert err <= tolerance(np.complex64, x.size), (i, shapes[i], err)
        assert emax <= tolerance(np.complex64, x.size), (i, shapes[i], emax)
    print(f"batch of 64 uneven ({'inverse' if inverse else 'forward'}): worst relative L2 {worst:.3e}")
