"""GPU parity: the CUDA path against the FP64 oracle, element by element.

Every case runs through the C ABI (fftu_plan / fftu_exec / fftu_exec_phase via
the ctypes binding) on seeded inputs from fftu_inputs, and compares with the
oracle on the exact same values (complex64 inputs are promoted exactly).
Tolerance (relative L2 over the whole array): 1e-12 for complex128 and
1e-5 * log2(N) for complex64.
"""
import math

import numpy as np
import pytest

import oracle
from fftu_inputs import complex_uniform
from oracle import cyclic_model as cm

pytestmark = pytest.mark.gpu


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


def run_gpu(f, x, p, inverse=False, schedule=0, inplace=False, phase=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    with f.Plan(x.shape, p, dtype=t.dtype, inverse=inverse, schedule=schedule) as plan:
        out = t if inplace else torch.empty_like(t)
        if phase is None:
            plan.exec(t, out)
        elif phase == f.FFTU_PHASE_B:
            out.copy_(t)
            plan.exec_phase(phase, None, out)
        else:
            plan.exec_phase(phase, t, out)
        torch.cuda.synchronize()
        plan.check_device_status()
        info = plan.info
    return out.cpu().numpy(), info


SMALL = [
    # (shape, p, dtype)
    ((64, 64, 64), (2, 2, 2), np.complex128),      # the 64^3 complex128 workload, p = 2x2x2
    ((8, 8, 8), (2, 2, 2), np.complex64),
    ((16, 16, 16), (4, 2, 1), np.complex64),
    ((32, 64, 16), (4, 8, 2), np.complex64),
    ((64, 64, 64), (4, 4, 4), np.complex64),
    ((64, 64, 64), (8, 8, 8), np.complex64),
    ((128, 32, 256), (8, 4, 16), np.complex64),
    ((128,), (8,), np.complex64),                   # d = 1: Algorithm 2.2
    ((4096,), (64,), np.complex64),                 # p_l > 16: per-axis phase B
    ((256, 256), (16, 16), np.complex64),           # n_l = p_l^2
    ((2, 1024, 8), (1, 16, 2), np.complex64),
    ((16, 8, 4, 4, 2), (2, 2, 2, 2, 1), np.complex64),
    ((8, 8, 8, 8), (2, 2, 2, 2), np.complex128),
    ((16, 16, 16, 16), (4, 4, 4, 4), np.complex128),
    ((1, 1, 64), (1, 1, 8), np.complex64),
    ((2,), (1,), np.complex64),
    ((1,), (1,), np.complex128),
    ((4, 8, 16), (1, 1, 1), np.complex64),          # p = 1: phase B only scales
]


def _id(case):
    shape, p, dt = case
    return "x".join(map(str, shape)) + "_p" + "x".join(map(str, p)) + ("_c128" if dt == np.complex128 else "_c64")


@pytest.mark.parametrize("case", SMALL, ids=_id)
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("schedule", [0, 1])
def test_matches_oracle(fftu, case, inverse, schedule):
    shape, p, dt = case
    x = complex_uniform(1000 + len(shape), shape, dtype=dt)
    y, info = run_gpu(fftu, x, p, inverse=inverse, schedule=schedule)
    ref = oracle.fftn(x.astype(np.complex128), inverse=inverse)
    N = int(np.prod(shape))
    err = oracle.rel_l2(y, ref)
    assert err <= tolerance(dt, N), (err, info)


@pytest.mark.parametrize("case", [((64, 64, 64), (4, 4, 4), np.complex64),
                                  ((32, 16, 8), (2, 2, 2), np.complex128)], ids=_id)
def test_in_place(fftu, case):
    shape, p, dt = case
    x = complex_uniform(77, shape, dtype=dt)
    y, _ = run_gpu(fftu, x, p, inplace=True)
    assert oracle.rel_l2(y, oracle.fftn(x.astype(np.complex128))) <= tolerance(dt, x.size)


@pytest.mark.parametrize("case", [((16, 8, 32), (4, 2, 4), np.complex128),
                                  ((64, 64, 64), (8, 8, 8), np.complex128),
                                  ((64, 16), (8, 2), np.complex64)], ids=_id)
@pytest.mark.parametrize("schedule", [0, 1])
def test_phases_match_model(fftu, case, schedule):
    """Phase A alone = Supersteps 0+1 of the CPU model; phase B alone = Superstep 2."""
    shape, p, dt = case
    x = complex_uniform(88, shape, dtype=dt)
    for inverse in (False, True):
        wa, _ = run_gpu(fftu, x, p, inverse=inverse, schedule=schedule, phase=fftu.FFTU_PHASE_A)
        w_ref = cm.phase_a(x.astype(np.complex128), p, inverse=inverse)
        assert oracle.rel_l2(wa, w_ref) <= tolerance(dt, x.size)
        w_in = w_ref.astype(dt)
        vb, _ = run_gpu(fftu, w_in, p, inverse=inverse, schedule=schedule, phase=fftu.FFTU_PHASE_B)
        v_ref = cm.phase_b(w_in.astype(np.complex128), p, inverse=inverse)
        assert oracle.rel_l2(vb, v_ref) <= tolerance(dt, x.size)


def test_round_trip_and_linearity(fftu):
    import torch
    shape, p = (128, 64, 32), (4, 4, 4)
    x = torch.from_numpy(complex_uniform(5, shape, dtype=np.complex64)).cuda()
    z = torch.from_numpy(complex_uniform(6, shape, dtype=np.complex64)).cuda()
    with fftu.Plan(shape, p) as fwd, fftu.Plan(shape, p, inverse=True) as inv:
        X, Z = fwd.exec(x), fwd.exec(z)
        back = inv.exec(X)
        lin = fwd.exec(2 * x - 3j * z)
        torch.cuda.synchronize()
    tol = tolerance(np.complex64, x.numel())
    assert oracle.rel_l2(back.cpu().numpy(), x.cpu().numpy()) <= tol
    assert oracle.rel_l2(lin.cpu().numpy(), (2 * X - 3j * Z).cpu().numpy()) <= tol


def test_plan_info(fftu):
    with fftu.Plan((64, 64, 64), (4, 4, 4)) as plan:
        info = plan.info
    assert info["N"] == 64 ** 3 and info["alg_bytes"] == 4 * 64 ** 3 * 8
    assert info["p"] == [4, 4, 4] and info["launches_phase_a"] >= 1 and info["launches_phase_b"] >= 1
    assert info["table_bytes"] == 3 * 64 * 8


def test_exec_rejects_bad_pointers(fftu):
    import torch
    with fftu.Plan((16, 16), (2, 2)) as plan:
        t = torch.zeros((16, 16), dtype=torch.complex64, device="cuda")
        with pytest.raises(fftu.FFTUError) as ei:
            fftu.fftu_exec(plan.handle, t.data_ptr() + 8, t.data_ptr(), 0)
        assert ei.value.status == 1
        with pytest.raises(fftu.FFTUError):
            fftu.fftu_exec_phase(plan.handle, fftu.FFTU_PHASE_B, t.data_ptr() + 16, t.data_ptr(), 0)


# ---- full-size workloads ------------------------------------------------------------------

FULL = [((512, 512, 512), (8, 8, 8)), ((512, 512, 512), (4, 4, 4))]


@pytest.mark.parametrize("shape,p", FULL, ids=["512c64_p8", "512c64_p4"])
def test_full_size_512_forward_inverse(fftu, shape, p):
    """512^3 complex64 forward against the full FP64 oracle, inverse by round trip."""
    import torch
    x = complex_uniform(2024, shape, dtype=np.complex64)
    xt = torch.from_numpy(x).cuda()
    with fftu.Plan(shape, p) as fwd, fftu.Plan(shape, p, inverse=True) as inv:
        y = fwd.exec(xt)
        back = inv.exec(y)
        torch.cuda.synchronize()
        fwd.check_device_status()
        inv.check_device_status()
    N = x.size
    ref = oracle.fftn(x.astype(np.complex128))
    yh = y.cpu().numpy()
    err, emax = oracle.rel_l2(yh, ref), oracle.max_abs_rel(yh, ref)
    print(f"{shape} p={p}: relative L2 {err:.3e}, max-abs / max|ref| {emax:.3e}")
    assert err <= tolerance(np.complex64, N)
    assert emax <= tolerance(np.complex64, N)  # the largest outputs carry most of the norm
    del ref
    assert oracle.rel_l2(back.cpu().numpy(), x) <= tolerance(np.complex64, N)


# ---- long lines (a tile holds part of the residue classes of a line) ------------------------

@pytest.mark.parametrize("case", [((32768,), (128,), np.complex64),
                                  ((16384, 16), (128, 4), np.complex64),
                                  ((8, 8192), (2, 64), np.complex128),
                                  # sub-FFT length x vectors above the tile: fewer vectors per tile
                                  ((16384, 64), (8, 4), np.complex64),
                                  ((8192, 32), (4, 2), np.complex128),
                                  ((32768,), (8,), np.complex64)], ids=_id)
@pytest.mark.parametrize("inverse", [False, True])
def test_long_lines(fftu, case, inverse):
    shape, p, dt = case
    x = complex_uniform(515, shape, dtype=dt)
    y, info = run_gpu(fftu, x, p, inverse=inverse)
    assert info["workspace_bytes"] == x.size * x.itemsize  # phase A alternates with a workspace
    assert oracle.rel_l2(y, oracle.fftn(x.astype(np.complex128), inverse=inverse)) <= tolerance(dt, x.size)


# ---- register-resident line passes (phase-A sub-FFTs of 256 ... 2048 points, complex64) ----------

LINE_CASES = [
    ((512, 512), (2, 2), np.complex64),          # len 256 on both axes: 16 lines per CTA
    ((1024, 64), (2, 4), np.complex64),          # len 512 on a strided axis (8 inner positions per CTA)
    ((64, 4096), (4, 4), np.complex64),          # len 1024 on the contiguous axis (4 classes per CTA)
    ((8192, 8), (4, 2), np.complex64),           # len 2048 on a strided axis
    ((4, 16384), (1, 16), np.complex64),         # len 1024, 16 classes of a 16384-point line
    ((256, 8, 1024), (1, 2, 4), np.complex64),   # three passes: one strided-pass axis, one line pass
    ((512, 4, 512), (2, 2, 2), np.complex64),    # three passes, two of them line passes
]


@pytest.mark.parametrize("case", LINE_CASES, ids=_id)
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("inplace", [False, True])
def test_line_passes_match_oracle(fftu, case, inverse, inplace):
    """Plans whose phase A runs sub-FFTs of 256 to 2048 points in registers (line_pass.cu), forward and
    inverse, in and out of place (in place with an odd number of passes runs the first one in its
    strided form), against the oracle; out of place leaves the input untouched."""
    import torch
    shape, p, dt = case
    x = complex_uniform(4242 + len(shape), shape, dtype=dt)
    t = torch.from_numpy(x).cuda()
    with fftu.Plan(shape, p, dtype=t.dtype, inverse=inverse) as plan:
        assert plan.info["workspace_bytes"] == x.size * x.itemsize  # phase A alternates with a workspace
        out = t if inplace else torch.empty_like(t)
        plan.exec(t, out)
        torch.cuda.synchronize()
        plan.check_device_status()
        y = out.cpu().numpy()
        if not inplace:
            assert np.array_equal(t.cpu().numpy(), x)
    ref = oracle.fftn(x.astype(np.complex128), inverse=inverse)
    assert oracle.rel_l2(y, ref) <= tolerance(dt, x.size)


@pytest.mark.parametrize("case", LINE_CASES[:4], ids=_id)
def test_line_pass_phase_a_matches_model(fftu, case):
    """Phase A alone through line passes = Supersteps 0 + 1 of the CPU model of Algorithm 2.3."""
    shape, p, dt = case
    x = complex_uniform(4343, shape, dtype=dt)
    for inverse in (False, True):
        wa, _ = run_gpu(fftu, x, p, inverse=inverse, phase=fftu.FFTU_PHASE_A)
        w_ref = cm.phase_a(x.astype(np.complex128), p, inverse=inverse)
        assert oracle.rel_l2(wa, w_ref) <= tolerance(dt, x.size)


# ---- two-axis pair passes (phase A of two adjacent axes with 8- or 16-point sub-FFTs, complex64) -------

PAIR_CASES = [
    ((64, 32, 32), (4, 4, 4), np.complex64),          # contiguous pair (4 planes per CTA), then one axis
    ((32, 32, 16), (4, 4, 2), np.complex64),          # one axis, then a strided pair (8 inner positions)
    ((64, 64), (8, 8), np.complex64),                 # one pair step only (p_a p_b = 64, 512 threads)
    ((2, 64, 64, 4), (1, 4, 4, 2), np.complex64),     # 16-point pair in the middle, three steps
    ((2, 32, 32, 32, 32), (1, 4, 4, 4, 4), np.complex64),  # two pairs and one axis (the 32^5 layout)
    ((32, 32, 32, 32), (4, 4, 4, 4), np.complex64),   # two pairs
]


@pytest.mark.parametrize("case", PAIR_CASES, ids=_id)
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("inplace", [False, True])
def test_pair_passes_match_oracle(fftu, case, inverse, inplace):
    """Plans whose phase A runs two adjacent axes per pass (pair_pass.cu), forward and inverse, in and out
    of place (in place with an odd number of steps runs the first one as two strided passes), against the
    oracle; out of place leaves the input untouched."""
    import torch
    shape, p, dt = case
    x = complex_uniform(5151 + len(shape), shape, dtype=dt)
    t = torch.from_numpy(x).cuda()
    with fftu.Plan(shape, p, dtype=t.dtype, inverse=inverse) as plan:
        assert plan.info["workspace_bytes"] == x.size * x.itemsize  # phase A alternates with a workspace
        out = t if inplace else torch.empty_like(t)
        plan.exec(t, out)
        torch.cuda.synchronize()
        plan.check_device_status()
        y = out.cpu().numpy()
        if not inplace:
            assert np.array_equal(t.cpu().numpy(), x)
    ref = oracle.fftn(x.astype(np.complex128), inverse=inverse)
    assert oracle.rel_l2(y, ref) <= tolerance(dt, x.size)


@pytest.mark.parametrize("case", PAIR_CASES[:4], ids=_id)
def test_pair_pass_phase_a_matches_model(fftu, case):
    """Phase A alone through pair passes = Supersteps 0 + 1 of the CPU model of Algorithm 2.3."""
    shape, p, dt = case
    x = complex_uniform(5252, shape, dtype=dt)
    for inverse in (False, True):
        wa, _ = run_gpu(fftu, x, p, inverse=inverse, phase=fftu.FFTU_PHASE_A)
        w_ref = cm.phase_a(x.astype(np.complex128), p, inverse=inverse)
        assert oracle.rel_l2(wa, w_ref) <= tolerance(dt, x.size)


# ---- three-axis passes (phase A of the last three axes with 8-point sub-FFTs, p_b p_c = 16) -----------

TRIPLE_CASES = [
    ((32, 32, 32), (4, 4, 4), np.complex64),              # one triple step only
    ((2, 32, 32, 32), (1, 4, 4, 4), np.complex64),        # triple, then one axis
    ((64, 16, 64), (8, 2, 8), np.complex64),              # p_b x p_c = 2 x 8
    ((16, 16, 64), (2, 2, 8), np.complex64),              # p_a = 2
    ((2, 32, 32, 32, 32), (1, 4, 4, 4, 4), np.complex64),  # triple and two axes (three steps)
    ((32, 32, 32, 32, 8), (4, 4, 4, 2, 1), np.complex64),  # no triple (p_c = 1): pairs and axes
]


@pytest.mark.parametrize("case", TRIPLE_CASES, ids=_id)
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("inplace", [False, True])
def test_triple_passes_match_oracle(fftu, case, inverse, inplace):
    """Plans whose phase A runs the last three axes in one pass (triple_pass.cu), forward and inverse, in and
    out of place (in place with an odd number of steps runs the first one as its strided passes), against
    the oracle; out of place leaves the input untouched."""
    import torch
    shape, p, dt = case
    x = complex_uniform(6161 + len(shape), shape, dtype=dt)
    t = torch.from_numpy(x).cuda()
    with fftu.Plan(shape, p, dtype=t.dtype, inverse=inverse) as plan:
        out = t if inplace else torch.empty_like(t)
        plan.exec(t, out)
        torch.cuda.synchronize()
        plan.check_device_status()
        y = out.cpu().numpy()
        if not inplace:
            assert np.array_equal(t.cpu().numpy(), x)
    ref = oracle.fftn(x.astype(np.complex128), inverse=inverse)
    assert oracle.rel_l2(y, ref) <= tolerance(dt, x.size)


@pytest.mark.parametrize("case", TRIPLE_CASES[:4], ids=_id)
def test_triple_pass_phase_a_matches_model(fftu, case):
    """Phase A alone through a three-axis pass = Supersteps 0 + 1 of the CPU model of Algorithm 2.3."""
    shape, p, dt = case
    x = complex_uniform(6262, shape, dtype=dt)
    for inverse in (False, True):
        wa, _ = run_gpu(fftu, x, p, inverse=inverse, phase=fftu.FFTU_PHASE_A)
        w_ref = cm.phase_a(x.astype(np.complex128), p, inverse=inverse)
        assert oracle.rel_l2(wa, w_ref) <= tolerance(dt, x.size)


@pytest.mark.parametrize("p", [(128, 128), (8, 8)], ids=["p128", "p8"])
def test_full_size_2d_16384(fftu, p):
    """The 2D 16384 x 16384 complex64 workload against the full FP64 oracle."""
    shape = (16384, 16384)
    x = complex_uniform(2025, shape, dtype=np.complex64)
    y, _ = run_gpu(fftu, x, p)
    ref = oracle.fftn(x.astype(np.complex128))
    err, emax = oracle.rel_l2(y, ref), oracle.max_abs_rel(y, ref)
    print(f"{shape} p={p}: relative L2 {err:.3e}, max-abs / max|ref| {emax:.3e}")
    assert err <= tolerance(np.complex64, x.size)
    assert emax <= tolerance(np.complex64, x.size)


# 1024^3 complex64 at every grid, 64^4, 32^5, the tuned 16384^2 plan and the 64-transform batch are
# compared with the oracle over the whole array in test_gpu_full_size.py.


# ---- forward, pointwise product, inverse (no reordering in between) --------------------------

@pytest.mark.parametrize("case", [((64, 64, 64), (4, 4, 4), np.complex64),      # product fused in phase B
                                  ((512, 512, 512), (8, 8, 8), np.complex64),   # ring phase A + fused product
                                  ((256, 256, 256), (16, 16, 8), np.complex64),  # product in the 16x16x8 phase B
                                  ((32, 16, 8), (2, 2, 2), np.complex128),      # separate product pass
                                  ((256, 128), (4, 8), np.complex64)], ids=_id)
@pytest.mark.parametrize("tmp_is_in", [False, True])
def test_pointwise_convolution(fftu, case, tmp_is_in):
    import torch
    shape, p, dt = case
    x = complex_uniform(909, shape, dtype=dt)
    m = complex_uniform(910, shape, dtype=dt)
    xt, mt = torch.from_numpy(x).cuda(), torch.from_numpy(m).cuda()
    with fftu.Plan(shape, p, dtype=xt.dtype) as fwd, fftu.Plan(shape, p, dtype=xt.dtype, inverse=True) as inv:
        tmp = xt.clone() if tmp_is_in else torch.empty_like(xt)
        src = tmp if tmp_is_in else xt
        out = torch.empty_like(xt)
        fftu.fftu_exec_pointwise(fwd.handle, inv.handle, src.data_ptr(), mt.data_ptr(), tmp.data_ptr(),
                                 out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    x128 = x.astype(np.complex128)
    ref = oracle.fftn(oracle.fftn(x128) * m.astype(np.complex128), inverse=True)
    assert oracle.rel_l2(out.cpu().numpy(), ref) <= tolerance(dt, x.size)


def test_pointwise_rejects_mismatched_plans(fftu):
    import torch
    x = torch.zeros((16, 16), dtype=torch.complex64, device="cuda")
    with fftu.Plan((16, 16), (2, 2)) as fwd, fftu.Plan((16, 16), (4, 2), inverse=True) as inv, \
            fftu.Plan((16, 16), (2, 2)) as fwd2:
        for a, b in ((fwd, inv), (fwd, fwd2)):
            with pytest.raises(fftu.FFTUError) as ei:
                fftu.fftu_exec_pointwise(a.handle, b.handle, x.data_ptr(), x.data_ptr(), x.data_ptr() + 0,
                                         x.data_ptr(), 0)
            assert ei.value.status == 1


# ---- strided-pass tile target and radix (the tuner's other coordinates) -----------------------

@pytest.mark.parametrize("case", [((64, 64, 64), (4, 4, 4), np.complex64),
                                  ((256, 64), (4, 2), np.complex64),
                                  ((32, 32, 32, 32), (2, 2, 2, 2), np.complex128),
                                  ((8192,), (4,), np.complex64),
                                  ((32768,), (128,), np.complex64)], ids=_id)
@pytest.mark.parametrize("tile,radix", [(0, 16), (2048, 8), (8192, 16), (1024, 16)])
@pytest.mark.parametrize("inverse", [False, True])
def test_tile_and_radix_options(fftu, case, tile, radix, inverse):
    import torch
    shape, p, dt = case
    if dt == np.complex128 and tile == 8192:
        pytest.skip("complex128 tiles stop at 4096")
    x = complex_uniform(616, shape, dtype=dt)
    t = torch.from_numpy(x).cuda()
    with fftu.Plan(shape, p, dtype=t.dtype, inverse=inverse, schedule=fftu.FFTU_SCHED_GENERIC, tile=tile,
                   radix=radix) as plan:
        assert plan.info["radix"] == radix and (tile == 0 or plan.info["tile"] == tile)
        y = plan.exec(t)
        torch.cuda.synchronize()
        plan.check_device_status()
    ref = oracle.fftn(x.astype(np.complex128), inverse=inverse)
    assert oracle.rel_l2(y.cpu().numpy(), ref) <= tolerance(dt, x.size)


def test_fused_plan_after_smaller_plan_on_same_kernel(fftu):
    """512^3 and 512 x 256 x 512 (p = 8 x 4 x 8) use the same fused phase-A kernel with different
    shared-memory sizes; making the second plan must not break the first."""
    import torch
    x = complex_uniform(4242, (512, 512, 512), dtype=np.complex64)
    xt = torch.from_numpy(x).cuda()
    with fftu.Plan(x.shape, (8, 8, 8)) as a:
        assert a.info["launches_phase_a"] == 1           # the fused ring kernel
        with fftu.Plan((512, 256, 512), (8, 4, 8)) as b:
            assert b.info["launches_phase_a"] == 1
            yb = b.exec(torch.from_numpy(complex_uniform(4243, (512, 256, 512), dtype=np.complex64)).cuda())
            y = a.exec(xt)
            torch.cuda.synchronize()
            a.check_device_status()
            b.check_device_status()
    idx = [(0, 0, 0), (1, 2, 3), (511, 77, 300), (256, 256, 256)]
    ref = oracle.dft_points(x.astype(np.complex128), idx)
    got = np.array([y[i].item() for i in idx])
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-4


@pytest.mark.parametrize("case", [((256, 128, 512), (4, 2, 8), 1), ((256, 256, 512), (2, 2, 4), 2)],
                         ids=["512rows_p4x2x8_ring", "512rows_p2x2x4_two_kernels"])
def test_fused_phase_a_matches_model(fftu, case):
    """The fused phase A alone (sub-FFTs and twiddle of Superstep 0, Put of Superstep 1) against the
    CPU model, n_0 != n_1 included, both directions, as the persistent ring kernel and as the
    two-kernel schedule (16 and 64 MiB residue units); then phase B alone on the model's W."""
    shape, p, launches = case
    x = complex_uniform(4244, shape, dtype=np.complex64)
    for inverse in (False, True):
        wa, info = run_gpu(fftu, x, p, inverse=inverse, phase=fftu.FFTU_PHASE_A)
        assert info["launches_phase_a"] == launches
        w_ref = cm.phase_a(x.astype(np.complex128), p, inverse=inverse)
        assert oracle.rel_l2(wa, w_ref) <= tolerance(np.complex64, x.size)
        assert oracle.max_abs_rel(wa, w_ref) <= tolerance(np.complex64, x.size)
        w_in = w_ref.astype(np.complex64)
        vb, _ = run_gpu(fftu, w_in, p, inverse=inverse, phase=fftu.FFTU_PHASE_B)
        assert oracle.rel_l2(vb, cm.phase_b(w_in.astype(np.complex128), p, inverse=inverse)) <= \
            tolerance(np.complex64, x.size)


@pytest.mark.parametrize("case", [((256, 256, 1024), (16, 16, 8)), ((256, 256, 256), (16, 16, 16))],
                         ids=lambda c: "x".join(map(str, c[1])))
@pytest.mark.parametrize("inverse", [False, True])
def test_phase_b_16_grids(fftu, case, inverse):
    """Phase B on 16 x 16 x 8 and 16^3 grids (single-element exchange stages) against the full oracle."""
    shape, p = case
    x = complex_uniform(717, shape, dtype=np.complex64)
    y, _ = run_gpu(fftu, x, p, inverse=inverse)
    assert oracle.rel_l2(y, oracle.fftn(x.astype(np.complex128), inverse=inverse)) <= tolerance(np.complex64, x.size)
