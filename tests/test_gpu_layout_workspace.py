"""The CYCLIC storage layout (fftu_options.layout) and caller-supplied workspaces
(fftu_workspace_size / fftu_set_workspace) on the GPU, against the FP64 oracle and, bit for bit,
against the NATURAL-layout plan-owned path they wrap."""
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


def to_cyclic(x, p):
    """Processor-major concatenation of the local arrays X^{(s)}[r] = x[s + r p] (Sec. 1.1)."""
    n = x.shape
    split = []
    for l in range(len(n)):
        split += [n[l] // p[l], p[l]]
    order = [2 * l + 1 for l in range(len(n))] + [2 * l for l in range(len(n))]
    return np.ascontiguousarray(x.reshape(split).transpose(order)).reshape(n)


def tol(x):
    return 1e-12 if x.dtype == np.complex128 else 1e-5 * max(1.0, math.log2(x.size))


CASES = [((16, 16, 16), (2, 2, 2), np.complex64),
         ((64, 32), (4, 2), np.complex64),
         ((64, 64, 64), (2, 2, 2), np.complex128),
         ((32768,), (128,), np.complex64),       # long lines: phase A alternates with the workspace
         ((512, 512, 512), (8, 8, 8), np.complex64)]   # the ring schedule


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
@pytest.mark.parametrize("inverse", [False, True], ids=["fwd", "inv"])
def test_cyclic_layout(fftu, case, inverse):
    import torch
    shape, p, dt = case
    x = complex_uniform(77, shape, dtype=dt)
    xn = torch.from_numpy(x).cuda()
    xc = torch.from_numpy(to_cyclic(x, p)).cuda()
    with fftu.Plan(shape, p, dtype=xn.dtype, inverse=inverse) as nat, \
            fftu.Plan(shape, p, dtype=xn.dtype, inverse=inverse, layout=fftu.FFTU_LAYOUT_CYCLIC) as cyc:
        assert cyc.info["layout"] == fftu.FFTU_LAYOUT_CYCLIC
        assert cyc.info["workspace_need"] >= x.nbytes
        yn = nat.exec(xn)
        yc = cyc.exec(xc)
        inplace = xc.clone()
        cyc.exec(inplace, inplace)
        # phases alone: W and V in CYCLIC layout
        wn = torch.empty_like(xn)
        nat.exec_phase(fftu.FFTU_PHASE_A, xn, wn)
        wc = torch.empty_like(xc)
        cyc.exec_phase(fftu.FFTU_PHASE_A, xc, wc)
        wc_b = wc.clone()
        cyc.exec_phase(fftu.FFTU_PHASE_B, None, wc_b)
        torch.cuda.synchronize()
        cyc.check_device_status()
    yn, yc, inplace = yn.cpu().numpy(), yc.cpu().numpy(), inplace.cpu().numpy()
    assert np.array_equal(yc, to_cyclic(yn, p))          # the same kernels on the natural view
    assert np.array_equal(inplace, yc)
    assert np.array_equal(wc.cpu().numpy(), to_cyclic(wn.cpu().numpy(), p))
    assert np.array_equal(wc_b.cpu().numpy(), yc)
    ref = oracle.fftn(x.astype(np.complex128), inverse=inverse)
    assert oracle.rel_l2(yc, to_cyclic(ref, p)) <= tol(x)


@pytest.mark.parametrize("case", [((512, 512, 512), (8, 8, 8)),    # ring: 3 scratch units + counters
                                  ((512, 512, 512), (4, 4, 4)),    # two kernels: N elements
                                  ((32768,), (128,)),              # ping-pong: N elements
                                  ((64, 64, 64), (4, 4, 4))],      # generic in place: none
                         ids=lambda c: "x".join(map(str, c[0])) + "_p" + str(c[1][0]))
def test_caller_workspace(fftu, case):
    import torch
    shape, p = case
    x = torch.from_numpy(complex_uniform(78, shape, dtype=np.complex64)).cuda()
    with fftu.Plan(shape, p) as own, fftu.Plan(shape, p, workspace_mode=fftu.FFTU_WORKSPACE_CALLER) as ext:
        need = fftu.fftu_workspace_size(ext.handle)
        assert need == own.info["workspace_need"] == ext.info["workspace_need"]
        assert ext.info["workspace_bytes"] == 0 and own.info["workspace_bytes"] == need
        y_own = own.exec(x)
        if need > 0:
            with pytest.raises(fftu.FFTUError) as ei:   # no workspace yet
                ext.exec(x)
            assert ei.value.status == 1
            with pytest.raises(fftu.FFTUError):          # too small
                fftu.fftu_set_workspace(ext.handle, x.data_ptr(), need - 1)
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=x.device)
        fftu.fftu_set_workspace(ext.handle, ws.data_ptr(), need)
        y_ext = ext.exec(x)
        # a plan-owned workspace can be swapped for the caller's too
        ws2 = torch.empty(max(need, 1), dtype=torch.uint8, device=x.device)
        fftu.fftu_set_workspace(own.handle, ws2.data_ptr(), need)
        assert own.info["workspace_bytes"] == 0
        y_own2 = own.exec(x)
        torch.cuda.synchronize()
        ext.check_device_status()
        own.check_device_status()
        if need > 0:
            fftu.fftu_set_workspace(ext.handle, None, 0)
            with pytest.raises(fftu.FFTUError):
                ext.exec(x)
    assert torch.equal(y_ext, y_own) and torch.equal(y_own2, y_own)


def test_cyclic_refused_where_unsupported(fftu):
    with fftu.Plan((32, 32, 32), None, layout=fftu.FFTU_LAYOUT_CYCLIC) as c:
        with pytest.raises(fftu.FFTUError) as ei:
            fftu.fftu_batch_create([c.handle])
        assert ei.value.status == 3
