"""Plan-time tuning of the cyclic grid (fftu_options.tune): the chosen grid is a valid
Algorithm 2.3 grid, the tuned plan matches the FP64 oracle, and wisdom is recorded and obeyed."""
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


@pytest.fixture(autouse=True)
def _clean_wisdom(fftu):
    """Wisdom is process-wide and plain plans with p = NULL use it: leave none behind."""
    fftu.fftu_wisdom_forget()
    yield
    fftu.fftu_wisdom_forget()


def _key(shape, dtype_code, direction):
    import torch
    name = torch.cuda.get_device_name(0).replace(" ", "_")
    return f"{len(shape)}:{','.join(str(v) for v in shape)}:{dtype_code}:{direction}:0:0:{name}"


@pytest.mark.parametrize("shape,inverse", [((64, 64, 64), False), ((128, 32), True), ((16, 16, 16, 16), False)])
def test_tuned_plan_is_valid_and_correct(fftu, tmp_path, shape, inverse):
    import torch
    fftu.fftu_wisdom_forget()
    x = complex_uniform(7, shape, dtype=np.complex64)
    t = torch.from_numpy(x).cuda()
    with fftu.Plan(shape, None, dtype=t.dtype, inverse=inverse, tune=True) as plan:
        info = plan.info
        assert info["tuned"] == 1
        for n_l, p_l in zip(shape, info["p"]):
            assert p_l >= 1 and (p_l & (p_l - 1)) == 0 and n_l % (p_l * p_l) == 0
        out = plan.exec(t)
        torch.cuda.synchronize()
        plan.check_device_status()
    ref = oracle.fftn(x.astype(np.complex128), inverse=inverse)
    assert oracle.rel_l2(out.cpu().numpy(), ref) < 1e-5 * math.log2(x.size)
    path = tmp_path / "w.txt"
    fftu.fftu_wisdom_export(str(path))
    code = fftu.FFTU_C64
    direction = fftu.FFTU_INVERSE if inverse else fftu.FFTU_FORWARD
    lines = [ln for ln in path.read_text().splitlines() if ln.split()[1] == _key(shape, code, direction)]
    assert len(lines) == 1
    tag, _, grid, sched, tile, radix = lines[0].split()
    assert tag == "fftu-wisdom-v2" and grid == ",".join(str(v) for v in info["p"])
    assert int(sched) == info["schedule"] or (int(sched) == 0 and info["schedule"] == fftu.FFTU_SCHED_FUSED)
    assert int(tile) in (0, info["tile"]) and int(radix) in (0, info["radix"])


def test_imported_wisdom_is_obeyed(fftu, tmp_path):
    import torch
    shape = (32, 32, 32)
    path = tmp_path / "w.txt"
    path.write_text(f"fftu-wisdom-v2 {_key(shape, fftu.FFTU_C64, fftu.FFTU_FORWARD)} 2,1,4 3 2048 16\n")
    fftu.fftu_wisdom_forget()
    fftu.fftu_wisdom_import(str(path))
    x = complex_uniform(8, shape, dtype=np.complex64)
    t = torch.from_numpy(x).cuda()
    with fftu.Plan(shape, None, dtype=t.dtype, tune=True) as plan:
        info = plan.info
        assert info["p"] == [2, 1, 4] and info["tuned"] == 1
        assert info["schedule"] == fftu.FFTU_SCHED_GENERIC_A and info["tile"] == 2048 and info["radix"] == 16
        out = plan.exec(t)
        torch.cuda.synchronize()
    assert oracle.rel_l2(out.cpu().numpy(), oracle.fftn(x.astype(np.complex128))) < 1e-4
    # a plain plan (no tuning requested) takes the same wisdom
    with fftu.Plan(shape, None, dtype=t.dtype) as plan:
        assert plan.info["p"] == [2, 1, 4] and plan.info["tuned"] == 1
    fftu.fftu_wisdom_forget()


def test_plain_plan_uses_wisdom(fftu, tmp_path):
    """p = NULL without tuning takes the process's wisdom for the problem, else the default grid."""
    import torch
    shape = (64, 64, 64)
    with fftu.Plan(shape, None) as plan:
        assert plan.info["p"] == [8, 8, 8] and plan.info["tuned"] == 0
    path = tmp_path / "w.txt"
    path.write_text(f"fftu-wisdom-v2 {_key(shape, fftu.FFTU_C64, fftu.FFTU_FORWARD)} 4,2,4 0 2048 8\n")
    fftu.fftu_wisdom_import(str(path))
    x = complex_uniform(9, shape, dtype=np.complex64)
    with fftu.Plan(shape, None) as plan:
        info = plan.info
        assert info["p"] == [4, 2, 4] and info["tuned"] == 1 and info["tile"] == 2048
        y = plan.exec(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
    assert oracle.rel_l2(y.cpu().numpy(), oracle.fftn(x.astype(np.complex128))) < 1e-4
    fftu.fftu_wisdom_forget()
    with fftu.Plan(shape, None) as plan:
        assert plan.info["p"] == [8, 8, 8]
