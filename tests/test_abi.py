"""The C-ABI library loads and exports every symbol include/fftu.h declares,
and host-side validation rejects bad plans before touching a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fftu.h")
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11795_gb300 import _build
    _build.build()
    return ctypes.CDLL(_build.LIB)


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fftu_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fftu_plan", "fftu_exec", "fftu_destroy", "fftu_exec_phase", "fftu_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2203_11795_gb300 import _build
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fftu_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    import paper_2203_11795_gb300 as f
    assert set(f.EXPORTS) == set(declared_functions())


def test_status_strings_and_version():
    import paper_2203_11795_gb300 as f
    for code in range(8):
        assert f.fftu_status_string(code).startswith(f.STATUS_NAMES[code])
    assert "sm_103a" in f.fftu_version()


@pytest.mark.parametrize("n,p,code", [
    ([64, 64, 64], [16, 2, 2], 2),   # 16^2 does not divide 64
    ([48, 64], [4, 2], 3),           # 48 is valid for the method but not a power of two
    ([64, 0], [1, 1], 1),            # n_l < 1
    ([64, 64], [0, 1], 1),           # p_l < 1
    ([64, 64], [1 << 32, 1], 2),     # p_l > n_l (p_l^2 would overflow 64 bits)
    ([1 << 40], [1 << 39], 2),       # p_l <= n_l but p_l^2 > n_l (and overflows 64 bits)
])
def test_plan_validation(n, p, code):
    import paper_2203_11795_gb300 as f
    with pytest.raises(f.FFTUError) as ei:
        f.fftu_plan(len(n), n, p, f.FFTU_C64, f.FFTU_FORWARD)
    assert ei.value.status == code
    assert f.fftu_last_error()


def test_bad_dtype_dir_and_d():
    import paper_2203_11795_gb300 as f
    for args in ((0, [8], [1], 1, -1), (9, [2] * 9, [1] * 9, 1, -1), (1, [8], [1], 3, -1), (1, [8], [1], 1, 0)):
        with pytest.raises(f.FFTUError) as ei:
            f.fftu_plan(*args)
        assert ei.value.status == 1  # FFTU_ERR_ARG


def test_server_config_validation():
    """Invalid server configs are refused before any CUDA call; bad handles are reported."""
    import paper_2203_11795_gb300 as f
    for cfg in ({"max_batch": 200}, {"streams": 17}, {"max_batch": -1}, {"max_inflight": 300}, {"copy_piece_mib": -1}):
        with pytest.raises(f.FFTUError) as ei:
            f.fftu_server_create(**cfg)
        assert ei.value.status == 1
    with pytest.raises(f.FFTUError):
        f.fftu_server_drain(None, 0.0)
    with pytest.raises(f.FFTUError):
        f.fftu_server_poll(None, 4)
    f.fftu_server_destroy(None)


def test_precision_option_validation():
    """Unknown precision values are refused before any device work."""
    import paper_2203_11795_gb300 as f
    with pytest.raises(f.FFTUError) as ei:
        f.fftu_plan_ex(3, [64, 64, 64], None, f.FFTU_C64, f.FFTU_FORWARD, precision=7)
    assert ei.value.status == 1
    with pytest.raises(f.FFTUError) as ei:
        f.fftu_plan_ex(3, [64, 64, 64], None, f.FFTU_C64, f.FFTU_FORWARD, schedule=9)
    assert ei.value.status == 1


def test_layout_and_workspace_validation():
    """Unknown layouts and workspace modes are refused before any device work; the workspace
    entry points reject NULL plans."""
    import paper_2203_11795_gb300 as f
    for kw in ({"layout": 5}, {"workspace_mode": 3}):
        with pytest.raises(f.FFTUError) as ei:
            f.fftu_plan_ex(3, [64, 64, 64], None, f.FFTU_C64, f.FFTU_FORWARD, **kw)
        assert ei.value.status == 1
    with pytest.raises(f.FFTUError):
        f.fftu_workspace_size(None)
    with pytest.raises(f.FFTUError):
        f.fftu_set_workspace(None, None, 0)


def test_selftest_limit_validation():
    import paper_2203_11795_gb300 as f
    for bad in (0.0, 5.0, float("nan")):
        with pytest.raises(f.FFTUError) as ei:
            f.fftu_selftest_bounded_wait(bad)
        assert ei.value.status == 1
