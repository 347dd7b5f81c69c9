"""The wisdom table of the plan-time tuner: text format round trip, merge and clear.
These entry points touch no GPU, so they run on the CPU."""
import pytest


@pytest.fixture(scope="module")
def fftu():
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as f
    return f


def test_wisdom_round_trip(fftu, tmp_path):
    src = tmp_path / "in.txt"
    src.write_text("fftu-wisdom-v1 3:512,512,512:1:-1:0:NVIDIA_GB300 8,8,8\n"
                   "some-other-tool ignored 1\n"
                   "fftu-wisdom-v1 2:16384,16384:2:1:0:NVIDIA_GB300 4,16\n")
    fftu.fftu_wisdom_forget()
    fftu.fftu_wisdom_import(str(src))
    dst = tmp_path / "out.txt"
    fftu.fftu_wisdom_export(str(dst))
    lines = sorted(dst.read_text().splitlines())
    assert lines == ["fftu-wisdom-v1 2:16384,16384:2:1:0:NVIDIA_GB300 4,16",
                     "fftu-wisdom-v1 3:512,512,512:1:-1:0:NVIDIA_GB300 8,8,8"]
    # a later import of the same key replaces the grid
    src.write_text("fftu-wisdom-v1 3:512,512,512:1:-1:0:NVIDIA_GB300 4,4,4\n")
    fftu.fftu_wisdom_import(str(src))
    fftu.fftu_wisdom_export(str(dst))
    assert "fftu-wisdom-v1 3:512,512,512:1:-1:0:NVIDIA_GB300 4,4,4" in dst.read_text().splitlines()
    fftu.fftu_wisdom_forget()
    fftu.fftu_wisdom_export(str(dst))
    assert dst.read_text() == ""


def test_wisdom_missing_file(fftu, tmp_path):
    with pytest.raises(fftu.FFTUError):
        fftu.fftu_wisdom_import(str(tmp_path / "does-not-exist.txt"))
