"""The wisdom table of the plan-time tuner: text format round trip, merge, the older v1 format,
and clear.  These entry points touch no GPU, so they run on the CPU."""
import pytest


@pytest.fixture(scope="module")
def fftu():
    from paper_2203_11795_gb300 import _build
    _build.build()
    import paper_2203_11795_gb300 as f
    return f


def test_wisdom_round_trip(fftu, tmp_path):
    src = tmp_path / "in.txt"
    src.write_text("fftu-wisdom-v2 3:512,512,512:1:-1:0:0:NVIDIA_GB300 8,8,8 0 0 0\n"
                   "some-other-tool ignored 1\n"
                   "fftu-wisdom-v2 2:16384,16384:1:1:0:0:NVIDIA_GB300 8,8 3 8192 16\n")
    fftu.fftu_wisdom_forget()
    fftu.fftu_wisdom_import(str(src))
    dst = tmp_path / "out.txt"
    fftu.fftu_wisdom_export(str(dst))
    lines = sorted(dst.read_text().splitlines())
    assert lines == ["fftu-wisdom-v2 2:16384,16384:1:1:0:0:NVIDIA_GB300 8,8 3 8192 16",
                     "fftu-wisdom-v2 3:512,512,512:1:-1:0:0:NVIDIA_GB300 8,8,8 0 0 0"]
    # a later import of the same key replaces the entry
    src.write_text("fftu-wisdom-v2 3:512,512,512:1:-1:0:0:NVIDIA_GB300 4,4,4 1 2048 8\n")
    fftu.fftu_wisdom_import(str(src))
    fftu.fftu_wisdom_export(str(dst))
    assert "fftu-wisdom-v2 3:512,512,512:1:-1:0:0:NVIDIA_GB300 4,4,4 1 2048 8" in dst.read_text().splitlines()
    fftu.fftu_wisdom_forget()
    fftu.fftu_wisdom_export(str(dst))
    assert dst.read_text() == ""


def test_wisdom_v1_lines(fftu, tmp_path):
    """v1 lines (grid only, no precision field in the key) import as precision 0, other choices open."""
    src = tmp_path / "v1.txt"
    src.write_text("fftu-wisdom-v1 2:16384,16384:2:1:0:NVIDIA_GB300 4,16\n")
    fftu.fftu_wisdom_forget()
    fftu.fftu_wisdom_import(str(src))
    dst = tmp_path / "out.txt"
    fftu.fftu_wisdom_export(str(dst))
    assert dst.read_text().splitlines() == ["fftu-wisdom-v2 2:16384,16384:2:1:0:0:NVIDIA_GB300 4,16 0 0 0"]
    fftu.fftu_wisdom_forget()


def test_wisdom_missing_file(fftu, tmp_path):
    with pytest.raises(fftu.FFTUError):
        fftu.fftu_wisdom_import(str(tmp_path / "does-not-exist.txt"))
