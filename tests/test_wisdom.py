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


def test_wisdom_import_skips_invalid_lines(fftu, tmp_path):
    """A wisdom file comes from outside the process: lines whose key or choices no plan would accept
    are dropped on import, so they can never reach a plan."""
    good = "fftu-wisdom-v2 3:64,64,64:1:-1:0:0:NVIDIA_GB300 2,4,2 3 2048 16"
    bad = [
        "fftu-wisdom-v2 3:64,64,64:1:-1:0:0:G 16,2,2 0 0 0",          # 16^2 does not divide 64
        "fftu-wisdom-v2 3:64,64,64:1:-1:0:0:G 0,1,1 0 0 0",           # p_l < 1
        "fftu-wisdom-v2 3:64,64,64:1:-1:0:0:G 2,2 0 0 0",             # grid of the wrong length
        "fftu-wisdom-v2 2:48,64:1:-1:0:0:G 1,2 0 0 0",                # n_l not a power of two
        "fftu-wisdom-v2 3:64,64,64:1:-1:0:0:G 2,2,2 0 12345 0",       # tile not a power of two
        "fftu-wisdom-v2 3:64,64,64:2:-1:0:0:G 2,2,2 0 8192 0",        # tile above the complex128 limit
        "fftu-wisdom-v2 3:64,64,64:1:-1:0:0:G 2,2,2 0 0 4",           # radix
        "fftu-wisdom-v2 3:64,64,64:1:-1:0:0:G 2,2,2 9 0 0",           # schedule
        "fftu-wisdom-v2 1:1099511627776:1:-1:0:0:G 549755813888 0 0 0",  # p^2 > n (would overflow)
        "fftu-wisdom-v2 3:64,64:1:-1:0:0:G 2,2,2 0 0 0",              # key: d = 3 with two n_l
        "fftu-wisdom-v2 3:64,64,64:3:-1:0:0:G 2,2,2 0 0 0",           # dtype
        "fftu-wisdom-v2 3:64,64,64:1:0:0:0:G 2,2,2 0 0 0",            # direction
        "fftu-wisdom-v2 3:64,64,64:1:-1:0:7:G 2,2,2 0 0 0",           # precision
        "fftu-wisdom-v2 3:64,64,64:1:-1:0:0 2,2,2 0 0 0",             # key without the GPU field
        "fftu-wisdom-v1 2:16384,16384:1:1:0:G 4,256",                  # v1 line with 256^2 not dividing
    ]
    src = tmp_path / "mixed.txt"
    src.write_text("\n".join(bad[:7] + [good] + bad[7:]) + "\n")
    fftu.fftu_wisdom_forget()
    fftu.fftu_wisdom_import(str(src))
    dst = tmp_path / "out.txt"
    fftu.fftu_wisdom_export(str(dst))
    assert dst.read_text().splitlines() == [good]
    fftu.fftu_wisdom_forget()
