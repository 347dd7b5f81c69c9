"""Host-side parts of bench.py on CPU: the reference arm's JSON line, the clock record's parsing,
the DRAM-traffic lookup keyed by source hash, and the workload helpers."""
import hashlib
import io
import json
import os
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(argv):
    old = sys.argv
    sys.argv = ["bench.py"] + argv
    try:
        return bench.parse_args()
    finally:
        sys.argv = old


def test_warmup_floor_and_defaults():
    a = _args(["--warmup", "0", "--steps", "2"])
    assert a.warmup == 3 and a.steps == 2 and a.gpus == 1
    assert bench.shape_of(a.shape) == (512, 512, 512) and bench.shape_of(a.p) == (8, 8, 8)


def test_reference_arm_line(monkeypatch):
    """--impl reference times the oracle and prints the contract's line (impl, cpu_baseline, e2e)."""
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    a = _args(["--impl", "reference", "--steps", "1", "--warmup", "3", "--shape", "16,16,16", "--p", "2,2,2"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(a)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    # the same workload and config keys the GPU arm reports for these arguments, the whole array per step
    assert line["config"] == bench.workload_config((16, 16, 16), [2, 2, 2], 8, a, 1)
    assert line["same_workload_per_step"] is True
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["higher_is_better"] is True
    assert line["metric"] == bench.METRIC and line["steps"] == 1 and line["warmup"] == 3
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # value = the sample's 4 N 8 bytes per transform, two transforms per step, over the step time
    assert line["value"] == pytest.approx(2 * 4 * 16 ** 3 * 8 / (line["ms_per_step"] * 1e-3) / 1e9)


def test_reference_arm_other_ranks_print_nothing(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    a = _args(["--impl", "reference", "--shape", "16,16,16", "--p", "2,2,2"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(a)
    assert buf.getvalue() == ""


def test_reference_arm_subsamples_beyond_its_budget(monkeypatch):
    """A workload whose warm-up plus timed steps would overrun the budget is timed on a sub-sample."""
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(bench, "REF_BUDGET_S", 1e-9)
    a = _args(["--impl", "reference", "--steps", "1", "--warmup", "3", "--shape", "64,64,64", "--p", "2,2,2"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(a)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["same_workload_per_step"] is False and "sub-sample" in line["cpu_baseline"]["sample"]
    assert line["config"]["shape"] == [64, 64, 64]


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_parsing(tmp_path):
    """Median SM clock, max clock and the throttle reasons seen active in any sample."""
    s = bench.ClockSampler(0)
    s.out = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 600.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    with open(s.out, "w") as f:
        f.write("\n".join(rows) + "\n")
    s.proc = _Done()
    rec = s.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["power_w_max"] == 1390.0 and rec["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(s.out)


def test_clock_record_flags_hardware_slowdown(tmp_path):
    s = bench.ClockSampler(0)
    s.out = str(tmp_path / "clocks.csv")
    with open(s.out, "w") as f:
        f.write("0, 1200, 2070, 900.0, 0x8, Active, Not Active, Active, Not Active\n")
    s.proc = _Done()
    assert s.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    """roofline.traffic is reported only while the profiled kernel source is unchanged."""
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    table = {"phase_a_x": {"bytes_per_launch": 123.0, "source": "kernel.cu", "source_sha": sha}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(table))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("phase_a_x") == 123.0
    assert bench.traffic_for("phase_b_x") is None
    src.write_text("// kernel v2\n")
    assert bench.traffic_for("phase_a_x") is None


def test_committed_traffic_entries_name_existing_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        table = json.load(f)
    for key, ent in table.items():
        assert os.path.exists(os.path.join(ROOT, ent["source"])), key
        assert ent["bytes_per_launch"] == pytest.approx(ent["read"] + ent["write"])
        assert ent["algorithmic_bytes"] == 2 * 512 ** 3 * 8
        assert "--clock-control none" in ent["command"]


def test_workload_helpers():
    assert bench.alg_bytes((512, 512, 512), 8) == 4 * 2 ** 27 * 8
    a = bench.uneven_shapes(64, 7)
    assert a == bench.uneven_shapes(64, 7) and len(a) == 64
    assert all(len(s) == 3 and set(s) <= {32, 64, 128} for s in a)
    c = bench.uneven_shapes(16, 7, cubes=True)
    assert all(s[0] == s[1] == s[2] for s in c)
    assert bench.whole_job_value(bytes_per_rank=4e9, ms=2.0, world=4) == pytest.approx(8000.0)
