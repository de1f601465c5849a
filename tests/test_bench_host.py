"""Host logic of bench.py that needs no GPU: the clock record taken from
nvidia-smi lines, the issue-rate roofline arithmetic, and the rule that a
committed DRAM-traffic or instruction record only counts while the LBM
kernel sources are the ones it was measured on."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _FakeProc:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_record_from_nvidia_smi_lines():
    lines = "\n".join([
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ])
    s = bench.ClockSampler(0)
    s.proc = _FakeProc(lines)
    rec = s.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_record_flags_thermal_slowdown():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc("0, 1500, 2070, 900.0, 0x40, Not Active, Active, Not Active, Not Active")
    assert s.stop()["reasons"] == ["hw_thermal_slowdown"]


def test_no_samples_give_no_record():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc("")
    assert s.stop() is None
    assert bench.ClockSampler(0).stop() is None          # nvidia-smi never started


def test_issue_rate_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "recorded_instructions", lambda kernel: 24.0)
    r = bench.alu_roofline("k", cells=1_000_000, ms=1.0, clocks={"sm_mhz": 2000.0}, sms=152)
    # 24 warp instructions per cell x 1e6 cells in 1 ms, against 152 SMs x 4 schedulers x 2 GHz
    assert r["achieved"] == pytest.approx(24e6 / 1e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 4 * 2000e6 / 1e12)
    assert r["frac"] == pytest.approx((24e6 / 1e-3) / (152 * 4 * 2000e6))
    # the SM count is the device's, not a constant
    r2 = bench.alu_roofline("k", cells=1_000_000, ms=1.0, clocks={"sm_mhz": 2000.0}, sms=76)
    assert r2["frac"] == pytest.approx(2 * r["frac"])
    assert bench.alu_roofline("k", 1, 1.0, None, 152) is None
    monkeypatch.setattr(bench, "recorded_instructions", lambda kernel: None)
    assert bench.alu_roofline("k", 1, 1.0, {"sm_mhz": 2000.0}, 152) is None


def test_epilogue_schedule_counts():
    """The label names the snapshots and mean samples the timed window takes."""
    sch = bench.schedule(20, 3)
    assert sch["snap_count"] == 1 and sch["snap_first"] == 3 + 20 - 1
    c = bench.epilogue_counts(sch, 3, 20)
    assert c == {"snapshots": 1, "mean_samples": 2, "force_rows": 20}
    sch = bench.schedule(500, 10)
    c = bench.epilogue_counts(sch, 10, 500)
    assert c == {"snapshots": 20, "mean_samples": 50, "force_rows": 500}


def _fake_tree(root, source):
    csrc = root / "paper_2606_16765_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "lbm_step.cuh").write_text(source)
    (csrc / "fno.cu").write_text("not an LBM source")
    (root / "profiles").mkdir()


def test_records_count_only_for_the_sources_they_were_measured_on(tmp_path, monkeypatch):
    _fake_tree(tmp_path, "kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        [{"kernel": "k", "workload": "w", "source_hash": h, "bytes_per_launch": 123}]))
    (tmp_path / "profiles" / "alu.json").write_text(json.dumps(
        [{"kernel": "k", "source_hash": h, "warp_instructions_per_cell": 7.5}]))
    assert bench.recorded_traffic("k", "w") == 123
    assert bench.recorded_traffic("k", "other workload") is None
    assert bench.recorded_instructions("k") == 7.5
    # an FNO source does not enter the hash; an LBM source does
    (tmp_path / "paper_2606_16765_gb300" / "csrc" / "fno.cu").write_text("changed")
    assert bench.kernel_source_hash() == h
    (tmp_path / "paper_2606_16765_gb300" / "csrc" / "lbm_step.cuh").write_text("kernel v2")
    assert bench.kernel_source_hash() != h
    assert bench.recorded_traffic("k", "w") is None
    assert bench.recorded_instructions("k") is None


def test_committed_records_are_well_formed():
    root = os.path.dirname(bench.__file__)
    for name, keys in (("traffic.json", {"kernel", "workload", "source_hash", "bytes_per_launch"}),
                       ("alu.json", {"kernel", "source_hash", "warp_instructions_per_cell"})):
        recs = json.load(open(os.path.join(root, "profiles", name)))
        assert recs and all(keys <= set(r) for r in recs)
